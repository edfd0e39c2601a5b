// Internal definitions of libgsr: device layout of a system, float-pair
// arithmetic and launch helpers. Not part of the public ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "gsr.h"

namespace gsr {

constexpr int NSLOT = 24;
constexpr int ROWS_PER_LANE = 4;                 // R consecutive rows per thread
constexpr int TILE_ROWS = 32 * ROWS_PER_LANE;    // rows per warp tile
constexpr int NUM_SMS_B300 = 148;

// ---------------------------------------------------------------------------
// Float-pair ("float-float") arithmetic. A value is hi + lo with |lo| <= ulp(hi)/2.
// The error-free transformations are Knuth's TwoSum and the FMA-based
// TwoProduct (Dekker 1971, Ogita-Rump-Oishi 2005). Every step uses the
// explicitly rounded intrinsics so that no multiply-add is contracted.
// ---------------------------------------------------------------------------
struct ff {
  float h, l;
};

__device__ __forceinline__ ff ff_zero() { return ff{0.0f, 0.0f}; }

// s + e == a + b exactly (TwoSum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float ab = __fsub_rn(s, bb);
  e = __fadd_rn(__fsub_rn(a, ab), __fsub_rn(b, bb));
}

__device__ __forceinline__ ff ff_add(ff a, ff b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  return ff{s, __fadd_rn(__fadd_rn(a.l, b.l), e)};
}

// Product of two pairs to ~2^-47 relative (the lo*lo term is dropped).
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  float c = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e));
  return ff{p, c};
}

// acc += a * b
__device__ __forceinline__ void ff_fma_acc(ff& acc, ff a, ff b) { acc = ff_add(acc, ff_mul(a, b)); }

// Product of an FP32 value with a pair.
__device__ __forceinline__ ff f_mul(float a, ff b) {
  float p = __fmul_rn(a, b.h);
  float e = __fmaf_rn(a, b.h, -p);
  return ff{p, __fmaf_rn(a, b.l, e)};
}

__device__ __forceinline__ ff ff_from_double(double d) {
  float h = __double2float_rn(d);
  float l = __double2float_rn(__dsub_rn(d, (double)h));
  return ff{h, l};
}

__device__ __forceinline__ double ff_to_double(ff a) { return __dadd_rn((double)a.h, (double)a.l); }

__device__ __forceinline__ ff ff_shfl_xor(ff a, int m) {
  return ff{__shfl_xor_sync(0xffffffffu, a.h, m), __shfl_xor_sync(0xffffffffu, a.l, m)};
}
__device__ __forceinline__ ff ff_shfl_up(ff a, int d) {
  return ff{__shfl_up_sync(0xffffffffu, a.h, d), __shfl_up_sync(0xffffffffu, a.l, d)};
}

// Warp all-reduce of a pair (every lane gets the sum).
__device__ __forceinline__ ff ff_warp_sum(ff a) {
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) a = ff_add(a, ff_shfl_xor(a, m));
  return a;
}

__device__ __forceinline__ double warp_sum_d(double a) {
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) a += __shfl_xor_sync(0xffffffffu, a, m);
  return a;
}

// ---------------------------------------------------------------------------
// Device layout of one system (all pointers are device memory owned by it).
// Rows are grouped in warp tiles of TILE_ROWS; lane l of a tile owns rows
// tile*128 + 4l + j (j = 0..3). Row order is the caller's (star-sorted) order.
// ---------------------------------------------------------------------------
struct Layout {
  int64_t n_rows, n_stars, n_knots, n_instr, n_unk;
  int32_t n_glob;
  int64_t n_tiles;
  int64_t att_base, instr_base, glob_col;
  // Values as float pairs: float4 at [((tile*24 + slot)*2 + q)*32 + lane] holds
  // rows 4l+2q, 4l+2q+1 as (hi0, lo0, hi1, lo1). 192 B per row.
  const float4* vals_ff;
  // FP32-rounded values (mixed precision): float2 at [((tile*24+slot)*2+q)*32+lane]
  // holds rows 4l+2q, 4l+2q+1. 96 B per row. Null unless F32_PLUS_F64.
  const float2* vals_f32;
  const int4* star;       // [tile*32 + lane] star index of rows 4l..4l+3
  const int4* att_s;      // [tile*32 + lane] start knot s_i of rows 4l..4l+3
  const int4* att_pos;    // [tile*32 + lane] position of the row in knot order
  const ushort4* instr;   // [(tile*6 + k)*32 + lane] instrumental index k of rows 4l..4l+3
  // Attitude coefficients in knot order (rows sorted by s, stable):
  const float2* att_knot_ff;   // [t][n_rows], t = 4*axis + j
  const float* att_knot_f32;   // [t][n_rows] FP32-rounded copy (or null)
  const int64_t* knot_start;   // [n_knots + 1] first position of start knot s
  const int32_t* att_warp_knot; // [n_att_warps + 1] start-knot range of each attitude warp
  int32_t n_att_warps;
  const int64_t* row_tile_warp; // [n_main_warps + 1] tile range of each star-order warp
  int32_t n_main_warps;
};

struct Scratch {
  double* red;          // partial-sum slots for last-block reductions
  unsigned int* count;  // arrival counters (one per reduction site)
  float2* x_ff;         // [n_unk] float-pair copy of an aprod 1 input
  double* y_knot;       // [n_rows] aprod 2 input in knot order
};

}  // namespace gsr

struct gsr_system {
  int device;
  int num_sms;
  gsr_dims dims;
  gsr::Layout L;
  gsr::Scratch S;
  // owned allocations
  float4* vals_ff;
  float2* vals_f32;
  int4* star;
  int4* att_s;
  int4* att_pos;
  ushort4* instr;
  float2* att_knot_ff;
  float* att_knot_f32;
  int64_t* knot_start;
  int32_t* att_warp_knot;
  int64_t* row_tile_warp;
  double* colnorm;       // [n_unk] ||A_:,j|| (FP64 values)
  // LSQR work vectors (allocated on first solve)
  double* u;             // [n_rows] unnormalised u
  double* u_knot;        // [n_rows] u in knot order
  double* v;             // [n_unk]
  double* w;             // [n_unk]
  double* xz;            // [n_unk] iterate of the scaled problem
  double* z;             // [n_unk] A^T u accumulator
  double* dscale;        // [n_unk] column scaling in use
  float2* v_ff;          // [n_unk] float-pair D v (aprod 1 input)
  double* scal;          // device LSQR scalars
  double* host_scal;     // pinned mirror of scal
  cudaStream_t side;     // second stream for the attitude part of aprod 2
  cudaEvent_t ev_fork, ev_join;
  int main_block, main_ctas, hist_bytes;
};

// Internal entry points shared between translation units.
namespace gsr {
// y = coef*y + A x (coef = *coef_dev if non-null); optional knot-order copy,
// ||y||^2 into *norm_slot; the kernel does nothing when *stop != 0.
int launch_aprod1(gsr_system* sys, int which_values, const float2* x_ff, double* y,
                  const double* coef_dev, double coef_host, double* y_knot, double* norm_slot,
                  const double* stop, cudaStream_t st);
// x += A^T y (y_knot = y in knot order); nothing when *stop != 0.
int launch_aprod2(gsr_system* sys, int which_values, const double* y, const double* y_knot,
                  double* x, const double* stop, cudaStream_t st);
int launch_to_ff(const double* x, const double* scale, float2* out, int64_t n, cudaStream_t st);
int launch_scatter_knot(gsr_system* sys, const double* y, double* y_knot, cudaStream_t st);
int cuda_status(cudaError_t e);
int set_kernel_attributes(int hist_bytes);
}  // namespace gsr
