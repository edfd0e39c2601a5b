// Internal definitions of libgsr: device layout of a system, float-pair
// arithmetic, TMA / mbarrier helpers and launch helpers. Not part of the ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "gsr.h"

namespace gsr {

constexpr int NSLOT = 24;
constexpr int REC_ROWS = 64;        // rows per record; lane l owns rows 2l, 2l+1
constexpr int CT_ROWS_MAX = 2048;   // rows per instrumental tile (at most)
constexpr int NUM_SMS_B300 = 148;
constexpr int MAX_HIST_INSTR = 24576;  // instrumental bins of one block's histogram
constexpr int INSTR_BIN_BITS = 15;     // bin field of an instrumental entry key
constexpr int INSTR_SMEM_BUDGET = 220 * 1024;  // dynamic shared memory of the instr kernel

// One tile buffer of the instrumental kernel: keys (4 B) and coefficients
// (8 B pair / 4 B FP32) of at most max_ent entries and u of the tile's
// ct_rows rows (8 B each), every part rounded up to 16 bytes.
__host__ __device__ constexpr int64_t instr_keys_bytes(int64_t max_ent) {
  return (max_ent * 4 + 15) & ~15LL;
}
__host__ __device__ constexpr int64_t instr_vals_bytes(int64_t max_ent, bool f32) {
  return (max_ent * (f32 ? 4 : 8) + 15) & ~15LL;
}
__host__ __device__ constexpr int64_t instr_tile_bytes(int64_t ct_rows, int64_t max_ent,
                                                       bool f32) {
  return instr_keys_bytes(max_ent) + instr_vals_bytes(max_ent, f32) + ct_rows * 8;
}
// Shared memory of the instrumental kernel: nbuf tile buffers (with two, the
// next tile streams in while the current one is processed) and the float-pair
// histogram of one group of hist_bins columns.
__host__ __device__ constexpr int64_t instr_smem_bytes(int64_t ct_rows, int64_t max_ent,
                                                       int64_t hist_bins, bool f32, int nbuf) {
  return nbuf * instr_tile_bytes(ct_rows, max_ent, f32) + hist_bins * 8;
}
// Two blocks of the instrumental kernel share an SM when each fits this much.
// Row blocks of the blocked knot order of u: as many as keep at least
// KBLK_MIN_PER_KNOT rows per (block, knot) on average, at most KBLK_MAX (the
// attitude kernel walks one segment per block and knot, one block per lane),
// and blocked at all only when that gives at least 2 blocks of at most
// KBLK_MAX_ROWS rows (the slice of u a block scatters into must stay well
// inside L2: 8 B per row).
constexpr int KBLK_MAX = 32;
constexpr int64_t KBLK_MIN_PER_KNOT = 16;
constexpr int64_t KBLK_MAX_ROWS = 1 << 21;
constexpr int INSTR_SMEM_HALF = 112 * 1024;

// ---------------------------------------------------------------------------
// Row records. One record = 64 consecutive rows, everything aprod 1 needs for
// them in one contiguous block (one TMA bulk copy). Per-slot chunks hold the
// two rows of each lane side by side. Byte offsets inside a record:
//   float pairs (REC_FF bytes)            FP32 copy (REC_F32 bytes)
//   slots 0-4       float4[5][32]  0      float2[5][32]   0
//   slot 23 (glob)  float4[32]     2560   float2[32]      1280
//   star            int2[32]       3072                   1536
//   slots 17-22     float4[6][32]  3328   float2[6][32]   1792
//   instr index     ushort2[6][32] 6400                   3328
//   slots 5-16      float4[12][32] 7168   float2[12][32]  4096
//   start knot s    int2[32]       13312                  7168
//   knot position   int2[32]       13568                  7424
// The star-ordered part of aprod 2 reads only the first 3328 (1792) bytes.
// ---------------------------------------------------------------------------
template <bool F32>
struct Rec;

template <>
struct Rec<false> {
  static constexpr int SLOT_BYTES = 512;
  static constexpr int BYTES = 13824;
  static constexpr int ASTRO = 0, GLOB = 2560, STAR = 3072, INSTR_V = 3328, INSTR_I = 6400,
                       ATT_V = 7168, ATT_S = 13312, POS = 13568;
};
template <>
struct Rec<true> {
  static constexpr int SLOT_BYTES = 256;
  static constexpr int BYTES = 7680;
  static constexpr int ASTRO = 0, GLOB = 1280, STAR = 1536, INSTR_V = 1792, INSTR_I = 3328,
                       ATT_V = 4096, ATT_S = 7168, POS = 7424;
};

// Byte offset of slot t's chunk inside a record.
template <bool F32>
__host__ __device__ constexpr int slot_offset(int t) {
  using R = Rec<F32>;
  return t < 5 ? R::ASTRO + t * R::SLOT_BYTES
         : t < 17 ? R::ATT_V + (t - 5) * R::SLOT_BYTES
         : t < 23 ? R::INSTR_V + (t - 17) * R::SLOT_BYTES
                  : R::GLOB;
}

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

// Renormalise a pair (exactly): after cancellation in ff_add the low part can
// be as large as the high part, and products below assume it is not.
__device__ __forceinline__ ff ff_norm(ff a) {
  float s, e;
  two_sum(a.h, a.l, s, e);
  return ff{s, e};
}

// Product of two pairs to ~2^-47 relative (the lo*lo term is dropped; the
// operands must be normalised pairs).
__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  float c = __fmaf_rn(a.h, b.l, __fmaf_rn(a.l, b.h, e));
  return ff{p, c};
}

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

// Exact widening of a float to double with integer instructions and selects
// only (no branch, no FP64 pipe), subnormal floats included: a subnormal is
// first scaled by 2^64 (exact, now normal) and the 64 is taken off the
// double's exponent.
__device__ __forceinline__ double f2d_exact(float f) {
  const uint32_t e0 = (__float_as_uint(f) >> 23) & 0xffu;
  const float g = e0 == 0u ? __fmul_rn(f, 0x1p64f) : f;
  const uint32_t b = __float_as_uint(g);
  const uint32_t s = b & 0x80000000u, e = (b >> 23) & 0xffu, m = b & 0x7fffffu;
  uint32_t ed = e == 0xffu ? 0x7ffu : e + 896u - (e0 == 0u ? 64u : 0u);
  ed = (b & 0x7fffffffu) == 0u ? 0u : ed;  // +-0
  return __hiloint2double((int)(s | (ed << 20) | (m >> 3)), (int)(m << 29));
}

// ---------------------------------------------------------------------------
// Range of the float-pair arithmetic. A pair carries FP32's exponent range, so
// the kernels work on an exactly rescaled problem (powers of two only): the
// stored coefficients are A' = 2^e_i A_ij 2^g_j (row and column exponents
// chosen at creation), and an input vector reaches the float-pair kernels only
// when every nonzero entry of its rescaled form lies in [2^VEC_BAND_LO,
// 2^VEC_BAND_HI). Then every product of a coefficient in [2^-40, 2^40] with a
// vector entry stays within [2^-100, 2^100]: both words of every pair are
// normal FP32 numbers and a product keeps its ~48 bits. Outside the band the
// same call runs FP64 kernels instead (the guard word decides on the device).
// ---------------------------------------------------------------------------
constexpr int MAT_BAND_LO = -40, MAT_BAND_HI = 40;  // ilogb range of coefficients kept as is
constexpr int MAT_WIDE_LO = -100;                   // below this after rescaling: unsupported
constexpr int VEC_BAND_LO = -60, VEC_BAND_HI = 60;  // ilogb range of vector entries

// True when the nonzero finite v (or zero) fits the vector band.
__device__ __forceinline__ bool vec_in_band(double v) {
  const double a = fabs(v);
  return a == 0.0 || (a >= 0x1p-60 && a < 0x1p60);
}

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
// TMA bulk copies (cp.async.bulk) completing on an mbarrier, with bounded
// waits. A wait that runs out sets the error word and returns false.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
// Make mbarrier initialisation and earlier generic shared-memory accesses
// visible to the async (TMA) proxy.
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tma_load(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// The same copy with an L2 eviction-priority policy (createpolicy). Data read
// once per product (the row records) is marked evict-first, so that L2 keeps the
// lines that are reused: gathered unknowns and partly written output sectors.
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ void tma_load_hint(void* dst, const void* src, uint32_t bytes,
                                              uint64_t* bar, uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
      : "memory");
}
// Hint: start moving bytes [src, src + bytes) from DRAM into L2 (no
// completion to wait for; 16-byte aligned address, size a multiple of 16).
__device__ __forceinline__ void prefetch_l2(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Record an error code in the system's error word. The word lives in mapped
// pinned host memory (the host reads it at the next call without a
// synchronisation), so a plain volatile store is used: every writer stores the
// same code, and atomics on host memory are not available everywhere.
__device__ __forceinline__ void set_error(int* err, int code) {
  *reinterpret_cast<volatile int*>(err) = code;
  __threadfence_system();
}
constexpr int WAIT_LIMIT = 1 << 22;  // try_wait rounds before giving up (seconds)
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err) {
  for (int i = 0; i < WAIT_LIMIT; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  if (err) set_error(err, GSR_E_TIMEOUT);
  return false;
}

// ---------------------------------------------------------------------------
// Device layout of one system (all pointers are device memory owned by it).
// ---------------------------------------------------------------------------
struct Layout {
  int64_t n_rows, n_stars, n_knots, n_instr, n_unk;
  int32_t n_glob;
  int64_t n_recs;                       // 64-row records (last one padded)
  int64_t att_base, instr_base, glob_col;
  const unsigned char* rec_ff;          // n_recs x Rec<false>::BYTES
  const unsigned char* rec_f32;         // n_recs x Rec<true>::BYTES, or null
  // Knot order: rows sorted by start knot s, stably (the rows of a knot in row
  // order); the attitude coefficients and the FP32-phase copies of u use it
  // (position gpos). When n_kblk > 1 the float-pair copy of u is blocked
  // instead (position pos): the rows are cut into n_kblk blocks of kblk_rows
  // consecutive rows and sorted by s inside each block, so that aprod 1, which
  // walks the rows in order, scatters u into one block's slice at a time (a
  // slice L2 holds while its sectors fill). Inside knot s the two orders agree:
  // the rows of s in block 0, then block 1, ...
  const int32_t* pos;                   // [n_rows] position of each row in the float-pair
                                        // copy of u (blocked when n_kblk > 1)
  const int32_t* gpos;                  // [n_rows] position in the knot order (== pos when
                                        // n_kblk == 1)
  const float2* att_knot_ff;            // [t][n_rows] in the knot order, t = 4*axis + j
  const float* att_knot_f32;            // [t][n_rows] FP32 copy (or null)
  const int32_t* kb_start;              // [n_kblk][n_knots - 2] first blocked position of
                                        // start knot s in block b (entry n_knots - 3: the
                                        // block's end); null when n_kblk == 1
  int32_t n_kblk;                       // row blocks (1: not blocked; at most KBLK_MAX)
  int64_t kblk_rows;                    // rows per block (a multiple of 64)
  const int64_t* knot_start;            // [n_knots - 3 + 1] first position of start knot s
                                        // in the knot order (rows with start knot < s)
  const int32_t* att_warp_knot;         // [n_att_warps + 1] start-knot range of each warp
  int32_t n_att_warps;
  // instrumental entries of each tile of ct_rows rows, in rounds of distinct bins
  int64_t n_ctiles;
  int32_t ct_rows;                      // power of two in [64, 2048]
  int32_t n_bgroups;                    // instrumental columns split into groups of
  int32_t bgroup_bins;                  // bgroup_bins; a block owns one group's histogram
  int32_t ct_max_ent;                   // most entries of one (tile, group) segment
  int32_t ct_bufs;                      // tile buffers per block (2: double-buffered)
  int32_t ct_per_sm;                    // blocks per SM: 2 (256 threads, 1 buffer) or
                                        // 1 (512 threads, 2 buffers)
  const longlong2* iseg;                // [n_ctiles * n_bgroups] (first entry, entries)
                                        // of each (tile, group) segment, tile-major
  const float2* ient_ff;                // coefficient (pair) of each entry; every segment
  const float* ient_f32;                // starts at a multiple of 4 entries (padding
  const uint32_t* ient_key;             // between); key (row in tile << 15) | column
  int* err;                             // error word (GSR_E_TIMEOUT), device alias of
                                        // mapped pinned host memory
  // exact power-of-two rescaling of the stored coefficients, A' = 2^e A 2^g
  // (null when every exponent is 0)
  const int16_t* row_exp;               // [n_rows] e_i
  const int16_t* col_exp;               // [n_unk]  g_j
};

// Positions of the knot-order copy of u that the products with FP32 values
// (FP32 records) or float-pair values read.
__host__ __device__ inline const int32_t* knot_positions(const Layout& L, int which_values) {
  return which_values == GSR_VALUES_F32 ? L.gpos : L.pos;
}

struct Scratch {
  double* red;          // partial-sum slots for last-block reductions
  unsigned int* count;  // arrival counters (one per reduction site)
  float2* x_ff;         // [n_unk] float-pair copy of an aprod 1 input
  float2* x3;           // [(n_knots-3) * 12] attitude part of an aprod 1 input,
                        // x[axis*K + s + j] at [s*12 + axis*4 + j] (96 B per start knot)
  float2* y_ff;         // [n_pad] float-pair copy of an aprod 2 input (zero padding)
  float2* y_knot;       // [n_rows] the same in knot order
  double* guard;        // [4] flags: [0] an aprod input left the float-pair band (the FP64
                        // kernels run), [1] column scaling check, [2] non-finite
                        // right-hand side, [3] the same for k right-hand sides
  int* iexp;            // [32] largest exponent of each right-hand side (LSQR scaling)
  double* zx;           // [n_unk] aprod 2 accumulator of a column-rescaled system (or null)
};

}  // namespace gsr
