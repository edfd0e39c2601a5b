// Library-side state of one system and the internal entry points shared
// between translation units (host code; the device layout and helpers are in
// gsr_internal.cuh).
#pragma once

#include "gsr_internal.cuh"

struct gsr_system {
  int device;
  int num_sms;
  gsr_dims dims;
  gsr::Layout L;
  gsr::Scratch S;
  // owned allocations
  unsigned char* rec_ff;
  unsigned char* rec_f32;
  int32_t* pos;
  float2* att_knot_ff;
  float* att_knot_f32;
  int64_t* knot_start;
  int32_t* att_warp_knot;
  longlong2* iseg;
  float2* ient_ff;
  float* ient_f32;
  uint32_t* ient_key;
  int* err;
  double* colnorm;       // [n_unk] ||A_:,j|| (FP64 values)
  // LSQR work vectors (allocated on first solve)
  float2* u;             // [n_pad] unnormalised u as float pairs (zero padding)
  float2* u_knot;        // [n_rows] u in knot order
  float2* v;             // [n_unk] v (float pairs)
  float2* w;             // [n_unk] w (float pairs)
  float2* xz;            // [n_unk] iterate of the scaled problem (float pairs)
  double* z;             // [n_unk] A^T u accumulator
  double* dscale;        // [n_unk] column scaling in use
  float2* dscale_ff;     // [n_unk] the same as float pairs
  float2* v_ff;          // [n_unk] float-pair D v (aprod 1 input)
  double* mx_x1;         // mixed precision: phase-1 solution [n_unk]
  double* mx_d;          // mixed precision: correction [n_unk]
  double* mx_r;          // mixed precision: residual b - A x1 [n_rows]
  double* scal;          // device LSQR scalars
  double* host_scal;     // pinned mirror of scal
  void* batch;           // multi-right-hand-side workspace (allocated on first use)
  int* instr_count;      // [n_instr] rows per instrumental column (learned features)
  cudaStream_t side;     // second stream for the attitude part of aprod 2
  cudaEvent_t ev_fork, ev_join;
  int main_block, main_ctas, main_smem;
  int a1_ctas;
};

// Internal entry points shared between translation units.
namespace gsr {
// Rows padded up to a whole number of instrumental tiles (float-pair vectors
// over the rows are allocated with this length, the padding zeroed).
inline int64_t padded_rows(const Layout& L) {
  const int64_t ct = L.ct_rows > 0 ? L.ct_rows : REC_ROWS;
  return ((L.n_rows + ct - 1) / ct) * ct + REC_ROWS;
}
// y = coef*y + A x on a double y (coef = *coef_dev if non-null), ||y||^2 into
// *norm_slot; y_knot must be null. The kernel does nothing when *stop != 0.
// The attitude unknowns are gathered from x_ff directly (no scratch).
int launch_aprod1(gsr_system* sys, int which_values, const float2* x_ff, double* y,
                  const double* coef_dev, double coef_host, double* y_knot, double* norm_slot,
                  const double* stop, cudaStream_t st);
// y += A x on a double y, the attitude unknowns read from sys->S.x3 (built by
// launch_att_x3 from the same x_ff).
int launch_aprod1_x3(gsr_system* sys, int which_values, const float2* x_ff, double* y,
                     cudaStream_t st);
// y = coef*y + A x on a float-pair y (LSQR's u), attitude from sys->S.x3, with
// the optional knot-order copy.
int launch_aprod1_ff(gsr_system* sys, int which_values, const float2* x_ff, float2* y,
                     const double* coef_dev, float2* y_knot, double* norm_slot,
                     const double* stop, cudaStream_t st);
// x += A^T y, y and y_knot (y in knot order) as float pairs, y zero-padded to
// padded_rows(); nothing when *stop != 0.
int launch_aprod2(gsr_system* sys, int which_values, const float2* y, const float2* y_knot,
                  double* x, const double* stop, cudaStream_t st);
int launch_to_ff(const double* x, const double* scale, float2* out, int64_t n, cudaStream_t st);
// out = -x as float pairs.
int launch_to_ff_neg(const double* x, float2* out, int64_t n, cudaStream_t st);
// Interleave the attitude part of a float-pair aprod 1 input by start knot
// (into sys->S.x3); aprod 1 reads it with three 32-byte loads per row.
int launch_att_x3(gsr_system* sys, const float2* x_ff, const double* stop, cudaStream_t st);
// y (double) -> y_ff (row order) and y_knot (knot order) as float pairs.
int launch_to_ff_knot(gsr_system* sys, const double* y, float2* y_ff, float2* y_knot,
                      cudaStream_t st);
int cuda_status(cudaError_t e);
int set_kernel_attributes();
void destroy_batch(gsr_system* s);
}  // namespace gsr
