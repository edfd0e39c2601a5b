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
  int32_t* kb_start;
  int32_t* gpos;  // null when the knot order is not blocked (L.gpos == pos)
  int32_t* att_warp_knot;
  longlong2* iseg;
  float2* ient_ff;
  float* ient_f32;
  uint32_t* ient_key;
  int* err;              // device alias of err_host
  int* err_host;         // mapped pinned word a kernel sets on a failed bounded wait
  int16_t* row_exp;      // [n_rows] rescaling exponents e_i (null: all 0)
  int16_t* col_exp;      // [n_unk] rescaling exponents g_j (null: all 0)
  bool row_scaled;       // some e_i differ: LSQR is not available (rows would be reweighted)
  bool wide;             // some rescaled coefficient is below 2^-40: direct products run FP64
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
  double* mx_r;          // mixed precision: residual b - A x1 [n_rows + n_con]
  int64_t mx_r_len;      // entries allocated for mx_r
  double* scal;          // device LSQR scalars
  double* host_scal;     // pinned mirror of scal
  void* batch;           // multi-right-hand-side workspace (allocated on first use)
  int* instr_count;      // [n_instr] rows per instrumental column (learned features)
  // constraint equations: n_con CSR rows after the n_rows observations (FP64)
  int64_t n_con, con_nnz, con_nseg;
  int64_t* con_col;      // [nnz] column of each entry
  double* con_val;       // [nnz] coefficient (original units)
  longlong2* con_seg;    // [nseg] (first entry, end) of each segment of <= CON_SEG entries
  int32_t* con_seg_row;  // [nseg] constraint row of each segment
  double* u_con;         // [n_con] LSQR's u on the constraint rows (FP64, scaled like b)
  double* colnorm_obs;   // [n_unk] host copy of the column norms without constraints
  cudaStream_t side;     // second stream for the attitude part of aprod 2
  cudaEvent_t ev_fork, ev_join;
  int main_block, main_ctas, main_smem;
  int a1_ctas;
};

// Internal entry points shared between translation units.
namespace gsr {
// Makes `device` current for the lifetime of the object and gives the caller's
// current device back afterwards (entry points leave it as they found it).
// The code a kernel of this system recorded (GSR_E_TIMEOUT), or GSR_OK. Read
// from mapped host memory: a failure becomes visible to the calls that follow
// it without a synchronisation.
inline int sticky_error(const gsr_system* s) {
  return s && s->err_host ? *reinterpret_cast<volatile const int*>(s->err_host) : GSR_OK;
}
struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int device) {
    if (cudaGetDevice(&prev) != cudaSuccess) {
      cudaGetLastError();
      prev = -1;
    }
    ok = prev == device || cudaSetDevice(device) == cudaSuccess;
  }
  ~DeviceGuard() {
    if (ok && prev >= 0) cudaSetDevice(prev);
  }
  DeviceGuard(const DeviceGuard&) = delete;
  DeviceGuard& operator=(const DeviceGuard&) = delete;
};

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
                     const double* stop, cudaStream_t st);
// y += A x (neg: y -= A x) for a double x and y on the original (unscaled)
// problem: rescales x, checks it against the float-pair band and runs either
// the float-pair kernels or, when the guard is set (or the system is wide),
// the FP64 kernel.
int aprod1_direct(gsr_system* sys, int which_values, const double* x, int neg, double* y,
                  cudaStream_t st);
// x += A^T y, the same two-way choice.
int aprod2_direct(gsr_system* sys, int which_values, const double* y, double* x,
                  cudaStream_t st);
// FP64 kernels on k interleaved vectors (x[col * k + j], y[row * k + j]);
// they run only when *guard != 0 (guard null: always).
int launch_aprod1_f64(gsr_system* sys, int which_values, const double* x, int k, int neg,
                      double* y, const double* guard, cudaStream_t st);
int launch_aprod2_f64(gsr_system* sys, int which_values, const double* y, int k, double* x,
                      const double* guard, cudaStream_t st);
// y = coef*y + A x on a float-pair y (LSQR's u), attitude from sys->S.x3, with
// the optional knot-order copy.
int launch_aprod1_ff(gsr_system* sys, int which_values, const float2* x_ff, float2* y,
                     const double* coef_dev, float2* y_knot, double* norm_slot,
                     const double* stop, cudaStream_t st);
// x += A^T y, y and y_knot (y in knot order) as float pairs, y zero-padded to
// padded_rows(); nothing when *stop != 0.
int launch_aprod2(gsr_system* sys, int which_values, const float2* y, const float2* y_knot,
                  double* x, const double* stop, cudaStream_t st);
// out = +-2^-cexp x (times scale) as float pairs; entries outside the
// vector band set *guard (cexp, scale and guard may be null).
int launch_to_ff(const double* x, const double* scale, const int16_t* cexp, int neg,
                 double* guard, float2* out, int64_t n, cudaStream_t st);
// Interleave the attitude part of a float-pair aprod 1 input by start knot
// (into sys->S.x3); aprod 1 reads it with three 32-byte loads per row.
int launch_att_x3(gsr_system* sys, const float2* x_ff, const double* stop, cudaStream_t st);
// y (double) -> y_ff (row order) and y_knot (the knot-order copy the products
// with `which_values` read) as float pairs.
int launch_to_ff_knot(gsr_system* sys, int which_values, const double* y, float2* y_ff,
                      float2* y_knot, double* guard, cudaStream_t st);
int cuda_status(cudaError_t e);
int set_kernel_attributes();
void destroy_batch(gsr_system* s);
void free_constraints(gsr_system* s);
// Constraint rows. Direct products on the original values and FP64 vectors:
// y[n_rows + c] += (or -=) A_con x, and x += A_con^T y[n_rows ..].
int con_aprod1_direct(gsr_system* s, const double* x, int neg, double* y, cudaStream_t st);
int con_aprod2_direct(gsr_system* s, const double* y, double* x, cudaStream_t st);
// LSQR forms (values times 2^g_j; x_ff = D' v float pairs; u_con FP64):
//   u_con = coef u_con + A'_con x_ff and ||u_con||^2 added to *unorm2,
//   z += A'_con^T u_con, and the start u_con = 2^-s b_con with ||u_con||^2 added.
// All return at once when *stop != 0.
int con_aprod1_lsqr(gsr_system* s, const float2* x_ff, const double* coef, double* unorm2,
                    const double* stop, cudaStream_t st);
int con_aprod2_lsqr(gsr_system* s, double* z, const double* stop, cudaStream_t st);
int con_init_lsqr(gsr_system* s, const double* b_con, const double* bexp_scal, double* unorm2,
                  cudaStream_t st);
}  // namespace gsr
