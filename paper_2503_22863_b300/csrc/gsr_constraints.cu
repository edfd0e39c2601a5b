// Constraint equations of the AVU-GSR system (Sec. 2: the overdetermined
// system needs a set of constraint equations for a unique solution; Sec. 2.1:
// they are about 1% of the system and are replicated on every process). The
// paper does not give their form, so they are generic sparse rows appended to
// A after the observations, in CSR form.
//
// They are few rows with many entries each (a condition over many stars or
// knots), so the work is split into segments of at most CON_SEG entries, one
// warp per segment: lanes stride over the segment, the warp sums in FP64 and
// one FP64 atomic per segment adds the sum into the row's result. All
// constraint arithmetic is FP64 (values, vectors, products): it is a small part
// of each product, and FP64 carries any coefficient range without rescaling.
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "gsr_system.cuh"

namespace gsr {

namespace {

constexpr int64_t CON_SEG = 1024;  // entries per segment (one warp)

// Row r of the segment table's segment g, and its entry range.
struct Seg {
  int64_t b, e;
  int row;
};
__device__ __forceinline__ Seg seg_at(const longlong2* segs, const int32_t* rows, int64_t g) {
  const longlong2 q = segs[g];
  return Seg{q.x, q.y, rows[g]};
}

// Direct aprod 1 on the constraint rows: y_con[row] +=/-= sum val x.
__global__ void k_con_aprod1(int64_t nseg, const longlong2* __restrict__ segs,
                             const int32_t* __restrict__ rows, const int64_t* __restrict__ col,
                             const double* __restrict__ val, const double* __restrict__ x,
                             int neg, double* __restrict__ y_con) {
  const int lane = threadIdx.x & 31;
  for (int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; g < nseg;
       g += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const Seg q = seg_at(segs, rows, g);
    double s = 0.0;
    for (int64_t k = q.b + lane; k < q.e; k += 32) s = __fma_rn(val[k], x[col[k]], s);
    s = warp_sum_d(s);
    if (lane == 0) atomicAdd(y_con + q.row, neg ? -s : s);
  }
}

// Direct aprod 2 on the constraint rows: x[col] += val y_con[row].
__global__ void k_con_aprod2(int64_t nseg, const longlong2* __restrict__ segs,
                             const int32_t* __restrict__ rows, const int64_t* __restrict__ col,
                             const double* __restrict__ val, const double* __restrict__ y_con,
                             double* __restrict__ x) {
  const int lane = threadIdx.x & 31;
  for (int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; g < nseg;
       g += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const Seg q = seg_at(segs, rows, g);
    const double yr = y_con[q.row];
    if (yr == 0.0) continue;
    for (int64_t k = q.b + lane; k < q.e; k += 32) atomicAdd(x + col[k], __dmul_rn(val[k], yr));
  }
}

// LSQR aprod 1 on the constraint rows: u_con[row] += sum (2^g val) x_ff (the
// float-pair D' v), after k_con_scale has multiplied u_con by coef.
__global__ void k_con_aprod1_lsqr(int64_t nseg, const longlong2* __restrict__ segs,
                                  const int32_t* __restrict__ rows,
                                  const int64_t* __restrict__ col, const double* __restrict__ val,
                                  const int16_t* __restrict__ cexp, const float2* __restrict__ x,
                                  double* __restrict__ u_con, const double* stop) {
  if (stop && *stop != 0.0) return;
  const int lane = threadIdx.x & 31;
  for (int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; g < nseg;
       g += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const Seg q = seg_at(segs, rows, g);
    double s = 0.0;
    for (int64_t k = q.b + lane; k < q.e; k += 32) {
      const int64_t j = col[k];
      const double a = cexp ? ldexp(val[k], (int)cexp[j]) : val[k];
      const float2 xv = x[j];
      s = __fma_rn(a, ff_to_double(ff{xv.x, xv.y}), s);
    }
    s = warp_sum_d(s);
    if (lane == 0) atomicAdd(u_con + q.row, s);
  }
}

// LSQR aprod 2 on the constraint rows: z[col] += (2^g val) u_con[row].
__global__ void k_con_aprod2_lsqr(int64_t nseg, const longlong2* __restrict__ segs,
                                  const int32_t* __restrict__ rows,
                                  const int64_t* __restrict__ col, const double* __restrict__ val,
                                  const int16_t* __restrict__ cexp,
                                  const double* __restrict__ u_con, double* __restrict__ z,
                                  const double* stop) {
  if (stop && *stop != 0.0) return;
  const int lane = threadIdx.x & 31;
  for (int64_t g = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; g < nseg;
       g += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const Seg q = seg_at(segs, rows, g);
    const double ur = u_con[q.row];
    if (ur == 0.0) continue;
    for (int64_t k = q.b + lane; k < q.e; k += 32) {
      const int64_t j = col[k];
      const double a = cexp ? ldexp(val[k], (int)cexp[j]) : val[k];
      atomicAdd(z + j, __dmul_rn(a, ur));
    }
  }
}

// Deterministic one-block sum (256 threads).
__device__ double block_sum_256(double v) {
  __shared__ double sh[8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_sum_d(v);
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < 8; ++w) t += sh[w];
  return t;  // valid in thread 0
}

// One block: u_con *= coef (before the products are added).
__global__ void k_con_scale(int64_t n_con, const double* coef, double* u_con, const double* stop) {
  if (stop && *stop != 0.0) return;
  const double c = *coef;
  for (int64_t i = threadIdx.x; i < n_con; i += blockDim.x) u_con[i] *= c;
}

// One block: *unorm2 += ||u_con||^2.
__global__ void k_con_norm(int64_t n_con, const double* u_con, double* unorm2,
                           const double* stop) {
  if (stop && *stop != 0.0) return;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n_con; i += blockDim.x) s = __fma_rn(u_con[i], u_con[i], s);
  s = block_sum_256(s);
  if (threadIdx.x == 0) *unorm2 += s;
}

// One block: u_con = 2^-s b_con (s from the LSQR scalars) and *unorm2 += ||u_con||^2.
__global__ void k_con_init(int64_t n_con, const double* b_con, const double* bexp, double* u_con,
                           double* unorm2) {
  const int sb = (int)*bexp;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n_con; i += blockDim.x) {
    const double v = ldexp(b_con[i], -sb);
    u_con[i] = v;
    s = __fma_rn(v, v, s);
  }
  s = block_sum_256(s);
  if (threadIdx.x == 0) *unorm2 += s;
}

int seg_blocks(const gsr_system* s) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((s->con_nseg + 7) / 8,
                                                     (int64_t)s->num_sms * 16));
}

}  // namespace

void free_constraints(gsr_system* s) {
  void* p[] = {s->con_col, s->con_val, s->con_seg, s->con_seg_row, s->u_con};
  for (void* q : p)
    if (q) cudaFree(q);
  s->con_col = nullptr;
  s->con_val = nullptr;
  s->con_seg = nullptr;
  s->con_seg_row = nullptr;
  s->u_con = nullptr;
  s->n_con = s->con_nnz = s->con_nseg = 0;
}

int con_aprod1_direct(gsr_system* s, const double* x, int neg, double* y, cudaStream_t st) {
  if (s->n_con == 0 || s->con_nseg == 0) return GSR_OK;
  k_con_aprod1<<<seg_blocks(s), 256, 0, st>>>(s->con_nseg, s->con_seg, s->con_seg_row,
                                              s->con_col, s->con_val, x, neg, y + s->L.n_rows);
  return cuda_status(cudaGetLastError());
}

int con_aprod2_direct(gsr_system* s, const double* y, double* x, cudaStream_t st) {
  if (s->n_con == 0 || s->con_nseg == 0) return GSR_OK;
  k_con_aprod2<<<seg_blocks(s), 256, 0, st>>>(s->con_nseg, s->con_seg, s->con_seg_row,
                                              s->con_col, s->con_val, y + s->L.n_rows, x);
  return cuda_status(cudaGetLastError());
}

int con_aprod1_lsqr(gsr_system* s, const float2* x_ff, const double* coef, double* unorm2,
                    const double* stop, cudaStream_t st) {
  if (s->n_con == 0) return GSR_OK;
  k_con_scale<<<1, 256, 0, st>>>(s->n_con, coef, s->u_con, stop);
  if (s->con_nseg > 0)
    k_con_aprod1_lsqr<<<seg_blocks(s), 256, 0, st>>>(s->con_nseg, s->con_seg, s->con_seg_row,
                                                     s->con_col, s->con_val, s->L.col_exp, x_ff,
                                                     s->u_con, stop);
  k_con_norm<<<1, 256, 0, st>>>(s->n_con, s->u_con, unorm2, stop);
  return cuda_status(cudaGetLastError());
}

int con_aprod2_lsqr(gsr_system* s, double* z, const double* stop, cudaStream_t st) {
  if (s->n_con == 0 || s->con_nseg == 0) return GSR_OK;
  k_con_aprod2_lsqr<<<seg_blocks(s), 256, 0, st>>>(s->con_nseg, s->con_seg, s->con_seg_row,
                                                   s->con_col, s->con_val, s->L.col_exp, s->u_con,
                                                   z, stop);
  return cuda_status(cudaGetLastError());
}

int con_init_lsqr(gsr_system* s, const double* b_con, const double* bexp_scal, double* unorm2,
                  cudaStream_t st) {
  if (s->n_con == 0) return GSR_OK;
  k_con_init<<<1, 256, 0, st>>>(s->n_con, b_con, bexp_scal, s->u_con, unorm2);
  return cuda_status(cudaGetLastError());
}

}  // namespace gsr

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

int gsr_set_constraints(gsr_system* sys, int64_t n_con, const int64_t* con_ptr,
                        const int64_t* con_col, const double* con_val, void* stream) {
  if (!sys || n_con < 0 || n_con >= (int64_t(1) << 31)) return GSR_E_ARG;
  if (n_con > 0 && !con_ptr) return GSR_E_ARG;
  const int64_t nnz = n_con > 0 ? con_ptr[n_con] : 0;
  if (n_con > 0 && (con_ptr[0] != 0 || nnz < 0)) return GSR_E_ARG;
  if (nnz > 0 && (!con_col || !con_val)) return GSR_E_ARG;
  // host validation before the device is touched
  const int64_t n_unk = sys->L.n_unk;
  for (int64_t c = 0; c < n_con; ++c)
    if (con_ptr[c + 1] < con_ptr[c]) return GSR_E_ARG;
  for (int64_t k = 0; k < nnz; ++k) {
    if (con_col[k] < 0 || con_col[k] >= n_unk) return GSR_E_INDEX;
    if (!std::isfinite(con_val[k])) return GSR_E_NONFINITE;
  }
  gsr::DeviceGuard dg(sys->device);
  if (!dg.ok) return GSR_E_CUDA;
  if (const int se = gsr::sticky_error(sys)) return se;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(st) != cudaSuccess) return GSR_E_CUDA;
  // the observation-only column norms, kept the first time
  if (!sys->colnorm_obs) {
    sys->colnorm_obs = new (std::nothrow) double[n_unk > 0 ? n_unk : 1];
    if (!sys->colnorm_obs) return GSR_E_OOM;
    if (cudaMemcpy(sys->colnorm_obs, sys->colnorm, n_unk * sizeof(double),
                   cudaMemcpyDeviceToHost) != cudaSuccess)
      return GSR_E_CUDA;
  }
  gsr::free_constraints(sys);
  // segments of at most CON_SEG entries
  std::vector<longlong2> seg;
  std::vector<int32_t> seg_row;
  for (int64_t c = 0; c < n_con; ++c)
    for (int64_t k = con_ptr[c]; k < con_ptr[c + 1]; k += gsr::CON_SEG) {
      seg.push_back(make_longlong2(k, std::min(k + gsr::CON_SEG, con_ptr[c + 1])));
      seg_row.push_back((int32_t)c);
    }
  // column norms with the constraint rows: sqrt(c_obs^2 + sum val^2) (long
  // double: the squares of any finite coefficient stay in range)
  std::vector<long double> add(n_unk, 0.0L);
  for (int64_t k = 0; k < nnz; ++k)
    add[con_col[k]] += (long double)con_val[k] * (long double)con_val[k];
  std::vector<double> cn(n_unk);
  for (int64_t j = 0; j < n_unk; ++j) {
    const long double c = sys->colnorm_obs[j];
    cn[j] = (double)std::sqrt(c * c + add[j]);
  }
  cudaError_t e = cudaSuccess;
  auto A = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes ? bytes : 8);
  };
  if (n_con > 0) {
    A((void**)&sys->con_col, nnz * sizeof(int64_t));
    A((void**)&sys->con_val, nnz * sizeof(double));
    A((void**)&sys->con_seg, seg.size() * sizeof(longlong2));
    A((void**)&sys->con_seg_row, seg_row.size() * sizeof(int32_t));
    A((void**)&sys->u_con, n_con * sizeof(double));
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    gsr::free_constraints(sys);
    return e == cudaErrorMemoryAllocation ? GSR_E_OOM : GSR_E_CUDA;
  }
  if (n_con > 0) {
    if (nnz > 0) {
      e = cudaMemcpy(sys->con_col, con_col, nnz * sizeof(int64_t), cudaMemcpyHostToDevice);
      if (e == cudaSuccess)
        e = cudaMemcpy(sys->con_val, con_val, nnz * sizeof(double), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess && !seg.empty())
      e = cudaMemcpy(sys->con_seg, seg.data(), seg.size() * sizeof(longlong2),
                     cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !seg_row.empty())
      e = cudaMemcpy(sys->con_seg_row, seg_row.data(), seg_row.size() * sizeof(int32_t),
                     cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(sys->u_con, 0, n_con * sizeof(double));
  }
  if (e == cudaSuccess)
    e = cudaMemcpy(sys->colnorm, cn.data(), n_unk * sizeof(double), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaGetLastError();
    gsr::free_constraints(sys);
    return GSR_E_CUDA;
  }
  sys->n_con = n_con;
  sys->con_nnz = nnz;
  sys->con_nseg = (int64_t)seg.size();
  return GSR_OK;
}

int64_t gsr_n_equations(const gsr_system* sys) { return sys ? sys->L.n_rows + sys->n_con : -1; }

}  // extern "C"
