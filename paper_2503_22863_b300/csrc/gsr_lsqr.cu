// Preconditioned LSQR (Paige & Saunders 1982, the solver of Sec. 2 / Sec. 2.1)
// on the column-scaled operator A D, with every scalar kept on the device.
//
// One iteration is five stream-ordered launches:
//   1. aprod 1:  u~ <- A (D v) - (alpha/beta) u~   and ||u~||^2        (Eq. 2)
//   2. z <- 0;   aprod 2: z <- A^T u~  (star-ordered + knot-ordered parts) (Eq. 3)
//   3. vec_a:    v~ <- D z / beta - beta v, ||v~||^2; the last block runs the
//                plane rotation (rho, c, s, theta, rhobar, phi, phibar)
//   4. vec_b:    x <- x + (phi/rho) w, w <- v~/alpha - (theta/rho) w, the
//                float-pair copy D v for the next aprod 1, ||x||, ||d_k||^2;
//                the last block evaluates the stopping tests
// u is kept unnormalised (u = u~/beta) so that no pass over the rows is spent
// on normalising it. Iterations are captured once into a CUDA graph and
// replayed in chunks; all kernels return immediately once the stop flag is
// set, so the host reads the flag only once per chunk.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <vector>

#include "gsr_system.cuh"

namespace gsr {

enum Scal {
  S_ALPHA = 0, S_BETA, S_RHOBAR, S_PHIBAR, S_ANORM2, S_DDNORM, S_BNORM, S_XNORM,
  S_RHO, S_C, S_S, S_THETA, S_PHI, S_T1, S_T2, S_RNORM, S_ARNORM, S_ACOND,
  S_ATOL, S_BTOL, S_CTOL, S_ITN, S_ITNLIM, S_ISTOP, S_DONE,
  S_UNORM2, S_VNORM2, S_COEF_U, S_ERR2, S_XREF2, S_RED3, S_RED3B, S_RED3C,
  S_BEXP,  // b is solved as 2^-S_BEXP b (largest |b_i| in [1, 2)); x, norms scaled back
  S_COUNT
};

// Grid of the vector kernels: three blocks per SM (their 72 and 80 registers
// per thread allow three 256-thread blocks). Their grid-wide sums end in one
// atomic per block and a last-block pass over the partials, which costs more
// than the extra memory parallelism of larger grids gains (measured on 5.16M
// unknowns: 0.184 ms per iteration at 8 blocks per SM, 0.163 at 4, 0.171 at 1;
// 0.143 at 2 against 0.137 at 3, back to back on the current kernels).
constexpr int RED_BLOCKS = 148 * 3;
constexpr int VEC_U = 4;             // elements per thread per step of the vector kernels

__device__ __forceinline__ double block_sum3(double& a, double& b, double& c, double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  a = warp_sum_d(a);
  b = warp_sum_d(b);
  c = warp_sum_d(c);
  __syncthreads();
  if (lane == 0) {
    sh[wid] = a;
    sh[32 + wid] = b;
    sh[64 + wid] = c;
  }
  __syncthreads();
  if (wid == 0) {
    a = lane < nw ? sh[lane] : 0.0;
    b = lane < nw ? sh[32 + lane] : 0.0;
    c = lane < nw ? sh[64 + lane] : 0.0;
    a = warp_sum_d(a);
    b = warp_sum_d(b);
    c = warp_sum_d(c);
  }
  return a;
}

// Deterministic grid reduction of three sums; returns true in the last block
// (thread 0 then holds the totals in a, b, c).
__device__ bool grid_sum3(double& a, double& b, double& c, double* part, unsigned int* counter) {
  __shared__ double sh[96];
  __shared__ int is_last;
  block_sum3(a, b, c, sh);
  if (threadIdx.x == 0) {
    part[3 * blockIdx.x] = a;
    part[3 * blockIdx.x + 1] = b;
    part[3 * blockIdx.x + 2] = c;
    __threadfence();
    unsigned int t = atomicAdd(counter, 1u);
    is_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  double x = 0.0, y = 0.0, z = 0.0;
  for (unsigned int i = threadIdx.x; i < gridDim.x; i += blockDim.x) {
    x += __ldcg(part + 3 * i);
    y += __ldcg(part + 3 * i + 1);
    z += __ldcg(part + 3 * i + 2);
  }
  block_sum3(x, y, z, sh);
  if (threadIdx.x == 0) {
    a = x;
    b = y;
    c = z;
    *counter = 0u;
  }
  return true;
}

// The same for four sums (vec_b): one shared-memory round per stage; returns
// true in the last block, thread 0 then holding the totals.
__device__ __forceinline__ void block_sum4(double v[4], double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < 4; ++q) v[q] = warp_sum_d(v[q]);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < 4; ++q) sh[32 * q + wid] = v[q];
  __syncthreads();
  if (wid == 0)
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = warp_sum_d(lane < nw ? sh[32 * q + lane] : 0.0);
}

__device__ bool grid_sum4(double& a, double& b, double& c, double& d, double* part,
                          unsigned int* counter) {
  __shared__ double sh4[128];
  __shared__ int is_last4;
  double v[4] = {a, b, c, d};
  block_sum4(v, sh4);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) part[4 * blockIdx.x + q] = v[q];
    __threadfence();
    is_last4 = (atomicAdd(counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!is_last4) return false;
  __threadfence();
  double t[4] = {0.0, 0.0, 0.0, 0.0};
  for (unsigned int i = threadIdx.x; i < gridDim.x; i += blockDim.x)
#pragma unroll
    for (int q = 0; q < 4; ++q) t[q] += __ldcg(part + 4 * i + q);
  block_sum4(t, sh4);
  if (threadIdx.x == 0) {
    a = t[0];
    b = t[1];
    c = t[2];
    d = t[3];
    *counter = 0u;
  }
  return true;
}

// ---------------------------------------------------------------------------
// Largest binary exponent over the nonzero entries of b into *mx (atomicMax,
// *mx preset very negative); a NaN or Inf entry sets *bad. LSQR is invariant
// under b -> 2^-s b (x and the residual norms scale by 2^-s), so the solve runs
// on b with its largest entry in [1, 2): whatever the magnitude of b, the
// float-pair vectors then neither overflow nor underflow as a whole.
// ---------------------------------------------------------------------------
__global__ void k_maxexp(const double* __restrict__ b, int64_t n, int* mx, double* bad) {
  int m = INT_MIN;
  bool nonfinite = false;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    const double v = b[r];
    if (!isfinite(v)) nonfinite = true;
    else if (v != 0.0) m = max(m, ilogb(v));
  }
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0 && m != INT_MIN) atomicMax(mx, m);
  if (nonfinite) *bad = 1.0;
}

// The exponent s of 2^-s b (0 for b = 0).
__device__ __forceinline__ int b_exponent(const int* mx) {
  const int m = *mx;
  return m < -4000 ? 0 : m;
}

// ---------------------------------------------------------------------------
// Start: u~ = 2^-s b (and its knot-order copy), ||u~||^2.
// ---------------------------------------------------------------------------
__global__ void k_init_u(Layout L, const double* __restrict__ b, const int* bexp,
                         float2* __restrict__ u, float2* __restrict__ u_knot,
                         const int32_t* __restrict__ pos, double* scal, double* part,
                         unsigned int* counter) {
  const int sb = b_exponent(bexp);
  if (blockIdx.x == 0 && threadIdx.x == 0) scal[S_BEXP] = sb;
  double s2 = 0.0, z0 = 0.0, z1 = 0.0;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < L.n_rows;
       r += (int64_t)gridDim.x * blockDim.x) {
    const double v = ldexp(b[r], -sb);
    const ff f = ff_from_double(v);
    u[r] = make_float2(f.h, f.l);
    u_knot[pos[r]] = make_float2(f.h, f.l);
    s2 = __fma_rn(v, v, s2);
  }
  if (grid_sum3(s2, z0, z1, part, counter) && threadIdx.x == 0) scal[S_UNORM2] = s2;
}

// ---------------------------------------------------------------------------
// vec_a: v~ = d z / beta - beta v (v absent on the first call); ||v~||^2;
// then (last block) the scalar step.
// ---------------------------------------------------------------------------
__global__ void k_vec_a(int64_t n, const float2* __restrict__ d, const double* __restrict__ z,
                        float2* __restrict__ v, double* scal, double* part, unsigned int* counter,
                        int first) {
  if (scal[S_DONE] != 0.0) return;
  const double beta = sqrt(scal[S_UNORM2]);
  const ff ib = ff_from_double(beta > 0.0 ? 1.0 / beta : 0.0), nbeta = ff_from_double(-beta);
  ff s2f = ff_zero();
  // VEC_U elements per thread per step, all loads issued first (latency)
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j0 < n;
       j0 += VEC_U * stride) {
    float2 dd[VEC_U], vv[VEC_U];
    double zz[VEC_U];
#pragma unroll
    for (int u = 0; u < VEC_U; ++u) {
      const int64_t j = j0 + u * stride;
      if (j < n) {
        dd[u] = d[j];
        zz[u] = z[j];
        if (!first) vv[u] = v[j];
      }
    }
#pragma unroll
    for (int u = 0; u < VEC_U; ++u) {
      const int64_t j = j0 + u * stride;
      if (j >= n) continue;
      ff t = ff_mul(ff_norm(ff_mul(ff{dd[u].x, dd[u].y}, ff_from_double(zz[u]))), ib);
      if (!first) t = ff_add(t, ff_mul(nbeta, ff{vv[u].x, vv[u].y}));
      t = ff_norm(t);
      v[j] = make_float2(t.h, t.l);
      s2f = ff_add(s2f, ff_mul(t, t));
    }
  }
  double s2 = ff_to_double(s2f), z0 = 0.0, z1 = 0.0;
  if (!grid_sum3(s2, z0, z1, part, counter) || threadIdx.x != 0) return;
  const double alpha = sqrt(s2);
  if (first) {
    scal[S_BETA] = beta;
    scal[S_BNORM] = beta;
    scal[S_ALPHA] = alpha;
    scal[S_RHOBAR] = alpha;
    scal[S_PHIBAR] = beta;
    scal[S_RNORM] = beta;
    scal[S_ARNORM] = alpha * beta;
    scal[S_COEF_U] = beta > 0.0 ? -alpha / beta : 0.0;
    if (alpha * beta == 0.0) {  // b = 0 or A^T b = 0: x = 0 is the solution
      scal[S_ISTOP] = 0.0;
      scal[S_DONE] = 1.0;
    }
    return;
  }
  const double alpha_old = scal[S_ALPHA];
  scal[S_ANORM2] += alpha_old * alpha_old + beta * beta;
  const double rhobar = scal[S_RHOBAR], phibar = scal[S_PHIBAR];
  const double rho = sqrt(rhobar * rhobar + beta * beta);
  const double c = rhobar / rho, s = beta / rho;
  const double theta = s * alpha;
  scal[S_RHO] = rho;
  scal[S_C] = c;
  scal[S_S] = s;
  scal[S_THETA] = theta;
  scal[S_RHOBAR] = -c * alpha;
  scal[S_PHI] = c * phibar;
  scal[S_PHIBAR] = s * phibar;
  scal[S_T1] = c * phibar / rho;
  scal[S_T2] = -theta / rho;
  scal[S_BETA] = beta;
  scal[S_ALPHA] = alpha;
  scal[S_COEF_U] = beta > 0.0 ? -alpha / beta : 0.0;
}

// ---------------------------------------------------------------------------
// vec_b: normalise v, update x and w, write D v as float pairs, ||x||,
// ||d_k||^2 and the variance; then (last block) the stopping tests.
// ---------------------------------------------------------------------------
// With column exponents (cexp) the float-pair D' = 2^-g D v carries them, so
// x = 2^g D' z is formed in FP64 for ||x|| and the error (its entries may span
// more than FP32's range).
__global__ void k_vec_b(int64_t n, const float2* __restrict__ d, float2* __restrict__ v,
                        float2* __restrict__ w, float2* __restrict__ xz,
                        float2* __restrict__ v_ff, double* __restrict__ var,
                        const double* __restrict__ x_ref, const double* __restrict__ x_off,
                        const int16_t* __restrict__ cexp, double* scal, double* part,
                        unsigned int* counter, int first, double* err_hist, double* rnorm_hist) {
  if (scal[S_DONE] != 0.0) return;
  const int sb = (int)scal[S_BEXP];
  double x2d = 0.0;
  const double alpha = scal[S_ALPHA];
  const ff ia = ff_from_double(alpha > 0.0 ? 1.0 / alpha : 0.0);
  const ff irho = ff_from_double(first ? 1.0 : 1.0 / scal[S_RHO]);
  const ff t1 = ff_from_double(first ? 0.0 : scal[S_T1]);
  const ff t2 = ff_from_double(first ? 0.0 : scal[S_T2]);
  ff dk2f = ff_zero(), x2f = ff_zero(), z2f = ff_zero();
  double e2 = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j0 < n;
       j0 += VEC_U * stride) {
    float2 vv[VEC_U], dv[VEC_U], wv[VEC_U], xv_[VEC_U];
#pragma unroll
    for (int u = 0; u < VEC_U; ++u) {
      const int64_t j = j0 + u * stride;
      if (j < n) {
        vv[u] = v[j];
        dv[u] = d[j];
        if (!first) {
          wv[u] = w[j];
          xv_[u] = xz[j];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < VEC_U; ++u) {
      const int64_t j = j0 + u * stride;
      if (j >= n) continue;
      const float2 vj = vv[u], djf = dv[u];
      const ff dj = ff{djf.x, djf.y};
      const ff vn = ff_norm(ff_mul(ff{vj.x, vj.y}, ia));
      ff xv = ff_zero();
      if (first) {
        w[j] = make_float2(vn.h, vn.l);
        xz[j] = make_float2(0.f, 0.f);
      } else {
        const float2 wf = wv[u], xf = xv_[u];
        const ff wj = ff{wf.x, wf.y};
        const ff dk = ff_mul(wj, irho);
        const ff dd = ff_mul(dk, dk);
        dk2f = ff_add(dk2f, dd);
        if (var) var[j] += ff_to_double(dd);
        const ff xn = ff_norm(ff_add(ff{xf.x, xf.y}, ff_mul(t1, wj)));
        xz[j] = make_float2(xn.h, xn.l);
        z2f = ff_add(z2f, ff_mul(xn, xn));
        const ff wn = ff_norm(ff_add(vn, ff_mul(t2, wj)));
        w[j] = make_float2(wn.h, wn.l);
        xv = ff_norm(ff_mul(dj, xn));
        if (cexp) {
          const double xd = ldexp(ff_to_double(xv), (int)cexp[j]);
          x2d = __fma_rn(xd, xd, x2d);
        } else {
          x2f = ff_add(x2f, ff_mul(xv, xv));
        }
      }
      v[j] = make_float2(vn.h, vn.l);
      const ff f = ff_norm(ff_mul(dj, vn));
      v_ff[j] = make_float2(f.h, f.l);
      if (x_ref) {
        double xd = ff_to_double(xv);
        xd = ldexp(xd, sb + (cexp ? (int)cexp[j] : 0));
        const double e = (x_off ? xd + x_off[j] : xd) - x_ref[j];
        e2 = __fma_rn(e, e, e2);
      }
    }
  }
  double dk2 = ff_to_double(dk2f), x2 = ff_to_double(x2f) + x2d, z2 = ff_to_double(z2f);
  if (!grid_sum4(dk2, x2, e2, z2, part, counter) || threadIdx.x != 0) return;
  if (first) return;
  const double itn = scal[S_ITN] + 1.0;
  scal[S_ITN] = itn;
  const double ddnorm = scal[S_DDNORM] + dk2;
  scal[S_DDNORM] = ddnorm;
  const double anorm = sqrt(scal[S_ANORM2]);
  const double acond = anorm * sqrt(ddnorm);
  const double rnorm = scal[S_PHIBAR];
  const double arnorm = alpha * fabs(scal[S_C]) * rnorm;
  const double xnorm = sqrt(x2);
  const double bnorm = scal[S_BNORM];
  scal[S_ACOND] = acond;
  scal[S_RNORM] = rnorm;
  scal[S_ARNORM] = arnorm;
  scal[S_XNORM] = xnorm;
  const int64_t k = (int64_t)itn - 1;
  if (err_hist) {
    const double xr2 = scal[S_XREF2];
    err_hist[k] = xr2 > 0.0 ? sqrt(e2 / xr2) : sqrt(e2);
  }
  if (rnorm_hist) rnorm_hist[k] = ldexp(rnorm, sb);
  const double atol = scal[S_ATOL], btol = scal[S_BTOL], ctol = scal[S_CTOL];
  // the tests belong to the preconditioned system the loop solves (Sec. 2,
  // solver step 2): ||A D|| and the norm of its iterate z; ||x|| is reported
  const double znorm = sqrt(z2);
  const double test1 = rnorm / bnorm;
  const double test2 = (anorm * rnorm > 0.0) ? arnorm / (anorm * rnorm) : 0.0;
  const double test3 = 1.0 / acond;
  const double t1n = test1 / (1.0 + anorm * znorm / bnorm);
  const double rtol = btol + atol * anorm * znorm / bnorm;
  int istop = 0;
  if (itn >= scal[S_ITNLIM]) istop = 7;
  if (1.0 + test3 <= 1.0) istop = 6;
  if (1.0 + test2 <= 1.0) istop = 5;
  if (1.0 + t1n <= 1.0) istop = 4;
  if (test3 <= ctol) istop = 3;
  if (test2 <= atol) istop = 2;
  if (test1 <= rtol) istop = 1;
  scal[S_ISTOP] = istop;
  if (istop != 0) scal[S_DONE] = 1.0;
}

// Sec. 2.2, Eq. 4 for the chosen pairs: cov[p] += d_k[j1] d_k[j2] with the
// direction d_k = w_k / rho_k of this iteration (w still the old one: the
// kernel runs after vec_a has computed rho and before vec_b updates w).
__global__ void k_cov(int64_t n_cov, const int64_t* __restrict__ pairs,
                      const float2* __restrict__ w, const double* scal,
                      double* __restrict__ cov) {
  if (scal[S_DONE] != 0.0) return;
  const double irho = 1.0 / scal[S_RHO];
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n_cov;
       p += (int64_t)gridDim.x * blockDim.x) {
    const float2 a = w[pairs[2 * p]], b = w[pairs[2 * p + 1]];
    const double d1 = ff_to_double(ff{a.x, a.y}) * irho, d2 = ff_to_double(ff{b.x, b.y}) * irho;
    cov[p] = __fma_rn(d1, d2, cov[p]);
  }
}

// *bad = 1 if any pair has an index outside [0, n).
__global__ void k_cov_check(int64_t n_cov, const int64_t* __restrict__ pairs, int64_t n,
                            double* bad) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < 2 * n_cov;
       p += (int64_t)gridDim.x * blockDim.x)
    if (pairs[p] < 0 || pairs[p] >= n) *bad = 1.0;
}

// cov[p] *= d[j1] d[j2] (de-precondition).
__global__ void k_cov_finish(int64_t n_cov, const int64_t* __restrict__ pairs,
                             const double* __restrict__ d, double* __restrict__ cov) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n_cov;
       p += (int64_t)gridDim.x * blockDim.x)
    cov[p] *= d[pairs[2 * p]] * d[pairs[2 * p + 1]];
}

__global__ void k_sumsq(int64_t n, const double* __restrict__ a, double* scal, int slot,
                        double* part, unsigned int* counter) {
  double s2 = 0.0, z0 = 0.0, z1 = 0.0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x)
    s2 = __fma_rn(a[j], a[j], s2);
  if (grid_sum3(s2, z0, z1, part, counter) && threadIdx.x == 0) scal[slot] = s2;
}

// Column scaling D (Sec. 2 solver step 2) in FP64, and the float pairs of
// D' = 2^-g D that the products use (A D = A' D' with A' = A 2^g). *bad = 2 for
// a scale that is not positive and finite, 1 for a D' outside the vector band.
__global__ void k_scale_setup(int64_t n, int mode, const double* __restrict__ colnorm,
                              const double* __restrict__ user, const int16_t* __restrict__ cexp,
                              double* __restrict__ d, float2* __restrict__ d_ff, double* bad) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    double s = 1.0;
    if (mode == GSR_PRECOND_COLNORM) {
      const double c = colnorm[j];
      s = c > 0.0 ? 1.0 / c : 1.0;
    } else if (mode == GSR_PRECOND_USER) {
      s = user[j];
    }
    d[j] = s;
    const double sp = cexp ? ldexp(s, -(int)cexp[j]) : s;
    if (!(s > 0.0) || !isfinite(s)) *bad = 2.0;
    else if (!vec_in_band(sp)) *bad = 1.0;
    const ff f = ff_from_double(sp);
    d_ff[j] = make_float2(f.h, f.l);
  }
}

// x = 2^s D z (de-precondition, Sec. 2 solver step 5, and undo the scaling of
// b); var = D^2 var.
__global__ void k_finish(int64_t n, const double* __restrict__ d, const float2* __restrict__ xz,
                         const double* scal, double* __restrict__ x, double* __restrict__ var) {
  const int sb = (int)scal[S_BEXP];
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    const double dj = d[j];
    const float2 z = xz[j];
    x[j] = dj * ldexp(ff_to_double(ff{z.x, z.y}), sb);
    if (var) var[j] *= dj * dj;
  }
}

__global__ void k_zero(int64_t n, double* __restrict__ a, const double* scal) {
  if (scal && scal[S_DONE] != 0.0) return;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x)
    a[j] = 0.0;
}

namespace {

int ensure_work(gsr_system* s) {
  if (s->u) return GSR_OK;
  const int64_t n = s->L.n_rows, m = s->L.n_unk;
  cudaError_t e = cudaSuccess;
  auto A = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes ? bytes : 8);
  };
  A((void**)&s->u, padded_rows(s->L) * 8);
  A((void**)&s->u_knot, n * 8);
  A((void**)&s->v, m * 8);
  A((void**)&s->w, m * 8);
  A((void**)&s->xz, m * 8);
  A((void**)&s->z, m * 8);
  A((void**)&s->dscale, m * 8);
  A((void**)&s->dscale_ff, m * 8);
  A((void**)&s->v_ff, m * 8);
  A((void**)&s->scal, S_COUNT * 8);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&s->host_scal, S_COUNT * 8);
  if (e == cudaSuccess) e = cudaMemset(s->u, 0, padded_rows(s->L) * 8);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? GSR_E_OOM : GSR_E_CUDA;
  }
  return GSR_OK;
}

struct Ctx {
  gsr_system* s;
  cudaStream_t st;
  int which_values;
  double* var;
  const double* x_ref;
  const double* x_off;
  double* err_dev;
  double* rn_dev;
  int64_t n_cov;
  const int64_t* cov_pairs;
  double* cov;
};

constexpr int LAUNCHES_PER_ITERATION = 8;  // x3, aprod1, zero, aprod2 (3), vec_a, vec_b

// Events (4 per iteration) bracket aprod 1, aprod 2 and the vector kernels;
// while the iteration is captured into a graph they are recorded as external
// event nodes (the flag is valid only during capture).
int enqueue_iteration(const Ctx& c, cudaEvent_t* ev, bool capturing) {
  const unsigned ev_flags = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
  gsr_system* s = c.s;
  const Layout& L = s->L;
  double* scal = s->scal;
  const int vb = (int)std::min<int64_t>(RED_BLOCKS, (L.n_unk + 255) / 256 + 1);
  if (ev) cudaEventRecordWithFlags(ev[0], c.st, ev_flags);
  int rc = launch_att_x3(s, s->v_ff, scal + S_DONE, c.st);
  if (rc != GSR_OK) return rc;
  rc = launch_aprod1_ff(s, c.which_values, s->v_ff, s->u, scal + S_COEF_U, s->u_knot,
                            scal + S_UNORM2, scal + S_DONE, c.st);
  if (rc != GSR_OK) return rc;
  rc = con_aprod1_lsqr(s, s->v_ff, scal + S_COEF_U, scal + S_UNORM2, scal + S_DONE, c.st);
  if (rc != GSR_OK) return rc;
  k_zero<<<vb, 256, 0, c.st>>>(L.n_unk, s->z, scal);
  if (ev) cudaEventRecordWithFlags(ev[1], c.st, ev_flags);
  rc = launch_aprod2(s, c.which_values, s->u, s->u_knot, s->z, scal + S_DONE, c.st);
  if (rc != GSR_OK) return rc;
  rc = con_aprod2_lsqr(s, s->z, scal + S_DONE, c.st);
  if (rc != GSR_OK) return rc;
  if (ev) cudaEventRecordWithFlags(ev[2], c.st, ev_flags);
  k_vec_a<<<vb, 256, 0, c.st>>>(L.n_unk, s->dscale_ff, s->z, s->v, scal, s->S.red,
                                s->S.count + 1, 0);
  if (c.n_cov > 0) {
    const int cb = (int)std::min<int64_t>((c.n_cov + 255) / 256, (int64_t)s->num_sms * 4);
    k_cov<<<cb, 256, 0, c.st>>>(c.n_cov, c.cov_pairs, s->w, scal, c.cov);
  }
  k_vec_b<<<vb, 256, 0, c.st>>>(L.n_unk, s->dscale_ff, s->v, s->w, s->xz, s->v_ff, c.var, c.x_ref,
                                c.x_off, L.col_exp, scal, s->S.red, s->S.count + 2, 0, c.err_dev,
                                c.rn_dev);
  if (ev) cudaEventRecordWithFlags(ev[3], c.st, ev_flags);
  return cuda_status(cudaGetLastError());
}

}  // namespace

// One LSQR solve of min ||A x - b|| on the chosen copy of the values. x_off
// (optional) is added to the iterate when measuring the error against x_ref
// (the correction phase of the mixed-precision solve).
int lsqr_run(gsr_system* s, const double* b, double* x, const gsr_lsqr_opts* o,
             gsr_lsqr_result* res, cudaStream_t st, int which_values, const double* x_off,
             int64_t itnlim) {
  const Layout& L = s->L;
  const int vb = (int)std::min<int64_t>(RED_BLOCKS, (L.n_unk + 255) / 256 + 1);
  const int rb = (int)std::min<int64_t>(RED_BLOCKS, (L.n_rows + 255) / 256 + 1);
  double* scal = s->scal;
  cudaError_t e = cudaSuccess;
  auto C = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
  };
  // scalars
  double h[S_COUNT];
  std::memset(h, 0, sizeof(h));
  h[S_ATOL] = o->atol;
  h[S_BTOL] = o->btol;
  h[S_CTOL] = o->conlim > 0.0 ? 1.0 / o->conlim : 0.0;
  h[S_ITNLIM] = (double)itnlim;
  C(cudaMemcpyAsync(scal, h, sizeof(h), cudaMemcpyHostToDevice, st));
  // exponent of the largest |b_i| (and a check that b is finite); the
  // covariance pairs' indexes
  const int64_t n_cov = (o->cov && o->cov_pairs) ? o->n_cov : 0;
  C(cudaMemsetAsync(s->S.iexp, 0x80, sizeof(int), st));
  C(cudaMemsetAsync(s->S.guard + 2, 0, 2 * sizeof(double), st));
  {
    const int64_t n_eq = L.n_rows + s->n_con;
    const int eb = (int)std::min<int64_t>(RED_BLOCKS, (n_eq + 255) / 256 + 1);
    k_maxexp<<<eb, 256, 0, st>>>(b, n_eq, s->S.iexp, s->S.guard + 2);
  }
  if (n_cov > 0)
    k_cov_check<<<(int)std::min<int64_t>((2 * n_cov + 255) / 256, 148 * 4), 256, 0, st>>>(
        n_cov, o->cov_pairs, L.n_unk, s->S.guard + 3);
  C(cudaGetLastError());
  double flags[2] = {0.0, 0.0};
  C(cudaMemcpyAsync(flags, s->S.guard + 2, sizeof(flags), cudaMemcpyDeviceToHost, st));
  C(cudaStreamSynchronize(st));  // h and flags are stack buffers
  if (e != cudaSuccess) return GSR_E_CUDA;
  if (flags[0] != 0.0) return GSR_E_NONFINITE;
  if (flags[1] != 0.0) return GSR_E_INDEX;
  if (n_cov > 0) C(cudaMemsetAsync(o->cov, 0, n_cov * sizeof(double), st));
  // per-iteration histories
  double* err_dev = nullptr;
  double* rn_dev = nullptr;
  if (o->err_hist && o->x_ref) C(cudaMallocAsync((void**)&err_dev, itnlim * 8 + 8, st));
  if (o->rnorm_hist) C(cudaMallocAsync((void**)&rn_dev, itnlim * 8 + 8, st));
  if (e != cudaSuccess) return GSR_E_CUDA;
  if (o->x_ref && err_dev)
    k_sumsq<<<vb, 256, 0, st>>>(L.n_unk, o->x_ref, scal, S_XREF2, s->S.red, s->S.count + 3);
  if (o->var) k_zero<<<vb, 256, 0, st>>>(L.n_unk, o->var, nullptr);
  k_zero<<<vb, 256, 0, st>>>(L.n_unk, reinterpret_cast<double*>(s->xz), nullptr);
  // start: beta_1 u_1 = b, alpha_1 v_1 = (A D)^T u_1, w_1 = v_1, x_0 = 0
  k_init_u<<<rb, 256, 0, st>>>(L, b, s->S.iexp, s->u, s->u_knot, knot_positions(L, which_values),
                               scal, s->S.red, s->S.count + 4);
  int rc = con_init_lsqr(s, b + L.n_rows, scal + S_BEXP, scal + S_UNORM2, st);
  if (rc != GSR_OK) return rc;
  k_zero<<<vb, 256, 0, st>>>(L.n_unk, s->z, nullptr);
  rc = launch_aprod2(s, which_values, s->u, s->u_knot, s->z, nullptr, st);
  if (rc != GSR_OK) return rc;
  rc = con_aprod2_lsqr(s, s->z, nullptr, st);
  if (rc != GSR_OK) return rc;
  k_vec_a<<<vb, 256, 0, st>>>(L.n_unk, s->dscale_ff, s->z, s->v, scal, s->S.red, s->S.count + 1,
                              1);
  k_vec_b<<<vb, 256, 0, st>>>(L.n_unk, s->dscale_ff, s->v, s->w, s->xz, s->v_ff, o->var,
                              o->x_ref && err_dev ? o->x_ref : nullptr, x_off, L.col_exp, scal,
                              s->S.red, s->S.count + 2, 1, nullptr, nullptr);
  C(cudaGetLastError());
  if (e != cudaSuccess) return GSR_E_CUDA;

  int64_t n_launches = 8 + (o->var ? 1 : 0) + ((o->x_ref && err_dev) ? 1 : 0) +
                       (s->n_con > 0 ? (s->con_nseg > 0 ? 2 : 1) : 0);
  Ctx c{s,      st,     which_values, o->var, (o->x_ref && err_dev) ? o->x_ref : nullptr,
        x_off,  err_dev, rn_dev,      n_cov,  o->cov_pairs,
        o->cov};
  if (n_cov > 0) n_launches += 1;  // the check
  // Capture a chunk of iterations once and replay it.
  const int chunk = 4;
  const bool prof = o->profile != 0;
  cudaEvent_t evs[4 * chunk];
  int n_ev = 0;
  if (prof) {
    for (; n_ev < 4 * chunk; ++n_ev)
      if (cudaEventCreate(&evs[n_ev]) != cudaSuccess) break;
    if (n_ev < 4 * chunk) {
      for (int i = 0; i < n_ev; ++i) cudaEventDestroy(evs[i]);
      return GSR_E_CUDA;
    }
  }
  double t_a1 = 0.0, t_a2 = 0.0, t_vec = 0.0;
  int64_t timed = 0, itn_seen = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool use_graph = true;
  {
    cudaStreamCaptureStatus cs;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
      use_graph = false;
  }
  if (use_graph && st != nullptr) {
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      int r2 = GSR_OK;
      for (int i = 0; i < chunk && r2 == GSR_OK; ++i)
        r2 = enqueue_iteration(c, prof ? evs + 4 * i : nullptr, true);
      cudaError_t ce = cudaStreamEndCapture(st, &graph);
      if (r2 != GSR_OK || ce != cudaSuccess ||
          cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
        cudaGetLastError();
        if (graph) cudaGraphDestroy(graph);
        graph = nullptr;
        exec = nullptr;
        use_graph = false;
      }
    } else {
      cudaGetLastError();
      use_graph = false;
    }
  } else {
    use_graph = false;
  }
  int64_t launched = 0;
  while (true) {
    if (use_graph) {
      C(cudaGraphLaunch(exec, st));
    } else {
      for (int i = 0; i < chunk && e == cudaSuccess; ++i) {
        rc = enqueue_iteration(c, prof ? evs + 4 * i : nullptr, false);
        if (rc != GSR_OK) break;
      }
    }
    launched += chunk;
    n_launches += (int64_t)chunk * (LAUNCHES_PER_ITERATION + (n_cov > 0 ? 1 : 0) +
                                    (s->n_con > 0 ? (s->con_nseg > 0 ? 4 : 2) : 0));
    C(cudaMemcpyAsync(s->host_scal, scal, S_COUNT * 8, cudaMemcpyDeviceToHost, st));
    C(cudaStreamSynchronize(st));
    if (e != cudaSuccess || rc != GSR_OK) break;
    if (prof) {
      // iterations of this chunk that did work (the rest returned at once)
      const int64_t itn_now = (int64_t)s->host_scal[S_ITN];
      const int64_t worked = std::min<int64_t>(chunk, itn_now - itn_seen);
      for (int i = 0; i < worked; ++i) {
        float a = 0.f, b2 = 0.f, v = 0.f;
        C(cudaEventElapsedTime(&a, evs[4 * i], evs[4 * i + 1]));
        C(cudaEventElapsedTime(&b2, evs[4 * i + 1], evs[4 * i + 2]));
        C(cudaEventElapsedTime(&v, evs[4 * i + 2], evs[4 * i + 3]));
        t_a1 += a;
        t_a2 += b2;
        t_vec += v;
      }
      timed += worked > 0 ? worked : 0;
      itn_seen = itn_now;
    }
    if (s->host_scal[S_DONE] != 0.0) break;
    if (launched > itnlim + chunk) break;  // cannot happen: istop = 7 at itnlim
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  for (int i = 0; i < n_ev; ++i) cudaEventDestroy(evs[i]);
  if (e != cudaSuccess || rc != GSR_OK) {
    if (err_dev) cudaFreeAsync(err_dev, st);
    if (rn_dev) cudaFreeAsync(rn_dev, st);
    return rc != GSR_OK ? rc : GSR_E_CUDA;
  }
  const double* hs = s->host_scal;
  const int64_t itn = (int64_t)hs[S_ITN];
  if (x) k_finish<<<vb, 256, 0, st>>>(L.n_unk, s->dscale, s->xz, scal, x, o->var);
  if (n_cov > 0) {
    k_cov_finish<<<(int)std::min<int64_t>((n_cov + 255) / 256, 148 * 4), 256, 0, st>>>(
        n_cov, o->cov_pairs, s->dscale, o->cov);
    ++n_launches;
  }
  if (o->err_hist && err_dev && itn > 0)
    C(cudaMemcpyAsync(o->err_hist, err_dev, itn * 8, cudaMemcpyDeviceToHost, st));
  if (o->rnorm_hist && rn_dev && itn > 0)
    C(cudaMemcpyAsync(o->rnorm_hist, rn_dev, itn * 8, cudaMemcpyDeviceToHost, st));
  if (err_dev) C(cudaFreeAsync(err_dev, st));
  if (rn_dev) C(cudaFreeAsync(rn_dev, st));
  C(cudaStreamSynchronize(st));
  if (e != cudaSuccess) return GSR_E_CUDA;
  const int sb = (int)hs[S_BEXP];
  res->istop = (int32_t)hs[S_ISTOP];
  res->itn = itn;
  res->rnorm = std::ldexp(hs[S_RNORM], sb);
  res->arnorm = std::ldexp(hs[S_ARNORM], sb);
  res->anorm = std::sqrt(hs[S_ANORM2]);
  res->acond = hs[S_ACOND];
  res->xnorm = std::ldexp(hs[S_XNORM], sb);
  res->n_launches = n_launches + (x ? 1 : 0);
  res->n_timed_itn = timed;
  res->t_aprod1_ms = t_a1;
  res->t_aprod2_ms = t_a2;
  res->t_vector_ms = t_vec;
  return GSR_OK;
}

__global__ void k_axpy_into(int64_t n, double a, const double* __restrict__ xa,
                            const double* __restrict__ xb, double* __restrict__ out) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x)
    out[j] = __fma_rn(a, xa[j], xb[j]);
}

// Mixed precision (FP32-stored A, FP64 correction):
//   phase 1: LSQR with the FP32-rounded values (half the matrix bytes; float-pair
//            arithmetic and FP64 vectors/scalars as everywhere) to about FP32 accuracy;
//   phase 2: r = b - A x1 with the full-precision values, then LSQR on
//            min ||A d - r|| with the full-precision values and the caller's
//            tolerances; x = x1 + d. Phase 2 uses the full-precision matrix in
//            both products, so its fixed point is the full-precision solution.
int lsqr_mixed(gsr_system* s, const double* b, double* x, const gsr_lsqr_opts* o,
               gsr_lsqr_result* res, cudaStream_t st, int64_t itnlim) {
  const int64_t n = s->L.n_rows + s->n_con, m = s->L.n_unk;  // equations, unknowns
  if (s->mx_r_len < n) {  // the residual vector follows the constraint count
    if (s->mx_r) cudaFree(s->mx_r);
    s->mx_r = nullptr;
    s->mx_r_len = 0;
    if (cudaMalloc((void**)&s->mx_r, (n > 0 ? n : 1) * 8) != cudaSuccess) {
      cudaGetLastError();
      return GSR_E_OOM;
    }
    s->mx_r_len = n;
  }
  if (!s->mx_x1) {
    cudaError_t e = cudaMalloc((void**)&s->mx_x1, m * 8);
    if (e == cudaSuccess) e = cudaMalloc((void**)&s->mx_d, m * 8);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return e == cudaErrorMemoryAllocation ? GSR_E_OOM : GSR_E_CUDA;
    }
  }
  constexpr double PHASE1_TOL = 1e-7;  // about the relative size of FP32 rounding of A
  gsr_lsqr_opts o1 = *o;
  int64_t lim1 = itnlim;
  if (o->mixed_switch_itn > 0) {
    o1.atol = o1.btol = 0.0;
    o1.conlim = 0.0;
    lim1 = std::min<int64_t>(itnlim, o->mixed_switch_itn);
  } else {
    o1.atol = std::max(o->atol, PHASE1_TOL);
    o1.btol = std::max(o->btol, PHASE1_TOL);
  }
  o1.rnorm_hist = nullptr;
  gsr_lsqr_result r1;
  std::memset(&r1, 0, sizeof(r1));
  int rc = lsqr_run(s, b, s->mx_x1, &o1, &r1, st, GSR_VALUES_F32, nullptr, lim1);
  if (rc != GSR_OK) return rc;
  // r = b - A x1 with the full-precision values
  const int vb = (int)std::min<int64_t>(RED_BLOCKS, (m + 255) / 256 + 1);
  cudaError_t e = cudaMemcpyAsync(s->mx_r, b, n * 8, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return GSR_E_CUDA;
  rc = aprod1_direct(s, GSR_VALUES_F64, s->mx_x1, 1, s->mx_r, st);
  if (rc != GSR_OK) return rc;
  // phase 2
  gsr_lsqr_opts o2 = *o;
  o2.var = nullptr;
  o2.n_cov = 0;
  o2.cov = nullptr;
  o2.cov_pairs = nullptr;
  const int64_t n1 = r1.itn;
  o2.err_hist = o->err_hist ? o->err_hist + n1 : nullptr;
  o2.rnorm_hist = o->rnorm_hist ? o->rnorm_hist + n1 : nullptr;
  const int64_t lim2 = std::max<int64_t>(1, itnlim - n1);
  rc = lsqr_run(s, s->mx_r, s->mx_d, &o2, res, st, GSR_VALUES_F64, s->mx_x1, lim2);
  if (rc != GSR_OK) return rc;
  k_axpy_into<<<vb, 256, 0, st>>>(m, 1.0, s->mx_d, s->mx_x1, x);
  if (cudaStreamSynchronize(st) != cudaSuccess) return GSR_E_CUDA;
  res->phase2_itn = (int32_t)res->itn;
  res->itn += n1;
  res->n_launches += r1.n_launches + 6;
  res->n_timed_itn += r1.n_timed_itn;
  res->t_aprod1_ms += r1.t_aprod1_ms;
  res->t_aprod2_ms += r1.t_aprod2_ms;
  res->t_vector_ms += r1.t_vector_ms;
  return GSR_OK;
}

// D and D'; GSR_E_ARG for a user scale that is not positive and finite,
// GSR_E_UNSUPPORTED for one that D' = 2^-g D takes outside the vector band.
int setup_scaling(gsr_system* s, const gsr_lsqr_opts* o, cudaStream_t st) {
  const int vb = (int)std::min<int64_t>(RED_BLOCKS, (s->L.n_unk + 255) / 256 + 1);
  if (cudaMemsetAsync(s->S.guard + 1, 0, sizeof(double), st) != cudaSuccess) return GSR_E_CUDA;
  k_scale_setup<<<vb, 256, 0, st>>>(s->L.n_unk, o->precond, s->colnorm, o->scale, s->L.col_exp,
                                    s->dscale, s->dscale_ff, s->S.guard + 1);
  double bad = 0.0;
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(&bad, s->S.guard + 1, sizeof(double), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return GSR_E_CUDA;
  if (bad == 2.0) return GSR_E_ARG;
  if (bad != 0.0) return GSR_E_UNSUPPORTED;
  return GSR_OK;
}

}  // namespace gsr

extern "C" {

void gsr_lsqr_default_opts(gsr_lsqr_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->atol = 1e-12;
  o->btol = 1e-12;
  o->conlim = 1e12;
  o->itnlim = 0;
  o->precond = GSR_PRECOND_COLNORM;
  o->precision = GSR_PREC_F64;
}

int gsr_lsqr_solve(gsr_system* sys, const double* b, double* x, const gsr_lsqr_opts* opts,
                   gsr_lsqr_result* res, void* stream) {
  if (!sys || !opts || !res) return GSR_E_ARG;
  if ((!b && sys->L.n_rows > 0) || (!x && sys->L.n_unk > 0)) return GSR_E_ARG;
  if (opts->precond < GSR_PRECOND_NONE || opts->precond > GSR_PRECOND_USER) return GSR_E_ARG;
  if (opts->precond == GSR_PRECOND_USER && !opts->scale) return GSR_E_ARG;
  if (opts->precision != GSR_PREC_F64 && opts->precision != GSR_PREC_MIXED) return GSR_E_ARG;
  if (opts->precision == GSR_PREC_MIXED && !sys->rec_f32) return GSR_E_ARG;
  if (opts->atol < 0 || opts->btol < 0 || opts->conlim < 0 || opts->itnlim < 0) return GSR_E_ARG;
  if ((opts->err_hist && !opts->x_ref)) return GSR_E_ARG;
  if (opts->n_cov < 0 || (opts->n_cov > 0 && (!opts->cov_pairs || !opts->cov))) return GSR_E_ARG;
  // rows rescaled by different powers of two cannot be folded into the column
  // preconditioner (they would reweight the least-squares problem)
  if (sys->row_scaled) return GSR_E_UNSUPPORTED;
  std::memset(res, 0, sizeof(*res));
  gsr::DeviceGuard dg(sys->device);
  if (!dg.ok) return GSR_E_CUDA;
  if (const int se = gsr::sticky_error(sys)) return se;  // an earlier launch failed
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc = gsr::ensure_work(sys);
  if (rc != GSR_OK) return rc;
  rc = gsr::setup_scaling(sys, opts, st);
  if (rc != GSR_OK) return rc;
  const int64_t itnlim = opts->itnlim > 0 ? opts->itnlim : 20 * std::max<int64_t>(1, sys->L.n_unk);
  if (sys->L.n_rows + sys->n_con == 0 || sys->L.n_unk == 0) {
    if (x && sys->L.n_unk > 0) cudaMemsetAsync(x, 0, sys->L.n_unk * 8, st);
    res->istop = 0;
    return gsr::cuda_status(cudaStreamSynchronize(st));
  }
  rc = opts->precision == GSR_PREC_MIXED
           ? gsr::lsqr_mixed(sys, b, x, opts, res, st, itnlim)
           : gsr::lsqr_run(sys, b, x, opts, res, st, GSR_VALUES_F64, nullptr, itnlim);
  // the solve has synchronised: a failed bounded wait of any of its kernels shows here
  if (rc == GSR_OK) rc = gsr::sticky_error(sys);
  return rc;
}

}  // extern "C"
