// aprod 1 (Eq. 2, y += A x) and aprod 2 (Eq. 3, x += A^T y) kernels for sm_103a.
//
// Both products are HBM-bound (about 0.2 flop per byte) and use no tensor
// cores. B300's FP64 pipe runs at ~1/64 of its FP32 rate, so every product
// and sum is done on the FP32 pipe as a float pair (hi, lo) with error-free
// transformations; only a few FP64 operations per row remain (converting u,
// forming the output, the norm).
#include "gsr_internal.cuh"

namespace gsr {

// ---------------------------------------------------------------------------
// Deterministic grid reduction: every block stores its partial sum, the last
// block to arrive adds the partials in index order and resets the counter.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double block_sum_d(double v, double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum_d(v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (wid == 0) {
    s = lane < nw ? sh[lane] : 0.0;
    s = warp_sum_d(s);
  }
  return s;  // valid in warp 0
}

__device__ void grid_sum_store(double v, double* part, unsigned int* counter, double* out) {
  __shared__ double sh[32];
  __shared__ int is_last;
  double s = block_sum_d(v, sh);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = s;
    __threadfence();
    unsigned int t = atomicAdd(counter, 1u);
    is_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (is_last) {
    __threadfence();
    double acc = 0.0;
    for (unsigned int i = threadIdx.x; i < gridDim.x; i += blockDim.x) acc += __ldcg(part + i);
    acc = block_sum_d(acc, sh);
    if (threadIdx.x == 0) {
      *out = acc;
      *counter = 0u;
    }
  }
}

// ---------------------------------------------------------------------------
// Element conversions.
// ---------------------------------------------------------------------------
__global__ void k_to_ff(const double* __restrict__ x, const double* __restrict__ scale,
                        float2* __restrict__ out, int64_t n) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    double v = x[j];
    if (scale) v *= scale[j];
    ff f = ff_from_double(v);
    out[j] = make_float2(f.h, f.l);
  }
}

__global__ void k_scatter_knot(Layout L, const double* __restrict__ y, double* __restrict__ y_knot) {
  const int32_t* pos = reinterpret_cast<const int32_t*>(L.att_pos);
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < L.n_rows;
       r += (int64_t)gridDim.x * blockDim.x)
    y_knot[pos[r]] = y[r];
}

// Value of slot `t` for rows 4*lane + 2q + c of a tile, as a pair.
template <bool F32>
struct Vals;

template <>
struct Vals<false> {
  float4 v;
  __device__ __forceinline__ void load(const Layout& L, int64_t tile, int t, int q, int lane) {
    v = __ldcs(L.vals_ff + ((tile * NSLOT + t) * 2 + q) * 32 + lane);
  }
  __device__ __forceinline__ ff get(int c) const {
    return c == 0 ? ff{v.x, v.y} : ff{v.z, v.w};
  }
  __device__ __forceinline__ ff mul(int c, ff u) const { return ff_mul(get(c), u); }
};

template <>
struct Vals<true> {
  float2 v;
  __device__ __forceinline__ void load(const Layout& L, int64_t tile, int t, int q, int lane) {
    v = __ldcs(L.vals_f32 + ((tile * NSLOT + t) * 2 + q) * 32 + lane);
  }
  __device__ __forceinline__ ff mul(int c, ff u) const { return f_mul(c == 0 ? v.x : v.y, u); }
};

__device__ __forceinline__ ff ldx(const float2* __restrict__ x, int64_t j) {
  float2 a = __ldg(x + j);
  return ff{a.x, a.y};
}

__device__ __forceinline__ int sel4(int4 a, int j) {
  return j == 0 ? a.x : j == 1 ? a.y : j == 2 ? a.z : a.w;
}
__device__ __forceinline__ int sel4u(ushort4 a, int j) {
  return j == 0 ? a.x : j == 1 ? a.y : j == 2 ? a.z : a.w;
}

// ---------------------------------------------------------------------------
// aprod 1: y[r] = coef * y[r] + (A x)[r] for every row; optionally
// y_knot[pos(r)] = y[r] (the knot-ordered copy aprod 2 reads) and a
// deterministic ||y||^2 into *norm_out. coef is *coef_dev if given.
// One warp per 128-row tile (grid-stride over tiles), 4 rows per lane.
// ---------------------------------------------------------------------------
template <bool F32>
__global__ void __launch_bounds__(256) k_aprod1(Layout L, const float2* __restrict__ x,
                                                double* __restrict__ y,
                                                const double* __restrict__ coef_dev,
                                                double coef_host, double* __restrict__ y_knot,
                                                double* part, unsigned int* counter,
                                                double* norm_out, const double* stop) {
  if (stop && *stop != 0.0) return;
  const int lane = threadIdx.x & 31;
  const int64_t gwarp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const double coef = coef_dev ? *coef_dev : coef_host;
  const bool glob = L.n_glob == 1;
  const ff xg = glob ? ldx(x, L.glob_col) : ff_zero();
  const int32_t* posv = reinterpret_cast<const int32_t*>(L.att_pos);
  double nrm = 0.0;
  int cur_star = -1;
  ff xa[5];
#pragma unroll
  for (int t = 0; t < 5; ++t) xa[t] = ff_zero();

  for (int64_t tile = gwarp; tile < L.n_tiles; tile += nwarps) {
    const int64_t row0 = tile * TILE_ROWS + lane * ROWS_PER_LANE;
    const int4 st = __ldcs(L.star + tile * 32 + lane);
    const int4 sv = __ldcs(L.att_s + tile * 32 + lane);
    ushort4 ins[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) ins[k] = __ldcs(L.instr + (tile * 6 + k) * 32 + lane);
    double yo[4];
    if (row0 + 3 < L.n_rows) {
      const double2 a = *reinterpret_cast<const double2*>(y + row0);
      const double2 b = *reinterpret_cast<const double2*>(y + row0 + 2);
      yo[0] = a.x; yo[1] = a.y; yo[2] = b.x; yo[3] = b.y;
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) yo[j] = (row0 + j < L.n_rows) ? y[row0 + j] : 0.0;
    }
    double yn[4];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      ff acc[2] = {ff_zero(), ff_zero()};
      // astrometric block: 5 consecutive columns of the row's star
      Vals<F32> va[5];
#pragma unroll
      for (int t = 0; t < 5; ++t) va[t].load(L, tile, t, q, lane);
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int s = sel4(st, 2 * q + c);
        if (s != cur_star) {
          cur_star = s;
#pragma unroll
          for (int t = 0; t < 5; ++t) xa[t] = ldx(x, 5 * (int64_t)s + t);
        }
#pragma unroll
        for (int t = 0; t < 5; ++t) acc[c] = ff_add(acc[c], va[t].mul(c, xa[t]));
      }
      // attitude: 3 axes x 4 consecutive knots from s_i
#pragma unroll
      for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          Vals<F32> v;
          v.load(L, tile, 5 + 4 * a + i, q, lane);
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            const int64_t col = L.att_base + (int64_t)a * L.n_knots + sel4(sv, 2 * q + c) + i;
            acc[c] = ff_add(acc[c], v.mul(c, ldx(x, col)));
          }
        }
      }
      // instrumental
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        Vals<F32> v;
        v.load(L, tile, 17 + k, q, lane);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const int64_t col = L.instr_base + sel4u(ins[k], 2 * q + c);
          acc[c] = ff_add(acc[c], v.mul(c, ldx(x, col)));
        }
      }
      if (glob) {
        Vals<F32> v;
        v.load(L, tile, 23, q, lane);
#pragma unroll
        for (int c = 0; c < 2; ++c) acc[c] = ff_add(acc[c], v.mul(c, xg));
      }
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int j = 2 * q + c;
        yn[j] = __fma_rn(coef, yo[j], ff_to_double(acc[c]));
      }
    }
    if (row0 + 3 < L.n_rows) {
      *reinterpret_cast<double2*>(y + row0) = make_double2(yn[0], yn[1]);
      *reinterpret_cast<double2*>(y + row0 + 2) = make_double2(yn[2], yn[3]);
#pragma unroll
      for (int j = 0; j < 4; ++j) nrm = __fma_rn(yn[j], yn[j], nrm);
      if (y_knot) {
        const int4 p = __ldcs(L.att_pos + tile * 32 + lane);
        y_knot[p.x] = yn[0];
        y_knot[p.y] = yn[1];
        y_knot[p.z] = yn[2];
        y_knot[p.w] = yn[3];
      }
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (row0 + j < L.n_rows) {
          y[row0 + j] = yn[j];
          nrm = __fma_rn(yn[j], yn[j], nrm);
          if (y_knot) y_knot[posv[row0 + j]] = yn[j];
        }
      }
    }
  }
  if (norm_out) grid_sum_store(nrm, part, counter, norm_out);
}

// ---------------------------------------------------------------------------
// aprod 2, star-ordered part: astrometric (segmented per-star sums over the
// star-sorted rows, no atomics inside a warp's range), instrumental
// (shared-memory histogram per block) and global (warp + block sums).
// Each warp owns a contiguous tile range; runs of one star that cross lanes
// are joined by a segmented warp scan and runs that cross tiles by a carry.
// Results are added into x (x += A^T y).
// ---------------------------------------------------------------------------
struct Astro {
  ff c[5];
};

__device__ __forceinline__ Astro astro_add(const Astro& a, const Astro& b) {
  Astro r;
#pragma unroll
  for (int t = 0; t < 5; ++t) r.c[t] = ff_add(a.c[t], b.c[t]);
  return r;
}
__device__ __forceinline__ Astro astro_zero() {
  Astro r;
#pragma unroll
  for (int t = 0; t < 5; ++t) r.c[t] = ff_zero();
  return r;
}
__device__ __forceinline__ Astro astro_shfl_up(const Astro& a, int d) {
  Astro r;
#pragma unroll
  for (int t = 0; t < 5; ++t) r.c[t] = ff_shfl_up(a.c[t], d);
  return r;
}
__device__ __forceinline__ Astro astro_shfl(const Astro& a, int src) {
  Astro r;
#pragma unroll
  for (int t = 0; t < 5; ++t)
    r.c[t] = ff{__shfl_sync(0xffffffffu, a.c[t].h, src), __shfl_sync(0xffffffffu, a.c[t].l, src)};
  return r;
}
__device__ __forceinline__ void astro_flush(double* __restrict__ x, int star, const Astro& a) {
#pragma unroll
  for (int t = 0; t < 5; ++t) atomicAdd(x + 5 * (int64_t)star + t, ff_to_double(a.c[t]));
}

template <bool F32>
__global__ void __launch_bounds__(512) k_aprod2_main(Layout L, const double* __restrict__ y,
                                                     double* __restrict__ x,
                                                     const double* stop) {
  if (stop && *stop != 0.0) return;
  extern __shared__ double hist[];  // [n_instr]
  const int lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < L.n_instr; i += blockDim.x) hist[i] = 0.0;
  __syncthreads();
  const int64_t gwarp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const bool glob = L.n_glob == 1;
  ff gacc = ff_zero();
  int carry_star = -1;
  Astro carry = astro_zero();
  if (gwarp < L.n_main_warps) {
    const int64_t t_begin = L.row_tile_warp[gwarp], t_end = L.row_tile_warp[gwarp + 1];
    for (int64_t tile = t_begin; tile < t_end; ++tile) {
      const int64_t row0 = tile * TILE_ROWS + lane * ROWS_PER_LANE;
      const int4 st = __ldcs(L.star + tile * 32 + lane);
      double ud[4];
      if (row0 + 3 < L.n_rows) {
        const double2 a = __ldcs(reinterpret_cast<const double2*>(y + row0));
        const double2 b = __ldcs(reinterpret_cast<const double2*>(y + row0 + 2));
        ud[0] = a.x; ud[1] = a.y; ud[2] = b.x; ud[3] = b.y;
      } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) ud[j] = (row0 + j < L.n_rows) ? y[row0 + j] : 0.0;
      }
      ff u[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) u[j] = ff_from_double(ud[j]);

      // products of the astrometric slots, per row
      Astro p[4];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
#pragma unroll
        for (int t = 0; t < 5; ++t) {
          Vals<F32> v;
          v.load(L, tile, t, q, lane);
          p[2 * q].c[t] = v.mul(0, u[2 * q]);
          p[2 * q + 1].c[t] = v.mul(1, u[2 * q + 1]);
        }
      }
      // global column
      if (glob) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          Vals<F32> v;
          v.load(L, tile, 23, q, lane);
          gacc = ff_add(gacc, v.mul(0, u[2 * q]));
          gacc = ff_add(gacc, v.mul(1, u[2 * q + 1]));
        }
      }
      // instrumental columns: block-private histogram
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        const ushort4 ik = __ldcs(L.instr + (tile * 6 + k) * 32 + lane);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          Vals<F32> v;
          v.load(L, tile, 17 + k, q, lane);
          atomicAdd(hist + sel4u(ik, 2 * q), ff_to_double(v.mul(0, u[2 * q])));
          atomicAdd(hist + sel4u(ik, 2 * q + 1), ff_to_double(v.mul(1, u[2 * q + 1])));
        }
      }

      // ---- astrometric segmented reduction ----
      const int s0 = st.x, s1 = st.y, s2 = st.z, s3 = st.w;
      const bool uniform = (s0 == s3);
      // head run: rows with star s0 (a prefix); tail run: rows with star s3 (a suffix)
      Astro head = p[0];
      if (s1 == s0) head = astro_add(head, p[1]);
      if (s2 == s0) head = astro_add(head, p[2]);
      if (s3 == s0) head = astro_add(head, p[3]);
      Astro tail;
      if (uniform) {
        tail = head;
      } else {
        tail = p[3];
        if (s2 == s3) tail = astro_add(tail, p[2]);
        if (s1 == s3) tail = astro_add(tail, p[1]);
        // interior runs (a star strictly inside the lane's four rows)
        if (s1 != s0 && s1 != s3) {
          Astro r = p[1];
          if (s2 == s1) r = astro_add(r, p[2]);
          astro_flush(x, s1, r);
        }
        if (s2 != s0 && s2 != s3 && s2 != s1) astro_flush(x, s2, p[2]);
      }
      // the carry from the previous tile joins lane 0's head run or is complete
      const int first_star = __shfl_sync(0xffffffffu, s0, 0);
      if (carry_star >= 0 && carry_star != first_star) {
        if (lane == 0) astro_flush(x, carry_star, carry);
        carry_star = -1;
      }
      if (lane == 0 && carry_star >= 0) {
        head = astro_add(head, carry);
        if (uniform) tail = head;
      }
      // segmented inclusive scan of the tail runs across lanes
      const int prev_last = __shfl_up_sync(0xffffffffu, s3, 1);
      int flag = (lane == 0) || !uniform || (s0 != prev_last);
      Astro V = tail;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const Astro vu = astro_shfl_up(V, d);
        const int fu = __shfl_up_sync(0xffffffffu, flag, d);
        if (lane >= d) {
          if (!flag) V = astro_add(V, vu);
          flag |= fu;
        }
      }
      const Astro vprev = astro_shfl_up(V, 1);
      if (!uniform) {
        Astro tot = head;
        if (lane > 0 && s0 == prev_last) tot = astro_add(tot, vprev);
        astro_flush(x, s0, tot);
      }
      const int s0_next = __shfl_down_sync(0xffffffffu, s0, 1);
      if (lane < 31 && s0_next != s3) astro_flush(x, s3, V);
      carry_star = __shfl_sync(0xffffffffu, s3, 31);
      carry = astro_shfl(V, 31);
    }
    if (carry_star >= 0 && lane == 0) astro_flush(x, carry_star, carry);
  }
  if (glob) {
    gacc = ff_warp_sum(gacc);
    if (lane == 0 && (gacc.h != 0.0f || gacc.l != 0.0f)) atomicAdd(x + L.glob_col, ff_to_double(gacc));
  }
  __syncthreads();
  for (int i = threadIdx.x; i < L.n_instr; i += blockDim.x) {
    const double h = hist[i];
    if (h != 0.0) atomicAdd(x + L.instr_base + i, h);
  }
}

// ---------------------------------------------------------------------------
// aprod 2, attitude part over the knot-sorted copy: a warp walks its range of
// start knots; positions with start knot s add into knots s..s+3 of each
// axis. A sliding 4-knot window per axis lives in registers; knot s is final
// (for this warp) once bucket s is done and is added into x.
// ---------------------------------------------------------------------------
template <bool F32>
__device__ __forceinline__ ff att_val(const Layout& L, int t, int64_t p) {
  if constexpr (F32) {
    return ff{__ldcs(L.att_knot_f32 + (int64_t)t * L.n_rows + p), 0.0f};
  } else {
    const float2 a = __ldcs(L.att_knot_ff + (int64_t)t * L.n_rows + p);
    return ff{a.x, a.y};
  }
}

template <bool F32>
__global__ void __launch_bounds__(256) k_aprod2_att(Layout L, const double* __restrict__ y_knot,
                                                    double* __restrict__ x, const double* stop) {
  if (stop && *stop != 0.0) return;
  const int lane = threadIdx.x & 31;
  const int64_t gwarp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  if (gwarp >= L.n_att_warps) return;
  const int s_begin = L.att_warp_knot[gwarp], s_end = L.att_warp_knot[gwarp + 1];
  if (s_begin >= s_end) return;
  ff win[3][4];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int j = 0; j < 4; ++j) win[a][j] = ff_zero();
  const int64_t K = L.n_knots;
  for (int s = s_begin; s < s_end; ++s) {
    const int64_t p0 = L.knot_start[s], p1 = L.knot_start[s + 1];
    ff acc[12];
#pragma unroll
    for (int t = 0; t < 12; ++t) acc[t] = ff_zero();
    int64_t p = p0 + lane;
    for (; p + 32 < p1; p += 64) {
      const ff ua = ff_from_double(__ldcs(y_knot + p));
      const ff ub = ff_from_double(__ldcs(y_knot + p + 32));
#pragma unroll
      for (int t = 0; t < 12; ++t) {
        const ff va = att_val<F32>(L, t, p);
        const ff vb = att_val<F32>(L, t, p + 32);
        acc[t] = ff_add(acc[t], ff_add(ff_mul(va, ua), ff_mul(vb, ub)));
      }
    }
    if (p < p1) {
      const ff ua = ff_from_double(__ldcs(y_knot + p));
#pragma unroll
      for (int t = 0; t < 12; ++t) acc[t] = ff_add(acc[t], ff_mul(att_val<F32>(L, t, p), ua));
    }
#pragma unroll
    for (int t = 0; t < 12; ++t) acc[t] = ff_warp_sum(acc[t]);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int j = 0; j < 4; ++j) win[a][j] = ff_add(win[a][j], acc[4 * a + j]);
    // knot s is complete for this warp
    if (lane < 3) {
      const ff w0 = lane == 0 ? win[0][0] : lane == 1 ? win[1][0] : win[2][0];
      atomicAdd(x + L.att_base + lane * K + s, ff_to_double(w0));
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      win[a][0] = win[a][1];
      win[a][1] = win[a][2];
      win[a][2] = win[a][3];
      win[a][3] = ff_zero();
    }
  }
  // the three knots after the last bucket also received contributions
  if (lane < 3) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const ff wj = lane == 0 ? win[0][j] : lane == 1 ? win[1][j] : win[2][j];
      atomicAdd(x + L.att_base + lane * K + s_end + j, ff_to_double(wj));
    }
  }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
int cuda_status(cudaError_t e) { return e == cudaSuccess ? GSR_OK : GSR_E_CUDA; }

int launch_to_ff(const double* x, const double* scale, float2* out, int64_t n, cudaStream_t st) {
  if (n <= 0) return GSR_OK;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 148 * 8) blocks = 148 * 8;
  k_to_ff<<<blocks, 256, 0, st>>>(x, scale, out, n);
  return cuda_status(cudaGetLastError());
}

int launch_scatter_knot(gsr_system* sys, const double* y, double* y_knot, cudaStream_t st) {
  if (sys->L.n_rows <= 0) return GSR_OK;
  int blocks = (int)((sys->L.n_rows + 255) / 256);
  if (blocks > sys->num_sms * 8) blocks = sys->num_sms * 8;
  k_scatter_knot<<<blocks, 256, 0, st>>>(sys->L, y, y_knot);
  return cuda_status(cudaGetLastError());
}

int launch_aprod1(gsr_system* sys, int which_values, const float2* x_ff, double* y,
                  const double* coef_dev, double coef_host, double* y_knot, double* norm_slot,
                  const double* stop, cudaStream_t st) {
  const Layout& L = sys->L;
  if (L.n_tiles <= 0) {
    if (norm_slot) return cuda_status(cudaMemsetAsync(norm_slot, 0, sizeof(double), st));
    return GSR_OK;
  }
  int blocks = sys->num_sms * 4;
  const int64_t need = (L.n_tiles + 7) / 8;
  if (need < blocks) blocks = (int)need;
  if (which_values == GSR_VALUES_F32)
    k_aprod1<true><<<blocks, 256, 0, st>>>(L, x_ff, y, coef_dev, coef_host, y_knot, sys->S.red,
                                           sys->S.count, norm_slot, stop);
  else
    k_aprod1<false><<<blocks, 256, 0, st>>>(L, x_ff, y, coef_dev, coef_host, y_knot, sys->S.red,
                                            sys->S.count, norm_slot, stop);
  return cuda_status(cudaGetLastError());
}

int launch_aprod2(gsr_system* sys, int which_values, const double* y, const double* y_knot,
                  double* x, const double* stop, cudaStream_t st) {
  const Layout& L = sys->L;
  if (L.n_rows <= 0) return GSR_OK;
  cudaError_t e;
  // attitude part on the side stream, concurrent with the star-ordered part
  if ((e = cudaEventRecord(sys->ev_fork, st)) != cudaSuccess) return GSR_E_CUDA;
  if ((e = cudaStreamWaitEvent(sys->side, sys->ev_fork, 0)) != cudaSuccess) return GSR_E_CUDA;
  const int att_blocks = (L.n_att_warps + 7) / 8;
  if (att_blocks > 0) {
    if (which_values == GSR_VALUES_F32)
      k_aprod2_att<true><<<att_blocks, 256, 0, sys->side>>>(L, y_knot, x, stop);
    else
      k_aprod2_att<false><<<att_blocks, 256, 0, sys->side>>>(L, y_knot, x, stop);
    if ((e = cudaGetLastError()) != cudaSuccess) return GSR_E_CUDA;
  }
  if (which_values == GSR_VALUES_F32)
    k_aprod2_main<true><<<sys->main_ctas, sys->main_block, sys->hist_bytes, st>>>(L, y, x, stop);
  else
    k_aprod2_main<false><<<sys->main_ctas, sys->main_block, sys->hist_bytes, st>>>(L, y, x, stop);
  if ((e = cudaGetLastError()) != cudaSuccess) return GSR_E_CUDA;
  if ((e = cudaEventRecord(sys->ev_join, sys->side)) != cudaSuccess) return GSR_E_CUDA;
  if ((e = cudaStreamWaitEvent(st, sys->ev_join, 0)) != cudaSuccess) return GSR_E_CUDA;
  return GSR_OK;
}

int set_kernel_attributes(int hist_bytes) {
  cudaError_t e = cudaFuncSetAttribute(k_aprod2_main<false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, hist_bytes);
  if (e != cudaSuccess) return GSR_E_CUDA;
  e = cudaFuncSetAttribute(k_aprod2_main<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           hist_bytes);
  return cuda_status(e);
}

}  // namespace gsr
