// Multi-right-hand-side aprod 1 / aprod 2 and LSQR (k systems A x_j = b_j
// sharing A, e.g. Monte-Carlo perturbed observation vectors for covariances).
//
// aprod becomes a sparse-times-dense-block product that reads A once for all
// k vectors. Vectors are stored with the right-hand sides interleaved,
// Y[row][KP] and X[col][KP] (KP = k rounded up to a power of two <= 32), so
// that lanes run over right-hand sides: a warp is split into 32/KP "streams"
// of KP lanes; every stream walks rows (or knot-ordered positions, or
// instrumental entries) while each of its lanes handles one right-hand side.
// Coefficients are broadcast within a stream and every x / y access is a
// contiguous KP-wide vector. All arithmetic is float pairs as in the
// single-right-hand-side kernels. The instrumental histogram (n_instr x KP
// pairs) does not fit one block's shared memory, so blocks split the
// right-hand sides into chunks of KC (a tuning parameter).
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <vector>

#include "gsr_system.cuh"

namespace gsr {

namespace {

// x += hi + lo as two L2 reductions, each word widened exactly with integer
// instructions (no FP64 arithmetic on the SM).
__device__ __forceinline__ void red_ff_b(double* x, ff a) {
  if (a.h != 0.0f) atomicAdd(x, f2d_exact(a.h));
  if (a.l != 0.0f) atomicAdd(x, f2d_exact(a.l));
}

// Record accessors for row r_in (0..63) of a record (L1/L2-cached loads; the
// KP lanes of a stream read the same address).
__device__ __forceinline__ ff rv(const unsigned char* rec, int t, int r_in) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(rec + slot_offset<false>(t) +
                                                         (r_in >> 1) * 16 + (r_in & 1) * 8));
  return ff{v.x, v.y};
}
__device__ __forceinline__ int ri(const unsigned char* rec, int off, int r_in) {
  return __ldg(reinterpret_cast<const int*>(rec + off) + r_in);
}
__device__ __forceinline__ int rinstr(const unsigned char* rec, int k, int r_in) {
  return __ldg(reinterpret_cast<const unsigned short*>(rec + Rec<false>::INSTR_I + k * 128) +
               r_in);
}
__device__ __forceinline__ ff ldf(const float2* p) {
  const float2 a = __ldg(p);
  return ff{a.x, a.y};
}

// Arithmetic of the two precisions of the batched kernels. F32 = false: the
// float-pair products and sums of the FP64-accurate path. F32 = true: the
// FP32-value phase of a mixed-precision solve - coefficients from the FP32
// copy of A, only the high word of each vector entry, one FP32 multiply-add
// per product (the low words stay zero).
template <bool F32>
__device__ __forceinline__ ff fma_t(ff c, ff x, ff acc) {
  if constexpr (F32) return ff{__fmaf_rn(c.h, x.h, acc.h), 0.0f};
  else return ff_add(acc, ff_mul(c, x));
}
template <bool F32>
__device__ __forceinline__ ff add_t(ff a, ff b) {
  if constexpr (F32) return ff{__fadd_rn(a.h, b.h), 0.0f};
  else return ff_add(a, b);
}
template <bool F32>
__device__ __forceinline__ ff mul_t(ff a, ff b) {
  if constexpr (F32) return ff{__fmul_rn(a.h, b.h), 0.0f};
  else return ff_mul(a, b);
}
template <bool F32>
__device__ __forceinline__ ff norm_t(ff a) {
  if constexpr (F32) return a;
  else return ff_norm(a);
}
template <bool F32>
__device__ __forceinline__ ff ldv(const float2* p) {
  if constexpr (F32) return ff{__ldg(reinterpret_cast<const float*>(p)), 0.0f};
  else return ldf(p);
}
template <bool F32>
__device__ __forceinline__ ff pair_t(float2 v) {
  if constexpr (F32) return ff{v.x, 0.0f};
  else return ff{v.x, v.y};
}
// Coefficient of slot t, row r_in, of a record of the given precision.
template <bool F32>
__device__ __forceinline__ ff rvt(const unsigned char* rec, int t, int r_in) {
  if constexpr (F32)
    return ff{__ldg(reinterpret_cast<const float*>(rec + slot_offset<true>(t)) + r_in), 0.0f};
  else return rv(rec, t, r_in);
}
template <bool F32>
__device__ __forceinline__ int rinstr_t(const unsigned char* rec, int k, int r_in) {
  return __ldg(reinterpret_cast<const unsigned short*>(rec + Rec<F32>::INSTR_I + k * 128) + r_in);
}
template <bool F32>
__device__ __forceinline__ const unsigned char* rec_at(const Layout& L, int64_t r) {
  return (F32 ? L.rec_f32 : L.rec_ff) + r * Rec<F32>::BYTES;
}

// Per-right-hand-side deterministic grid reduction of NV values per lane:
// lanes of a block with the same j = threadIdx.x % KP are summed, blocks store
// part[(block*NV + v)*KP + j], and the last block adds them into tot[v*32 + j]
// (shared, visible to the whole last block on return true): thread group q of
// blockDim/KP groups sums blocks q, q + groups, ... in order, and the group
// sums are added in group order (a fixed order, independent of timing).
// Blocks of at most 256 threads.
template <int KP, int NV>
__device__ bool grid_sum_kv(const double* v, double* part, unsigned int* counter, double* tot) {
  __shared__ double sh[NV][8][32];
  __shared__ double gs[NV][256];
  __shared__ int is_last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int a = 0; a < NV; ++a) {
    double x = v[a];
#pragma unroll
    for (int m = 16; m >= KP; m >>= 1) x += __shfl_xor_sync(0xffffffffu, x, m);
    if (lane < KP) sh[a][wid][lane] = x;
  }
  __syncthreads();
  if (threadIdx.x < KP) {
#pragma unroll
    for (int a = 0; a < NV; ++a) {
      double x = 0.0;
      for (int w = 0; w < nw; ++w) x += sh[a][w][threadIdx.x];
      part[((size_t)blockIdx.x * NV + a) * KP + threadIdx.x] = x;
    }
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  {
    const int groups = (int)blockDim.x / KP, q = (int)threadIdx.x / KP,
              j = (int)threadIdx.x % KP;
#pragma unroll
    for (int a = 0; a < NV; ++a) {
      double x = 0.0;
      for (unsigned int b = q; b < gridDim.x; b += groups)
        x += __ldcg(part + ((size_t)b * NV + a) * KP + j);
      gs[a][threadIdx.x] = x;
    }
    __syncthreads();
    if (threadIdx.x < KP) {
#pragma unroll
      for (int a = 0; a < NV; ++a) {
        double x = 0.0;
        for (int g = 0; g < groups; ++g) x += gs[a][g * KP + threadIdx.x];
        tot[a * 32 + threadIdx.x] = x;
      }
    }
  }
  if (threadIdx.x == 0) *counter = 0u;
  __syncthreads();
  return true;
}

// ---------------------------------------------------------------------------
// aprod 1, k right-hand sides: Y[r][j] = coef[j] Y[r][j] + (A X_j)[r]; optional
// knot-order copy and per-right-hand-side ||Y_j||^2 into norm_out[j]. A warp
// takes a record; its 32/KP streams take contiguous slices of the 64 rows.
// ---------------------------------------------------------------------------
template <int KP, bool F32>
__global__ void __launch_bounds__(256) k_aprod1_b(Layout L, const float2* __restrict__ X,
                                                  float2* __restrict__ Y,
                                                  const double* __restrict__ coef,
                                                  float2* __restrict__ Yk, double* part,
                                                  unsigned int* counter, double* norm_out,
                                                  const double* stop) {
  if (stop && *stop != 0.0) return;
  __shared__ double tot[32];
  constexpr int S = 32 / KP, RPS = REC_ROWS / S;
  const int lane = threadIdx.x & 31, q = lane / KP, j = lane % KP;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const ff cf = coef ? ff_from_double(coef[j]) : ff{1.0f, 0.0f};
  const bool glob = L.n_glob == 1;
  const int64_t K = L.n_knots;
  ff nrm = ff_zero();
  for (int64_t r = gw; r < L.n_recs; r += nw) {
    const unsigned char* rec = rec_at<F32>(L, r);
    // The record's column indices, two rows per lane, loaded up front so the
    // x gathers of a row wait for a shuffle rather than a load: register h of
    // lane (q, p) holds row q * RPS + h * KP + p (RPS = 2 KP), so at step
    // (h, p) every stream reads register h of lane q * KP + p.
    int pst[2], psk[2], ppos[2], pin[2][3];  // instrumental indices packed in pairs
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int rr = q * RPS + h * KP + j;
      pst[h] = ri(rec, Rec<F32>::STAR, rr);
      psk[h] = ri(rec, Rec<F32>::ATT_S, rr);
      ppos[h] = Yk ? ri(rec, Rec<F32>::POS, rr) : 0;
#pragma unroll
      for (int k = 0; k < 3; ++k)
        pin[h][k] = rinstr_t<F32>(rec, 2 * k, rr) | (rinstr_t<F32>(rec, 2 * k + 1, rr) << 16);
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
#pragma unroll 2
      for (int p = 0; p < KP; ++p) {
        const int src = q * KP + p;
        const int r_in = q * RPS + h * KP + p;
        const int64_t row = r * REC_ROWS + r_in;
        const int st = __shfl_sync(0xffffffffu, pst[h], src);
        const int sk = __shfl_sync(0xffffffffu, psk[h], src);
        const int pos = __shfl_sync(0xffffffffu, ppos[h], src);
        int ins[6];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const int v = __shfl_sync(0xffffffffu, pin[h][k], src);
          ins[2 * k] = v & 0xffff;
          ins[2 * k + 1] = (int)((unsigned)v >> 16);
        }
        if (row >= L.n_rows) continue;  // padding rows of the last record
        ff a0 = ff_zero(), a1 = ff_zero(), a2 = ff_zero(), a3 = ff_zero(), a4 = ff_zero();
#pragma unroll
        for (int t = 0; t < 5; ++t)
          a0 = fma_t<F32>(rvt<F32>(rec, t, r_in), ldv<F32>(X + (5 * (int64_t)st + t) * KP + j), a0);
#pragma unroll
        for (int i4 = 0; i4 < 4; ++i4) {
          a1 = fma_t<F32>(rvt<F32>(rec, 5 + i4, r_in),
                          ldv<F32>(X + (L.att_base + sk + i4) * KP + j), a1);
          a2 = fma_t<F32>(rvt<F32>(rec, 9 + i4, r_in),
                          ldv<F32>(X + (L.att_base + K + sk + i4) * KP + j), a2);
          a3 = fma_t<F32>(rvt<F32>(rec, 13 + i4, r_in),
                          ldv<F32>(X + (L.att_base + 2 * K + sk + i4) * KP + j), a3);
        }
#pragma unroll
        for (int k = 0; k < 6; ++k)
          a4 = fma_t<F32>(rvt<F32>(rec, 17 + k, r_in),
                          ldv<F32>(X + (L.instr_base + ins[k]) * KP + j), a4);
        if (glob) a4 = fma_t<F32>(rvt<F32>(rec, 23, r_in), ldv<F32>(X + L.glob_col * KP + j), a4);
        const ff acc = add_t<F32>(add_t<F32>(add_t<F32>(a0, a1), add_t<F32>(a2, a3)), a4);
        const ff yo = pair_t<F32>(Y[row * KP + j]);
        const ff yn = norm_t<F32>(add_t<F32>(mul_t<F32>(cf, yo), acc));
        Y[row * KP + j] = make_float2(yn.h, yn.l);
        if (Yk) Yk[(int64_t)pos * KP + j] = make_float2(yn.h, yn.l);
        nrm = add_t<F32>(nrm, mul_t<F32>(yn, yn));
      }
    }
  }
  const double nv = ff_to_double(nrm);
  if (norm_out && grid_sum_kv<KP, 1>(&nv, part, counter, tot) && threadIdx.x < KP)
    norm_out[threadIdx.x] = tot[threadIdx.x];
}

// ---------------------------------------------------------------------------
// aprod 2, k right-hand sides, astrometric + global part: a stream walks a
// slice of a record's rows keeping per-star sums; a finished (or slice-ending)
// run is added into X with L2 reductions (KP-wide, contiguous).
// ---------------------------------------------------------------------------
template <int KP, bool F32>
__global__ void __launch_bounds__(256) k_aprod2_astro_b(Layout L, const float2* __restrict__ Y,
                                                        double* __restrict__ X,
                                                        const double* stop) {
  if (stop && *stop != 0.0) return;
  constexpr int S = 32 / KP, RPS = REC_ROWS / S;
  const int lane = threadIdx.x & 31, q = lane / KP, j = lane % KP;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const bool glob = L.n_glob == 1;
  ff g = ff_zero();
  for (int64_t r = gw; r < L.n_recs; r += nw) {
    const unsigned char* rec = rec_at<F32>(L, r);
    int cur = -1;
    ff a[5];
#pragma unroll
    for (int t = 0; t < 5; ++t) a[t] = ff_zero();
    for (int i = 0; i < RPS; ++i) {
      const int r_in = q * RPS + i;
      const int64_t row = r * REC_ROWS + r_in;
      if (row >= L.n_rows) break;
      const int st = ri(rec, Rec<F32>::STAR, r_in);
      if (st != cur) {
        if (cur >= 0)
#pragma unroll
          for (int t = 0; t < 5; ++t) red_ff_b(X + (5 * (int64_t)cur + t) * KP + j, a[t]);
#pragma unroll
        for (int t = 0; t < 5; ++t) a[t] = ff_zero();
        cur = st;
      }
      const ff u = pair_t<F32>(__ldcs(Y + row * KP + j));
#pragma unroll
      for (int t = 0; t < 5; ++t) a[t] = fma_t<F32>(rvt<F32>(rec, t, r_in), u, a[t]);
      if (glob) g = fma_t<F32>(rvt<F32>(rec, 23, r_in), u, g);
    }
    if (cur >= 0)
#pragma unroll
      for (int t = 0; t < 5; ++t) red_ff_b(X + (5 * (int64_t)cur + t) * KP + j, a[t]);
  }
  if (glob) {
#pragma unroll
    for (int m = 16; m >= KP; m >>= 1) g = add_t<F32>(g, ff_shfl_xor(g, m));
    if (q == 0) red_ff_b(X + L.glob_col * KP + j, g);
  }
}

// ---------------------------------------------------------------------------
// aprod 2, k right-hand sides, attitude part: a warp walks its start-knot
// range; within a bucket the streams split the positions, then sums are joined
// across streams and the 4-knot window per axis advances as in the single form.
// ---------------------------------------------------------------------------
constexpr int ATT_B_SPLIT = 2;  // warps per knot range of the single-vector partition
constexpr int VEC_U = 4;        // elements per thread per step of the vector kernels

template <int KP, bool F32>
__global__ void __launch_bounds__(256, 2) k_aprod2_att_b(Layout L, const float2* __restrict__ Yk,
                                                         double* __restrict__ X,
                                                         const double* stop) {
  if (stop && *stop != 0.0) return;
  constexpr int S = 32 / KP;
  const int lane = threadIdx.x & 31, q = lane / KP, j = lane % KP;
  // ATT_B_SPLIT warps share each knot range of the single-vector partition
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t gwarp = gw / ATT_B_SPLIT;
  const int part = (int)(gw % ATT_B_SPLIT);
  if (gwarp >= L.n_att_warps) return;
  const int r0 = L.att_warp_knot[gwarp], r1 = L.att_warp_knot[gwarp + 1];
  const int s_begin = r0 + (int)(((int64_t)(r1 - r0) * part) / ATT_B_SPLIT);
  const int s_end = r0 + (int)(((int64_t)(r1 - r0) * (part + 1)) / ATT_B_SPLIT);
  if (s_begin >= s_end) return;
  const int64_t K = L.n_knots;
  ff win[3][4];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int i = 0; i < 4; ++i) win[a][i] = ff_zero();
  const int64_t kb_w = L.n_knots - 2;
  // the float-pair copy of Y is blocked when n_kblk > 1, the FP32 one never
  const bool blk = !F32 && L.n_kblk > 1;
  const int nbk = blk ? L.n_kblk : 1;
  for (int s = s_begin; s < s_end; ++s) {
    ff acc[12];
#pragma unroll
    for (int t = 0; t < 12; ++t) acc[t] = ff_zero();
    constexpr int U = 2;  // positions per stream per step, all loads issued first
    // the rows of knot s: one run of the knot order (coefficients, from g0) and
    // of the copy of Y, or one segment per row block of its blocked copy
    int64_t g0 = L.knot_start[s];
    for (int bk = 0; bk < nbk; ++bk) {
      const int64_t p0 = blk ? L.kb_start[bk * kb_w + s] : g0;
      const int64_t n = blk ? L.kb_start[bk * kb_w + s + 1] - p0 : L.knot_start[s + 1] - g0;
      for (int64_t ib = q; ib < n; ib += U * S) {
        ff u[U];
        ff v[12][U];
#pragma unroll
        for (int i = 0; i < U; ++i) {
          const int64_t k = ib + (int64_t)i * S;
          const bool in = k < n;
          const int64_t p = p0 + k, g = g0 + k;
          u[i] = in ? pair_t<F32>(__ldcs(Yk + p * KP + j)) : ff_zero();
#pragma unroll
          for (int t = 0; t < 12; ++t) {
            if constexpr (F32)
              v[t][i] = ff{in ? __ldg(L.att_knot_f32 + (int64_t)t * L.n_rows + g) : 0.0f, 0.0f};
            else
              v[t][i] = in ? ldf(L.att_knot_ff + (int64_t)t * L.n_rows + g) : ff_zero();
          }
        }
#pragma unroll
        for (int t = 0; t < 12; ++t) {
          ff sum = mul_t<F32>(v[t][0], u[0]);
#pragma unroll
          for (int i = 1; i < U; ++i) sum = fma_t<F32>(v[t][i], u[i], sum);
          acc[t] = add_t<F32>(acc[t], sum);
        }
      }
      g0 += n;
    }
#pragma unroll
    for (int t = 0; t < 12; ++t)
#pragma unroll
      for (int m = 16; m >= KP; m >>= 1) acc[t] = add_t<F32>(acc[t], ff_shfl_xor(acc[t], m));
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int i = 0; i < 4; ++i) win[a][i] = add_t<F32>(win[a][i], acc[4 * a + i]);
    if (q == 0)
#pragma unroll
      for (int a = 0; a < 3; ++a) red_ff_b(X + (L.att_base + a * K + s) * KP + j, win[a][0]);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      win[a][0] = win[a][1];
      win[a][1] = win[a][2];
      win[a][2] = win[a][3];
      win[a][3] = ff_zero();
    }
  }
  if (q == 0)
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int i = 0; i < 3; ++i)
        red_ff_b(X + (L.att_base + a * K + s_end + i) * KP + j, win[a][i]);
}

// ---------------------------------------------------------------------------
// aprod 2, k right-hand sides, instrumental part. A histogram of all KP
// right-hand sides per instrumental column does not fit one block's shared
// memory, so the entries are regrouped instead: rows are cut into tiles of
// 2^tile_log rows and the entries of every (tile, column) bucket are stored
// contiguously (built once per system, InstrCsc). A stream of KP lanes owns a
// bucket: it sums coef * Y[row][j] over the bucket in registers (no shared
// memory, no barriers, no races) and adds the sum into X with one L2
// reduction per lane. Buckets are taken tile-major so that the Y rows of the
// tiles in flight stay in L2 while their 6 entries per row are gathered.
// ---------------------------------------------------------------------------
struct InstrCsc {
  int tile_log = 0;
  int64_t n_tiles = 0, n_bins = 0;
  int64_t* off = nullptr;        // [n_tiles * n_bins + 1] first entry of each bucket
  int32_t* row = nullptr;        // [6 n_rows] row of each entry
  float2* val = nullptr;         // [6 n_rows] coefficient (pair)
  unsigned int* cnt = nullptr;   // [n_tiles * n_bins] build scratch
  int64_t cap_buckets = 0;
};

__global__ void k_csc_count(Layout L, int tile_log, int64_t n_bins, unsigned int* __restrict__ cnt) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < L.n_rows;
       r += (int64_t)gridDim.x * blockDim.x) {
    const unsigned char* rec = L.rec_ff + (r >> 6) * Rec<false>::BYTES;
    const int64_t t = (r >> tile_log) * n_bins;
#pragma unroll
    for (int k = 0; k < 6; ++k) atomicAdd(cnt + t + rinstr(rec, k, (int)(r & 63)), 1u);
  }
}

// Exclusive prefix sum of n counts into off[0..n] (one block).
__global__ void k_csc_scan(const unsigned int* __restrict__ cnt, int64_t n, int64_t* __restrict__ off) {
  __shared__ int64_t part[1024];
  const int64_t per = (n + blockDim.x - 1) / blockDim.x;
  const int64_t a0 = (int64_t)threadIdx.x * per;
  const int64_t a = a0 < n ? a0 : n, b = a + per < n ? a + per : n;
  int64_t sum = 0;
  for (int64_t i = a; i < b; ++i) sum += cnt[i];
  part[threadIdx.x] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t run = 0;
    for (unsigned int t = 0; t < blockDim.x; ++t) {
      const int64_t v = part[t];
      part[t] = run;
      run += v;
    }
    off[n] = run;
  }
  __syncthreads();
  int64_t run = part[threadIdx.x];
  for (int64_t i = a; i < b; ++i) {
    off[i] = run;
    run += cnt[i];
  }
}

// Scatter the entries into their buckets (cnt reused as zeroed cursors; the
// order inside a bucket follows the atomics).
__global__ void k_csc_fill(Layout L, int tile_log, int64_t n_bins, const int64_t* __restrict__ off,
                           unsigned int* __restrict__ cur, int32_t* __restrict__ row,
                           float2* __restrict__ val) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < L.n_rows;
       r += (int64_t)gridDim.x * blockDim.x) {
    const unsigned char* rec = L.rec_ff + (r >> 6) * Rec<false>::BYTES;
    const int r_in = (int)(r & 63);
    const int64_t t = (r >> tile_log) * n_bins;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const int64_t bkt = t + rinstr(rec, k, r_in);
      const int64_t pos = off[bkt] + atomicAdd(cur + bkt, 1u);
      row[pos] = (int32_t)r;
      const ff v = rv(rec, 17 + k, r_in);
      val[pos] = make_float2(v.h, v.l);
    }
  }
}

template <int KP, bool F32>
__global__ void __launch_bounds__(256) k_aprod2_instr_csc(Layout L, const int64_t* __restrict__ off,
                                                          const int32_t* __restrict__ erow,
                                                          const float2* __restrict__ eval,
                                                          int64_t n_buckets, int64_t n_bins,
                                                          const float2* __restrict__ Y,
                                                          double* __restrict__ X,
                                                          const double* stop) {
  if (stop && *stop != 0.0) return;
  constexpr int S = 32 / KP;
  const int lane = threadIdx.x & 31, q = lane / KP, j = lane % KP;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u0 = gw * S; u0 < n_buckets; u0 += nw * S) {
    const int64_t u = u0 + q;
    if (u >= n_buckets) continue;
    const int64_t e0 = off[u], e1 = off[u + 1];
    if (e0 == e1) continue;
    ff acc = ff_zero();
    constexpr int U = 4;  // entries per step, loads first
    int64_t e = e0;
    for (; e + U <= e1; e += U) {
      int r[U];
      float2 v[U], y[U];
#pragma unroll
      for (int i = 0; i < U; ++i) {
        r[i] = __ldg(erow + e + i);
        v[i] = __ldg(eval + e + i);
      }
#pragma unroll
      for (int i = 0; i < U; ++i) y[i] = __ldg(Y + (int64_t)r[i] * KP + j);
#pragma unroll
      for (int i = 0; i < U; ++i) acc = fma_t<F32>(pair_t<F32>(v[i]), pair_t<F32>(y[i]), acc);
    }
    for (; e < e1; ++e) {
      const float2 v = __ldg(eval + e);
      const float2 y = __ldg(Y + (int64_t)__ldg(erow + e) * KP + j);
      acc = fma_t<F32>(pair_t<F32>(v), pair_t<F32>(y), acc);
    }
    red_ff_b(X + (L.instr_base + u % n_bins) * KP + j, acc);
  }
}

// ---------------------------------------------------------------------------
// Conversions between the caller layout [n][k] (double) and [n][KP] pairs.
// ---------------------------------------------------------------------------
// in [n][k] -> 2^-cexp[i] in as pairs [n][KP] (padding lanes 0); an entry
// outside the vector band sets *guard.
__global__ void k_pack_ff(const double* __restrict__ in, int k, int KP, int64_t n,
                          const int16_t* __restrict__ cexp, double* guard,
                          float2* __restrict__ out, int neg) {
  bool out_of_band = false;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * KP;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / KP;
    const int j = (int)(e % KP);
    double v = j < k ? in[i * k + j] : 0.0;
    if (cexp) v = ldexp(v, -(int)cexp[i]);
    if (neg) v = -v;
    if (!vec_in_band(v)) out_of_band = true;
    const ff f = ff_from_double(v);
    out[e] = make_float2(f.h, f.l);
  }
  if (guard && out_of_band) *guard = 1.0;
}
// Y [n_rows][k] -> 2^-e_i Y as pairs in row order and knot order.
__global__ void k_pack_ff_knot(Layout L, const double* __restrict__ in, int k, int KP,
                               double* guard, float2* __restrict__ out,
                               float2* __restrict__ outk) {
  bool out_of_band = false;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < L.n_rows * KP;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / KP;
    const int j = (int)(e % KP);
    double v = j < k ? in[i * k + j] : 0.0;
    if (L.row_exp) v = ldexp(v, -(int)L.row_exp[i]);
    if (!vec_in_band(v)) out_of_band = true;
    const ff f = ff_from_double(v);
    out[e] = make_float2(f.h, f.l);
    outk[(int64_t)L.pos[i] * KP + j] = make_float2(f.h, f.l);
  }
  if (guard && out_of_band) *guard = 1.0;
}
// Y[n][k] += 2^-e_i U (the pairs of a batched aprod 1), unless *guard.
__global__ void k_unpack_add(const float2* __restrict__ in, int k, int KP, int64_t n,
                             const int16_t* __restrict__ rexp, const double* guard,
                             double* __restrict__ out) {
  if (guard && *guard != 0.0) return;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * k;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / k;
    const float2 v = in[i * KP + e % k];
    const double a = ff_to_double(ff{v.x, v.y});
    out[e] += rexp ? ldexp(a, -(int)rexp[i]) : a;
  }
}
// X[n][k] += 2^-g_i Z (a batched aprod 2 accumulator), unless *guard.
__global__ void k_add_cols(const double* __restrict__ in, int k, int KP, int64_t n,
                           const int16_t* __restrict__ cexp, const double* guard,
                           double* __restrict__ out) {
  if (guard && *guard != 0.0) return;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * k;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / k;
    const double a = in[i * KP + e % k];
    out[e] += cexp ? ldexp(a, -(int)cexp[i]) : a;
  }
}
__global__ void k_zero_d(double* __restrict__ a, int64_t n, const double* stop) {
  if (stop && *stop != 0.0) return;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    a[e] = 0.0;
}

// ---------------------------------------------------------------------------
// Batched LSQR. Per-right-hand-side scalars at sc[s*KP + j] (s an enum BS
// slot), global words after them. A right-hand side whose stopping test fired
// is frozen: its coefficient and D v are zeroed so its u stays 0, and its x
// and w stop changing; all kernels return at once when every one stopped.
// ---------------------------------------------------------------------------
enum BS {
  B_ALPHA = 0, B_BETA, B_RHOBAR, B_PHIBAR, B_ANORM2, B_DDNORM, B_BNORM, B_RHO, B_C, B_T1, B_T2,
  B_RNORM, B_ARNORM, B_ACOND, B_XNORM, B_ITN, B_ISTOP, B_DONE, B_UNORM2, B_COEF, B_XREF2,
  B_BEXP,  // right-hand side j is solved as 2^-s_j b_j (largest entry in [1, 2))
  B_COUNT
};
enum BG { G_ALLDONE = 0, G_ATOL, G_BTOL, G_CTOL, G_ITNLIM, G_K, G_ITER, G_COUNT };

// Largest binary exponent of each right-hand side into mx[j] (atomicMax, mx
// preset very negative); a NaN or Inf sets *bad. LSQR is invariant under
// b_j -> 2^-s b_j, so every right-hand side is solved with its largest entry
// in [1, 2) and its x and residual norms are scaled back.
template <int KP>
__global__ void __launch_bounds__(256) k_maxexp_b(const double* __restrict__ B, int k, int64_t n,
                                                  int* mx, double* bad) {
  const int j = (int)(threadIdx.x % KP);
  int m = INT_MIN;
  bool nonfinite = false;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * KP;
       e += (int64_t)gridDim.x * blockDim.x) {
    if (j >= k) continue;
    const double v = B[(e / KP) * k + j];
    if (!isfinite(v)) nonfinite = true;
    else if (v != 0.0) m = max(m, ilogb(v));
  }
#pragma unroll
  for (int o = 16; o >= KP; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) < KP && j < k && m != INT_MIN) atomicMax(mx + j, m);
  if (nonfinite) *bad = 1.0;
}

template <int KP>
__global__ void __launch_bounds__(256) k_init_b(Layout L, const double* __restrict__ B, int k,
                                                const int* bexp, float2* __restrict__ U,
                                                float2* __restrict__ Uk,
                                                const int32_t* __restrict__ kp, double* sc,
                                                double* part, unsigned int* counter) {
  __shared__ double tot[32];
  double s2 = 0.0;
  const int jt = (int)(threadIdx.x % KP);
  const int sb = jt < k && bexp[jt] > -4000 ? bexp[jt] : 0;
  if (blockIdx.x == 0 && threadIdx.x < KP) sc[B_BEXP * KP + jt] = sb;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < L.n_rows * KP;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / KP;
    const int j = (int)(e % KP);
    const double v = j < k ? ldexp(B[i * k + j], -sb) : 0.0;
    const ff f = ff_from_double(v);
    U[e] = make_float2(f.h, f.l);
    Uk[(int64_t)kp[i] * KP + j] = make_float2(f.h, f.l);
    s2 = __fma_rn(v, v, s2);
  }
  if (grid_sum_kv<KP, 1>(&s2, part, counter, tot) && threadIdx.x < KP)
    sc[B_UNORM2 * KP + threadIdx.x] = tot[threadIdx.x];
}

// ||x_ref_j||^2 for the error history.
template <int KP>
__global__ void __launch_bounds__(256) k_xref2_b(int64_t n, const double* __restrict__ xr,
                                                 double* sc, double* part, unsigned int* counter) {
  __shared__ double tot[32];
  double s2 = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * KP;
       e += (int64_t)gridDim.x * blockDim.x)
    s2 = __fma_rn(xr[e], xr[e], s2);
  if (grid_sum_kv<KP, 1>(&s2, part, counter, tot) && threadIdx.x < KP)
    sc[B_XREF2 * KP + threadIdx.x] = tot[threadIdx.x];
}

template <int KP>
__global__ void __launch_bounds__(256) k_vec_a_b(int64_t n, const float2* __restrict__ d,
                                                 const double* __restrict__ Z,
                                                 float2* __restrict__ V, double* sc, double* part,
                                                 unsigned int* counter, int first) {
  __shared__ double tot[32];
  const double* g = sc + B_COUNT * KP;
  if (g[G_ALLDONE] != 0.0) return;
  const int j = threadIdx.x % KP;
  const double beta = sqrt(sc[B_UNORM2 * KP + j]);
  const ff ib = ff_from_double(beta > 0.0 ? 1.0 / beta : 0.0), nbeta = ff_from_double(-beta);
  const bool frozen = sc[B_DONE * KP + j] != 0.0;
  ff s2f = ff_zero();
  if (!frozen) {
    // VEC_U elements per thread per step, all loads issued first (latency)
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e0 < n * KP;
         e0 += VEC_U * stride) {
      float2 dd[VEC_U], vv[VEC_U];
      double zz[VEC_U];
#pragma unroll
      for (int u = 0; u < VEC_U; ++u) {
        const int64_t e = e0 + u * stride;
        if (e < n * KP) {
          dd[u] = d[e / KP];
          zz[u] = Z[e];
          if (!first) vv[u] = V[e];
        }
      }
#pragma unroll
      for (int u = 0; u < VEC_U; ++u) {
        const int64_t e = e0 + u * stride;
        if (e >= n * KP) continue;
        ff t = ff_mul(ff_norm(ff_mul(ff{dd[u].x, dd[u].y}, ff_from_double(zz[u]))), ib);
        if (!first) t = ff_add(t, ff_mul(nbeta, ff{vv[u].x, vv[u].y}));
        t = ff_norm(t);
        V[e] = make_float2(t.h, t.l);
        s2f = ff_add(s2f, ff_mul(t, t));
      }
    }
  }
  const double s2 = ff_to_double(s2f);
  if (!grid_sum_kv<KP, 1>(&s2, part, counter, tot) || threadIdx.x >= KP) return;
  // last block: plane rotation of right-hand side jj (Paige-Saunders)
  const int jj = threadIdx.x;
  if (jj >= (int)g[G_K] || sc[B_DONE * KP + jj] != 0.0) return;
  const double be = sqrt(sc[B_UNORM2 * KP + jj]);
  const double alpha = sqrt(tot[jj]);
  if (first) {
    sc[B_BETA * KP + jj] = be;
    sc[B_BNORM * KP + jj] = be;
    sc[B_ALPHA * KP + jj] = alpha;
    sc[B_RHOBAR * KP + jj] = alpha;
    sc[B_PHIBAR * KP + jj] = be;
    sc[B_RNORM * KP + jj] = be;
    sc[B_ARNORM * KP + jj] = alpha * be;
    sc[B_COEF * KP + jj] = be > 0.0 ? -alpha / be : 0.0;
    if (alpha * be == 0.0) {  // b_j = 0 or A^T b_j = 0: x_j = 0
      sc[B_ISTOP * KP + jj] = 0.0;
      sc[B_DONE * KP + jj] = 1.0;
      sc[B_COEF * KP + jj] = 0.0;
    }
    return;
  }
  const double alpha_old = sc[B_ALPHA * KP + jj];
  sc[B_ANORM2 * KP + jj] += alpha_old * alpha_old + be * be;
  const double rhobar = sc[B_RHOBAR * KP + jj], phibar = sc[B_PHIBAR * KP + jj];
  const double rho = sqrt(rhobar * rhobar + be * be);
  const double c = rhobar / rho, s = be / rho;
  const double theta = s * alpha;
  sc[B_RHO * KP + jj] = rho;
  sc[B_C * KP + jj] = c;
  sc[B_RHOBAR * KP + jj] = -c * alpha;
  sc[B_PHIBAR * KP + jj] = s * phibar;
  sc[B_T1 * KP + jj] = c * phibar / rho;
  sc[B_T2 * KP + jj] = -theta / rho;
  sc[B_BETA * KP + jj] = be;
  sc[B_ALPHA * KP + jj] = alpha;
  sc[B_COEF * KP + jj] = be > 0.0 ? -alpha / be : 0.0;
}

template <int KP>
__global__ void __launch_bounds__(256) k_vec_b_b(int64_t n, const float2* __restrict__ d,
                                                 float2* __restrict__ V, float2* __restrict__ W,
                                                 float2* __restrict__ XZ,
                                                 float2* __restrict__ Vff,
                                                 const double* __restrict__ xref,
                                                 const double* __restrict__ xoff,
                                                 const int16_t* __restrict__ cexp, double* sc,
                                                 double* part, unsigned int* counter, int first,
                                                 double* err_hist) {
  __shared__ double tot[4 * 32];
  double* g = sc + B_COUNT * KP;
  if (g[G_ALLDONE] != 0.0) return;
  const int j = threadIdx.x % KP;
  const int sb = (int)sc[B_BEXP * KP + j];
  double x2d = 0.0;
  const bool frozen = sc[B_DONE * KP + j] != 0.0 || j >= (int)g[G_K];
  const double alpha = sc[B_ALPHA * KP + j];
  const ff ia = ff_from_double(alpha > 0.0 ? 1.0 / alpha : 0.0);
  const ff irho = ff_from_double(first ? 1.0 : 1.0 / sc[B_RHO * KP + j]);
  const ff t1 = ff_from_double(first ? 0.0 : sc[B_T1 * KP + j]);
  const ff t2 = ff_from_double(first ? 0.0 : sc[B_T2 * KP + j]);
  ff dk2f = ff_zero(), x2f = ff_zero(), z2f = ff_zero();  // ||d_k||^2, ||x||^2, ||z||^2
  double e2 = 0.0;                       // ||x - x_ref||^2
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e0 < n * KP;
       e0 += VEC_U * stride) {
    float2 dv[VEC_U], vv[VEC_U], wv[VEC_U], xv_[VEC_U];
#pragma unroll
    for (int u = 0; u < VEC_U; ++u) {
      const int64_t e = e0 + u * stride;
      if (e < n * KP) {
        dv[u] = d[e / KP];
        if (!frozen) vv[u] = V[e];
        if (!first) {
          if (!frozen) wv[u] = W[e];
          xv_[u] = XZ[e];
        }
      }
    }
#pragma unroll
    for (int u = 0; u < VEC_U; ++u) {
      const int64_t e = e0 + u * stride;
      if (e >= n * KP) continue;
      const float2 djf = dv[u];
      const ff dj = ff{djf.x, djf.y};
      ff xv = ff_zero();
      if (frozen) {
        Vff[e] = make_float2(0.f, 0.f);
        if (!first) {
          const float2 xf = xv_[u];
          xv = ff_norm(ff_mul(dj, ff{xf.x, xf.y}));
        }
      } else {
        const float2 vf = vv[u];
        const ff vn = ff_norm(ff_mul(ff{vf.x, vf.y}, ia));
        if (first) {
          W[e] = make_float2(vn.h, vn.l);
          XZ[e] = make_float2(0.f, 0.f);
        } else {
          const float2 wf = wv[u], xf = xv_[u];
          const ff wj = ff{wf.x, wf.y};
          const ff dk = ff_mul(wj, irho);
          dk2f = ff_add(dk2f, ff_mul(dk, dk));
          const ff xn = ff_norm(ff_add(ff{xf.x, xf.y}, ff_mul(t1, wj)));
          XZ[e] = make_float2(xn.h, xn.l);
          z2f = ff_add(z2f, ff_mul(xn, xn));
          const ff wn = ff_norm(ff_add(vn, ff_mul(t2, wj)));
          W[e] = make_float2(wn.h, wn.l);
          xv = ff_norm(ff_mul(dj, xn));
        }
        V[e] = make_float2(vn.h, vn.l);
        const ff f = ff_norm(ff_mul(dj, vn));
        Vff[e] = make_float2(f.h, f.l);
      }
      // x = 2^g D' z: in FP64 when the system has column exponents
      double xd = 0.0;
      if (cexp) {
        xd = ldexp(ff_to_double(xv), (int)cexp[e / KP]);
        x2d = __fma_rn(xd, xd, x2d);
      } else {
        x2f = ff_add(x2f, ff_mul(xv, xv));
        if (xref) xd = ff_to_double(xv);
      }
      if (xref) {  // xoff: the first phase's solution in a mixed-precision solve
        const double ex = ldexp(xd, sb) + (xoff ? xoff[e] : 0.0) - xref[e];
        e2 = __fma_rn(ex, ex, e2);
      }
    }
  }
  double acc[4] = {ff_to_double(dk2f), ff_to_double(x2f) + x2d, e2, ff_to_double(z2f)};
  if (!grid_sum_kv<KP, 4>(acc, part, counter, tot)) return;
  const int K = (int)g[G_K];
  if (first) {
    if (threadIdx.x == 0) {
      bool all = true;
      for (int q = 0; q < K; ++q) all = all && sc[B_DONE * KP + q] != 0.0;
      if (all) g[G_ALLDONE] = 1.0;
    }
    return;
  }
  const int64_t it = (int64_t)g[G_ITER];
  const int jj = threadIdx.x;
  if (jj < K) {
    if (err_hist) {
      const double xr2 = sc[B_XREF2 * KP + jj];
      err_hist[it * K + jj] = xr2 > 0.0 ? sqrt(tot[64 + jj] / xr2) : sqrt(tot[64 + jj]);
    }
    if (sc[B_DONE * KP + jj] == 0.0) {
      const double itn = sc[B_ITN * KP + jj] + 1.0;
      sc[B_ITN * KP + jj] = itn;
      const double ddnorm = sc[B_DDNORM * KP + jj] + tot[jj];
      sc[B_DDNORM * KP + jj] = ddnorm;
      const double anorm = sqrt(sc[B_ANORM2 * KP + jj]);
      const double acond = anorm * sqrt(ddnorm);
      const double rnorm = sc[B_PHIBAR * KP + jj];
      const double arnorm = sc[B_ALPHA * KP + jj] * fabs(sc[B_C * KP + jj]) * rnorm;
      const double xnorm = sqrt(tot[32 + jj]);
      const double bnorm = sc[B_BNORM * KP + jj];
      sc[B_ACOND * KP + jj] = acond;
      sc[B_RNORM * KP + jj] = rnorm;
      sc[B_ARNORM * KP + jj] = arnorm;
      sc[B_XNORM * KP + jj] = xnorm;
      const double atol = g[G_ATOL], btol = g[G_BTOL], ctol = g[G_CTOL];
      const double test1 = rnorm / bnorm;
      const double test2 = (anorm * rnorm > 0.0) ? arnorm / (anorm * rnorm) : 0.0;
      const double test3 = 1.0 / acond;
      // tests on the preconditioned system: ||A D|| and the norm of its iterate z
      const double znorm = sqrt(tot[96 + jj]);
      const double t1n = test1 / (1.0 + anorm * znorm / bnorm);
      const double rtol = btol + atol * anorm * znorm / bnorm;
      int istop = 0;
      if (itn >= g[G_ITNLIM]) istop = 7;
      if (1.0 + test3 <= 1.0) istop = 6;
      if (1.0 + test2 <= 1.0) istop = 5;
      if (1.0 + t1n <= 1.0) istop = 4;
      if (test3 <= ctol) istop = 3;
      if (test2 <= atol) istop = 2;
      if (test1 <= rtol) istop = 1;
      sc[B_ISTOP * KP + jj] = istop;
      if (istop != 0) {
        sc[B_DONE * KP + jj] = 1.0;
        sc[B_COEF * KP + jj] = 0.0;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    g[G_ITER] = (double)(it + 1);
    bool all = true;
    for (int q = 0; q < K; ++q) all = all && sc[B_DONE * KP + q] != 0.0;
    if (all || it + 1 >= (int64_t)g[G_ITNLIM]) g[G_ALLDONE] = 1.0;
  }
}

// x_j = 2^s_j D z_j into the caller layout [n][k].
__global__ void k_finish_b(int64_t n, int k, int KP, const double* __restrict__ d,
                           const float2* __restrict__ XZ, const double* __restrict__ sc,
                           double* __restrict__ x) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * k;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / k;
    const int j = (int)(e % k);
    const float2 z = XZ[i * KP + j];
    x[e] = d[i] * ldexp(ff_to_double(ff{z.x, z.y}), (int)sc[B_BEXP * KP + j]);
  }
}
// D (FP64) and the pairs of D' = 2^-g D; *bad as for the single solve (2: a
// scale not positive and finite, 1: D' outside the vector band).
__global__ void k_scale_b(int64_t n, int mode, const double* __restrict__ colnorm,
                          const double* __restrict__ user, const int16_t* __restrict__ cexp,
                          double* __restrict__ dsc, float2* __restrict__ dsc_ff, double* bad) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    double s = 1.0;
    if (mode == GSR_PRECOND_COLNORM) {
      const double c = colnorm[j];
      s = c > 0.0 ? 1.0 / c : 1.0;
    } else if (mode == GSR_PRECOND_USER) {
      s = user[j];
    }
    dsc[j] = s;
    const double sp = cexp ? ldexp(s, -(int)cexp[j]) : s;
    if (!(s > 0.0) || !isfinite(s)) *bad = 2.0;
    else if (!vec_in_band(sp)) *bad = 1.0;
    const ff f = ff_from_double(sp);
    dsc_ff[j] = make_float2(f.h, f.l);
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side: workspace, launchers, autotuner, driver.
// ---------------------------------------------------------------------------
struct BatchWork {
  int KP = 0;
  int64_t n_rows = 0, n_unk = 0;
  float2 *U = nullptr, *Uk = nullptr, *Vff = nullptr;
  float2 *V = nullptr, *W = nullptr, *XZ = nullptr, *Dff = nullptr;  // float pairs
  double *Z = nullptr, *D = nullptr;
  double *sc = nullptr, *hsc = nullptr, *part = nullptr;
  unsigned int* count = nullptr;
  int threads = 256;  // block width of the row/knot kernels (tuned)
  InstrCsc csc;       // instrumental buckets; csc.tile_log is tuned
  bool tuned = false;
  // mixed precision (allocated on first use): phase-1 solution [n_unk][k],
  // residual [n_rows][k], phase-1 solution in the padded layout [n_unk][KP]
  double *X1 = nullptr, *R = nullptr, *X1p = nullptr;
};

static void free_batch(BatchWork* w) {
  if (!w) return;
  void* p[] = {w->U,    w->Uk,   w->Vff,        w->V,          w->W,          w->XZ,
               w->Z,    w->D,    w->Dff,        w->sc,         w->part,       w->count,
               w->csc.off, w->csc.row, w->csc.val, w->csc.cnt, w->X1, w->R, w->X1p};
  for (void* q : p)
    if (q) cudaFree(q);
  if (w->hsc) cudaFreeHost(w->hsc);
  delete w;
}

void destroy_batch(gsr_system* s) {
  free_batch(static_cast<BatchWork*>(s->batch));
  s->batch = nullptr;
}

static int kpad(int k) {
  int p = 1;
  while (p < k) p <<= 1;
  return p;
}

// (Re)build the instrumental buckets for tiles of 2^tile_log rows.
static int build_csc(gsr_system* s, BatchWork* w, int tile_log, cudaStream_t st) {
  InstrCsc& C = w->csc;
  const Layout& L = s->L;
  const int64_t n_tiles = (L.n_rows + ((int64_t)1 << tile_log) - 1) >> tile_log;
  const int64_t nb = n_tiles * L.n_instr;
  cudaError_t e = cudaSuccess;
  if (!C.row) {
    if (e == cudaSuccess) e = cudaMalloc((void**)&C.row, std::max<int64_t>(6 * L.n_rows, 1) * 4);
    if (e == cudaSuccess) e = cudaMalloc((void**)&C.val, std::max<int64_t>(6 * L.n_rows, 1) * 8);
  }
  if (e == cudaSuccess && nb > C.cap_buckets) {
    if (C.off) cudaFree(C.off);
    if (C.cnt) cudaFree(C.cnt);
    C.off = nullptr;
    C.cnt = nullptr;
    e = cudaMalloc((void**)&C.off, (nb + 1) * 8);
    if (e == cudaSuccess) e = cudaMalloc((void**)&C.cnt, std::max<int64_t>(nb, 1) * 4);
    C.cap_buckets = e == cudaSuccess ? nb : 0;
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? GSR_E_OOM : GSR_E_CUDA;
  }
  C.tile_log = tile_log;
  C.n_tiles = n_tiles;
  C.n_bins = L.n_instr;
  const int rb = (int)std::max<int64_t>(1, std::min<int64_t>((L.n_rows + 255) / 256,
                                                             (int64_t)s->num_sms * 16));
  if (cudaMemsetAsync(C.cnt, 0, nb * 4, st) != cudaSuccess) return GSR_E_CUDA;
  k_csc_count<<<rb, 256, 0, st>>>(L, tile_log, L.n_instr, C.cnt);
  k_csc_scan<<<1, 1024, 0, st>>>(C.cnt, nb, C.off);
  if (cudaMemsetAsync(C.cnt, 0, nb * 4, st) != cudaSuccess) return GSR_E_CUDA;
  k_csc_fill<<<rb, 256, 0, st>>>(L, tile_log, L.n_instr, C.off, C.cnt, C.row, C.val);
  return cuda_status(cudaGetLastError());
}

// Tile height whose Y rows (KP pairs each) take about 32 MB of L2.
static int default_tile_log(int KP) {
  int lg = 12;
  while (lg < 20 && ((int64_t)1 << (lg + 1)) * KP * 8 <= ((int64_t)32 << 20)) ++lg;
  return lg;
}

static int batch_work(gsr_system* s, int KP, BatchWork** out, cudaStream_t st) {
  BatchWork* w = static_cast<BatchWork*>(s->batch);
  if (w && w->KP == KP) {
    *out = w;
    return GSR_OK;
  }
  free_batch(w);
  s->batch = nullptr;
  w = new BatchWork();
  w->KP = KP;
  w->n_rows = s->L.n_rows;
  w->n_unk = s->L.n_unk;
  const int64_t np = padded_rows(s->L), m = s->L.n_unk;
  cudaError_t e = cudaSuccess;
  auto A = [&](void** p, size_t bytes) {
    if (e == cudaSuccess) e = cudaMalloc(p, bytes ? bytes : 8);
  };
  A((void**)&w->U, np * KP * 8);
  A((void**)&w->Uk, (s->L.n_rows + 1) * KP * 8);
  A((void**)&w->Vff, m * KP * 8);
  A((void**)&w->V, m * KP * 8);
  A((void**)&w->W, m * KP * 8);
  A((void**)&w->XZ, m * KP * 8);
  A((void**)&w->Z, m * KP * 8);
  A((void**)&w->D, m * 8);
  A((void**)&w->Dff, m * 8);
  A((void**)&w->sc, (B_COUNT * KP + G_COUNT) * 8);
  A((void**)&w->part, (size_t)148 * 16 * 3 * 32 * 8);
  A((void**)&w->count, 16 * 4);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&w->hsc, (B_COUNT * KP + G_COUNT) * 8);
  if (e == cudaSuccess) e = cudaMemset(w->U, 0, np * KP * 8);
  if (e == cudaSuccess) e = cudaMemset(w->count, 0, 16 * 4);
  if (e != cudaSuccess) {
    cudaGetLastError();
    free_batch(w);
    return e == cudaErrorMemoryAllocation ? GSR_E_OOM : GSR_E_CUDA;
  }
  s->batch = w;
  const int rc = build_csc(s, w, default_tile_log(KP), st);
  if (rc != GSR_OK) {
    destroy_batch(s);
    return rc;
  }
  *out = w;
  return GSR_OK;
}

template <int KP, bool F32>
static int launch_aprod1_bt(gsr_system* s, BatchWork* w, const float2* X, float2* Y,
                            const double* coef, float2* Yk, double* norm_out, const double* stop,
                            cudaStream_t st) {
  const Layout& L = s->L;
  if (L.n_recs <= 0) return GSR_OK;
  const int wpb = w->threads / 32;
  const int blocks = (int)std::min<int64_t>((L.n_recs + wpb - 1) / wpb, (int64_t)s->num_sms * 16);
  k_aprod1_b<KP, F32><<<blocks, w->threads, 0, st>>>(L, X, Y, coef, Yk, w->part, w->count + 0,
                                                     norm_out, stop);
  return cuda_status(cudaGetLastError());
}

template <int KP, bool F32>
static int launch_aprod2_bt(gsr_system* s, BatchWork* w, const float2* Y, const float2* Yk,
                            double* X, const double* stop, cudaStream_t st) {
  const Layout& L = s->L;
  if (L.n_rows <= 0) return GSR_OK;
  if (cudaEventRecord(s->ev_fork, st) != cudaSuccess) return GSR_E_CUDA;
  if (cudaStreamWaitEvent(s->side, s->ev_fork, 0) != cudaSuccess) return GSR_E_CUDA;
  const int att_blocks = (L.n_att_warps * ATT_B_SPLIT + 7) / 8;
  if (att_blocks > 0) k_aprod2_att_b<KP, F32><<<att_blocks, 256, 0, s->side>>>(L, Yk, X, stop);
  if (cudaGetLastError() != cudaSuccess) return GSR_E_CUDA;
  const InstrCsc& C = w->csc;
  const int64_t nbk = C.n_tiles * C.n_bins;
  if (nbk > 0) {
    const int64_t warps = (nbk + (32 / KP) - 1) / (32 / KP);
    const int ib = (int)std::min<int64_t>((warps + 7) / 8, (int64_t)s->num_sms * 16);
    k_aprod2_instr_csc<KP, F32><<<ib, 256, 0, st>>>(L, C.off, C.row, C.val, nbk, C.n_bins, Y, X,
                                                    stop);
  }
  if (cudaGetLastError() != cudaSuccess) return GSR_E_CUDA;
  const int wpb = w->threads / 32;
  const int ab = (int)std::min<int64_t>((L.n_recs + wpb - 1) / wpb, (int64_t)s->num_sms * 16);
  k_aprod2_astro_b<KP, F32><<<ab, w->threads, 0, st>>>(L, Y, X, stop);
  if (cudaGetLastError() != cudaSuccess) return GSR_E_CUDA;
  if (cudaEventRecord(s->ev_join, s->side) != cudaSuccess) return GSR_E_CUDA;
  if (cudaStreamWaitEvent(st, s->ev_join, 0) != cudaSuccess) return GSR_E_CUDA;
  return GSR_OK;
}

#define GSR_KP_DISPATCH(KPV, CALL)                 \
  switch (KPV) {                                   \
    case 1: { constexpr int KP = 1; return CALL; } \
    case 2: { constexpr int KP = 2; return CALL; } \
    case 4: { constexpr int KP = 4; return CALL; } \
    case 8: { constexpr int KP = 8; return CALL; } \
    case 16: { constexpr int KP = 16; return CALL; } \
    case 32: { constexpr int KP = 32; return CALL; } \
    default: return GSR_E_ARG;                     \
  }

// f32: the FP32-value kernels of a mixed-precision solve (needs the FP32 copy).
static int aprod1_b(gsr_system* s, BatchWork* w, const float2* X, float2* Y, const double* coef,
                    float2* Yk, double* norm_out, const double* stop, cudaStream_t st,
                    bool f32 = false) {
  if (f32)
    GSR_KP_DISPATCH(w->KP, (launch_aprod1_bt<KP, true>(s, w, X, Y, coef, Yk, norm_out, stop, st)));
  GSR_KP_DISPATCH(w->KP, (launch_aprod1_bt<KP, false>(s, w, X, Y, coef, Yk, norm_out, stop, st)));
}
static int aprod2_b(gsr_system* s, BatchWork* w, const float2* Y, const float2* Yk, double* X,
                    const double* stop, cudaStream_t st, bool f32 = false) {
  if (f32) GSR_KP_DISPATCH(w->KP, (launch_aprod2_bt<KP, true>(s, w, Y, Yk, X, stop, st)));
  GSR_KP_DISPATCH(w->KP, (launch_aprod2_bt<KP, false>(s, w, Y, Yk, X, stop, st)));
}

// The autotuner: times aprod 1 + aprod 2 for every (block width, instrumental
// tile height) candidate on the system's own data and keeps the fastest.
static int autotune(gsr_system* s, BatchWork* w, cudaStream_t st) {
  if (w->tuned) return GSR_OK;
  const int widths[] = {128, 256};
  const int d = default_tile_log(w->KP);
  const int tiles[] = {d - 1, d, d + 1};
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return GSR_E_CUDA;
  float best = 1e30f;
  int bw = 256, bt = d;
  int rc = GSR_OK;
  for (int tl : tiles) {
    if ((rc = build_csc(s, w, tl, st)) != GSR_OK) break;
    for (int width : widths) {
      w->threads = width;
      float t_min = 1e30f;
      for (int rep = 0; rep < 3 && rc == GSR_OK; ++rep) {
        cudaMemsetAsync(w->Z, 0, w->n_unk * w->KP * 8, st);
        cudaEventRecord(e0, st);
        rc = aprod1_b(s, w, w->Vff, w->U, nullptr, nullptr, nullptr, nullptr, st);
        if (rc == GSR_OK) rc = aprod2_b(s, w, w->U, w->Uk, w->Z, nullptr, st);
        cudaEventRecord(e1, st);
        if (rc == GSR_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = GSR_E_CUDA;
        float ms = 0.f;
        if (rc == GSR_OK) cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) t_min = std::min(t_min, ms);
      }
      if (rc != GSR_OK) break;
      if (t_min < best) {
        best = t_min;
        bw = width;
        bt = tl;
      }
    }
    if (rc != GSR_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != GSR_OK) return rc;
  w->threads = bw;
  if (w->csc.tile_log != bt && (rc = build_csc(s, w, bt, st)) != GSR_OK) return rc;
  w->tuned = true;
  return GSR_OK;
}

template <int KP>
static int enqueue_b(gsr_system* s, BatchWork* w, const double* xref, const double* xoff,
                     double* err_dev, cudaStream_t st, int first, bool f32) {
  const int64_t m = s->L.n_unk;
  double* stop = w->sc + B_COUNT * KP + G_ALLDONE;
  const int vb = (int)std::min<int64_t>((m * KP + 255) / 256, (int64_t)s->num_sms * 8);
  int rc = GSR_OK;
  if (!first) {
    rc = aprod1_b(s, w, w->Vff, w->U, w->sc + B_COEF * KP, w->Uk, w->sc + B_UNORM2 * KP, stop, st,
                  f32);
    if (rc != GSR_OK) return rc;
  }
  k_zero_d<<<vb, 256, 0, st>>>(w->Z, m * KP, first ? nullptr : stop);
  rc = aprod2_b(s, w, w->U, w->Uk, w->Z, first ? nullptr : stop, st, f32);
  if (rc != GSR_OK) return rc;
  k_vec_a_b<KP><<<vb, 256, 0, st>>>(m, w->Dff, w->Z, w->V, w->sc, w->part, w->count + 1, first);
  k_vec_b_b<KP><<<vb, 256, 0, st>>>(m, w->Dff, w->V, w->W, w->XZ, w->Vff, first ? nullptr : xref,
                                    xoff, s->L.col_exp, w->sc, w->part, w->count + 2, first,
                                    first ? nullptr : err_dev);
  return cuda_status(cudaGetLastError());
}
static int enqueue_iter_b(gsr_system* s, BatchWork* w, const double* xref, const double* xoff,
                          double* err_dev, cudaStream_t st, int first, bool f32) {
  GSR_KP_DISPATCH(w->KP, (enqueue_b<KP>(s, w, xref, xoff, err_dev, st, first, f32)));
}
template <int KP>
static int init_b(gsr_system* s, BatchWork* w, const double* B, int k, const double* xref,
                  cudaStream_t st, bool f32) {
  const int64_t rb = std::min<int64_t>((s->L.n_rows * KP + 255) / 256, (int64_t)s->num_sms * 8);
  k_init_b<KP><<<(int)std::max<int64_t>(rb, 1), 256, 0, st>>>(
      s->L, B, k, s->S.iexp, w->U, w->Uk,
      knot_positions(s->L, f32 ? GSR_VALUES_F32 : GSR_VALUES_F64), w->sc, w->part, w->count + 3);
  if (xref) {
    const int vb = (int)std::min<int64_t>((s->L.n_unk * KP + 255) / 256, (int64_t)s->num_sms * 8);
    k_xref2_b<KP><<<vb, 256, 0, st>>>(s->L.n_unk, xref, w->sc, w->part, w->count + 4);
  }
  return cuda_status(cudaGetLastError());
}
static int init_iter_b(gsr_system* s, BatchWork* w, const double* B, int k, const double* xref,
                       cudaStream_t st, bool f32) {
  GSR_KP_DISPATCH(w->KP, (init_b<KP>(s, w, B, k, xref, st, f32)));
}

__global__ void k_pack_xref(const double* __restrict__ in, int k, int KP, int64_t n,
                            double* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * KP;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e % KP);
    out[e] = j < k ? in[(e / KP) * k + j] : 0.0;
  }
}

// One LSQR run on the k right-hand sides with the float-pair kernels (f32 =
// false) or the FP32-value ones (f32 = true). xoff (packed [n_unk][KP]) is
// added to the iterate when measuring the error against x_ref (the second
// phase of a mixed-precision solve).
static int lsqr_batch_run(gsr_system* s, int k, const double* B, double* X,
                          const gsr_lsqr_opts* o, gsr_lsqr_result* res, cudaStream_t st,
                          bool f32, const double* xoff, int64_t itnlim) {
  const int KP = kpad(k);
  BatchWork* w = nullptr;
  int rc = batch_work(s, KP, &w, st);
  if (rc != GSR_OK) return rc;
  const int64_t m = s->L.n_unk;
  cudaError_t e = cudaSuccess;
  auto C = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
  };
  const int vb = (int)std::min<int64_t>((m + 255) / 256, (int64_t)s->num_sms * 8);
  // column scaling D and the pairs of D' = 2^-g D (checked), exponent of each
  // right-hand side (and a check that B is finite)
  C(cudaMemsetAsync(s->S.guard + 1, 0, 3 * sizeof(double), st));
  C(cudaMemsetAsync(s->S.iexp, 0x80, 32 * sizeof(int), st));
  k_scale_b<<<vb, 256, 0, st>>>(m, o->precond, s->colnorm, o->scale, s->L.col_exp, w->D, w->Dff,
                                s->S.guard + 1);
  {
    const int rb = (int)std::max<int64_t>(
        1, std::min<int64_t>((s->L.n_rows * KP + 255) / 256, (int64_t)s->num_sms * 8));
    switch (KP) {
      case 1: k_maxexp_b<1><<<rb, 256, 0, st>>>(B, k, s->L.n_rows, s->S.iexp, s->S.guard + 3); break;
      case 2: k_maxexp_b<2><<<rb, 256, 0, st>>>(B, k, s->L.n_rows, s->S.iexp, s->S.guard + 3); break;
      case 4: k_maxexp_b<4><<<rb, 256, 0, st>>>(B, k, s->L.n_rows, s->S.iexp, s->S.guard + 3); break;
      case 8: k_maxexp_b<8><<<rb, 256, 0, st>>>(B, k, s->L.n_rows, s->S.iexp, s->S.guard + 3); break;
      case 16: k_maxexp_b<16><<<rb, 256, 0, st>>>(B, k, s->L.n_rows, s->S.iexp, s->S.guard + 3); break;
      default: k_maxexp_b<32><<<rb, 256, 0, st>>>(B, k, s->L.n_rows, s->S.iexp, s->S.guard + 3); break;
    }
    double flags[3] = {0.0, 0.0, 0.0};
    C(cudaGetLastError());
    C(cudaMemcpyAsync(flags, s->S.guard + 1, sizeof(flags), cudaMemcpyDeviceToHost, st));
    C(cudaStreamSynchronize(st));
    if (e != cudaSuccess) return GSR_E_CUDA;
    if (flags[0] == 2.0) return GSR_E_ARG;
    if (flags[0] != 0.0) return GSR_E_UNSUPPORTED;
    if (flags[2] != 0.0) return GSR_E_NONFINITE;
  }
  // the autotuner runs once per system and k, on the (so far unused) work vectors
  if (!w->tuned) {
    C(cudaMemsetAsync(w->Vff, 0, m * KP * 8, st));
    C(cudaMemsetAsync(w->Uk, 0, s->L.n_rows * KP * 8, st));
    if ((rc = autotune(s, w, st)) != GSR_OK) return rc;
  }
  std::vector<double> h(B_COUNT * KP + G_COUNT, 0.0);
  double* g = h.data() + B_COUNT * KP;
  g[G_ATOL] = o->atol;
  g[G_BTOL] = o->btol;
  g[G_CTOL] = o->conlim > 0.0 ? 1.0 / o->conlim : 0.0;
  g[G_ITNLIM] = (double)itnlim;
  g[G_K] = k;
  for (int j = k; j < KP; ++j) h[B_DONE * KP + j] = 1.0;  // padding lanes never run
  C(cudaMemcpyAsync(w->sc, h.data(), h.size() * 8, cudaMemcpyHostToDevice, st));
  C(cudaStreamSynchronize(st));
  double* xref = nullptr;
  double* err_dev = nullptr;
  if (o->x_ref && o->err_hist) {
    C(cudaMallocAsync((void**)&xref, m * KP * 8, st));
    C(cudaMallocAsync((void**)&err_dev, (itnlim + 1) * k * 8, st));
    if (e != cudaSuccess) return GSR_E_CUDA;
    k_pack_xref<<<vb, 256, 0, st>>>(o->x_ref, k, KP, m, xref);
  }
  if (e != cudaSuccess) return GSR_E_CUDA;
  rc = init_iter_b(s, w, B, k, xref, st, f32);
  if (rc == GSR_OK) rc = enqueue_iter_b(s, w, xref, xoff, err_dev, st, 1, f32);
  if (rc != GSR_OK) return rc;
  int64_t n_launches = 12;
  // iterations: graph of a chunk of iterations, replayed until every RHS stopped
  const int chunk = 4;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool use_graph = st != nullptr;
  if (use_graph) {
    cudaStreamCaptureStatus cs;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
      use_graph = false;
  }
  if (use_graph && cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    int r2 = GSR_OK;
    for (int i = 0; i < chunk && r2 == GSR_OK; ++i)
      r2 = enqueue_iter_b(s, w, xref, xoff, err_dev, st, 0, f32);
    const cudaError_t ce = cudaStreamEndCapture(st, &graph);
    if (r2 != GSR_OK || ce != cudaSuccess || cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
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
  const size_t hbytes = (B_COUNT * KP + G_COUNT) * 8;
  int64_t launched = 0;
  while (true) {
    if (use_graph) {
      C(cudaGraphLaunch(exec, st));
    } else {
      for (int i = 0; i < chunk && rc == GSR_OK; ++i)
        rc = enqueue_iter_b(s, w, xref, xoff, err_dev, st, 0, f32);
    }
    launched += chunk;
    n_launches += (int64_t)chunk * 8;
    C(cudaMemcpyAsync(w->hsc, w->sc, hbytes, cudaMemcpyDeviceToHost, st));
    C(cudaStreamSynchronize(st));
    if (e != cudaSuccess || rc != GSR_OK) break;
    if (w->hsc[B_COUNT * KP + G_ALLDONE] != 0.0) break;
    if (launched > itnlim + chunk) break;
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  if (e != cudaSuccess || rc != GSR_OK) {
    if (xref) cudaFreeAsync(xref, st);
    if (err_dev) cudaFreeAsync(err_dev, st);
    return rc != GSR_OK ? rc : GSR_E_CUDA;
  }
  k_finish_b<<<vb, 256, 0, st>>>(m, k, KP, w->D, w->XZ, w->sc, X);
  const int64_t iters = (int64_t)w->hsc[B_COUNT * KP + G_ITER];
  if (o->err_hist && err_dev && iters > 0)
    C(cudaMemcpyAsync(o->err_hist, err_dev, iters * k * 8, cudaMemcpyDeviceToHost, st));
  if (xref) C(cudaFreeAsync(xref, st));
  if (err_dev) C(cudaFreeAsync(err_dev, st));
  C(cudaStreamSynchronize(st));
  if (e != cudaSuccess) return GSR_E_CUDA;
  const double* hs = w->hsc;
  for (int j = 0; j < k; ++j) {
    gsr_lsqr_result& r = res[j];
    std::memset(&r, 0, sizeof(r));
    const int sb = (int)hs[B_BEXP * KP + j];
    r.istop = (int32_t)hs[B_ISTOP * KP + j];
    r.itn = (int64_t)hs[B_ITN * KP + j];
    r.rnorm = std::ldexp(hs[B_RNORM * KP + j], sb);
    r.arnorm = std::ldexp(hs[B_ARNORM * KP + j], sb);
    r.anorm = std::sqrt(hs[B_ANORM2 * KP + j]);
    r.acond = hs[B_ACOND * KP + j];
    r.xnorm = std::ldexp(hs[B_XNORM * KP + j], sb);
    r.n_launches = n_launches;
    r.n_timed_itn = iters;
  }
  return GSR_OK;
}

// Y[n][k] += (or -=, neg) A X[n_unk][k] on the observation rows: the
// float-pair kernels when the rescaled X is within the band, else FP64.
static int batch_aprod1_direct(gsr_system* sys, BatchWork* w, int k, const double* X, int neg,
                               double* Y, cudaStream_t st) {
  const int64_t m = sys->L.n_unk, n = sys->L.n_rows;
  if (n == 0) return GSR_OK;
  if (sys->wide) return launch_aprod1_f64(sys, GSR_VALUES_F64, X, k, neg, Y, nullptr, st);
  const int KP = w->KP;
  const int bm = (int)std::min<int64_t>((m * KP + 255) / 256 + 1, sys->num_sms * 8);
  const int bn = (int)std::min<int64_t>((n * KP + 255) / 256 + 1, sys->num_sms * 8);
  double* guard = sys->S.guard;
  if (cudaMemsetAsync(guard, 0, sizeof(double), st) != cudaSuccess) return GSR_E_CUDA;
  // U = A' X' (pairs, from zero), then Y += 2^-e U in FP64
  if (cudaMemsetAsync(w->U, 0, (size_t)n * KP * sizeof(float2), st) != cudaSuccess)
    return GSR_E_CUDA;
  k_pack_ff<<<bm, 256, 0, st>>>(X, k, KP, m, sys->L.col_exp, guard, w->Vff, neg);
  int rc = aprod1_b(sys, w, w->Vff, w->U, nullptr, nullptr, nullptr, guard, st);
  if (rc != GSR_OK) return rc;
  k_unpack_add<<<bn, 256, 0, st>>>(w->U, k, KP, n, sys->L.row_exp, guard, Y);
  if (cudaGetLastError() != cudaSuccess) return GSR_E_CUDA;
  return launch_aprod1_f64(sys, GSR_VALUES_F64, X, k, neg, Y, guard, st);
}

// Mixed precision for k right-hand sides, as for one: phase 1 runs LSQR with
// the FP32-value kernels (coefficients of the FP32 copy of A, one FP32
// multiply-add per product) to about FP32 accuracy; then R = B - A X1 with the
// full-precision values; phase 2 runs LSQR with the float-pair kernels on
// min ||A D - R|| to the caller's tolerances (its fixed point is the
// full-precision solution); X = X1 + D. Each right-hand side keeps its own
// stopping tests and masks in both phases.
static int lsqr_batch_mixed(gsr_system* s, int k, const double* B, double* X,
                            const gsr_lsqr_opts* o, gsr_lsqr_result* res, cudaStream_t st,
                            int64_t itnlim) {
  const int KP = kpad(k);
  BatchWork* w = nullptr;
  int rc = batch_work(s, KP, &w, st);
  if (rc != GSR_OK) return rc;
  const int64_t n = s->L.n_rows, m = s->L.n_unk;
  if (!w->X1) {
    cudaError_t e = cudaMalloc((void**)&w->X1, (size_t)std::max<int64_t>(m, 1) * k * 8);
    if (e == cudaSuccess) e = cudaMalloc((void**)&w->R, (size_t)std::max<int64_t>(n, 1) * k * 8);
    if (e == cudaSuccess) e = cudaMalloc((void**)&w->X1p, (size_t)std::max<int64_t>(m, 1) * KP * 8);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return e == cudaErrorMemoryAllocation ? GSR_E_OOM : GSR_E_CUDA;
    }
  }
  // phase 1: FP32 values; FP32 products limit it to about 1e-6
  constexpr double PHASE1_TOL = 1e-6;
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
  std::vector<gsr_lsqr_result> r1(k);
  rc = lsqr_batch_run(s, k, B, w->X1, &o1, r1.data(), st, true, nullptr, lim1);
  if (rc != GSR_OK) return rc;
  const int64_t n1 = r1[0].n_timed_itn;  // iterations phase 1 ran (its longest right-hand side)
  // R = B - A X1 with the full-precision values
  if (cudaMemcpyAsync(w->R, B, (size_t)n * k * 8, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return GSR_E_CUDA;
  rc = batch_aprod1_direct(s, w, k, w->X1, 1, w->R, st);
  if (rc != GSR_OK) return rc;
  const double* xoff = nullptr;
  if (o->err_hist && o->x_ref) {
    const int vb = (int)std::min<int64_t>((m * KP + 255) / 256, (int64_t)s->num_sms * 8);
    k_pack_xref<<<vb, 256, 0, st>>>(w->X1, k, KP, m, w->X1p);
    xoff = w->X1p;
  }
  // phase 2: full precision on the residual
  gsr_lsqr_opts o2 = *o;
  o2.err_hist = o->err_hist ? o->err_hist + n1 * k : nullptr;
  const int64_t lim2 = std::max<int64_t>(1, itnlim - n1);
  rc = lsqr_batch_run(s, k, w->R, X, &o2, res, st, false, xoff, lim2);
  if (rc != GSR_OK) return rc;
  const int vb = (int)std::min<int64_t>((m * k + 255) / 256, (int64_t)s->num_sms * 8);
  k_add_cols<<<vb, 256, 0, st>>>(w->X1, k, k, m, nullptr, nullptr, X);  // X = D + X1
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
    return GSR_E_CUDA;
  for (int j = 0; j < k; ++j) {
    res[j].phase2_itn = (int32_t)res[j].itn;
    res[j].itn += r1[j].itn;
    res[j].n_timed_itn += n1;
    res[j].n_launches += r1[j].n_launches + 6;
  }
  return GSR_OK;
}

int lsqr_batch(gsr_system* s, int k, const double* B, double* X, const gsr_lsqr_opts* o,
               gsr_lsqr_result* res, cudaStream_t st) {
  const int64_t itnlim = o->itnlim > 0 ? o->itnlim : 20 * std::max<int64_t>(1, s->L.n_unk);
  if (o->precision == GSR_PREC_MIXED) return lsqr_batch_mixed(s, k, B, X, o, res, st, itnlim);
  return lsqr_batch_run(s, k, B, X, o, res, st, false, nullptr, itnlim);
}

}  // namespace gsr

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

int gsr_aprod1_batch(gsr_system* sys, int k, const double* X, double* Y, void* stream) {
  if (!sys || k < 1 || k > 32 || (!X && sys->L.n_unk > 0) || (!Y && sys->L.n_rows > 0))
    return GSR_E_ARG;
  if (sys->n_con > 0) return GSR_E_UNSUPPORTED;  // constraint rows: single-vector forms only
  gsr::DeviceGuard dg(sys->device);
  if (!dg.ok) return GSR_E_CUDA;
  if (const int se = gsr::sticky_error(sys)) return se;  // an earlier launch failed
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (sys->L.n_rows == 0) return GSR_OK;
  gsr::BatchWork* w = nullptr;
  int rc = gsr::batch_work(sys, gsr::kpad(k), &w, st);
  if (rc != GSR_OK) return rc;
  return gsr::batch_aprod1_direct(sys, w, k, X, 0, Y, st);
}

int gsr_aprod2_batch(gsr_system* sys, int k, const double* Y, double* X, void* stream) {
  if (!sys || k < 1 || k > 32 || (!X && sys->L.n_unk > 0) || (!Y && sys->L.n_rows > 0))
    return GSR_E_ARG;
  if (sys->n_con > 0) return GSR_E_UNSUPPORTED;  // constraint rows: single-vector forms only
  gsr::DeviceGuard dg(sys->device);
  if (!dg.ok) return GSR_E_CUDA;
  if (const int se = gsr::sticky_error(sys)) return se;  // an earlier launch failed
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (sys->L.n_rows == 0) return GSR_OK;
  if (sys->wide) return gsr::launch_aprod2_f64(sys, GSR_VALUES_F64, Y, k, X, nullptr, st);
  const int KP = gsr::kpad(k);
  gsr::BatchWork* w = nullptr;
  int rc = gsr::batch_work(sys, KP, &w, st);
  if (rc != GSR_OK) return rc;
  const int64_t m = sys->L.n_unk;
  const int bm = (int)std::min<int64_t>((m * KP + 255) / 256 + 1, sys->num_sms * 8);
  const int bn = (int)std::min<int64_t>((sys->L.n_rows * KP + 255) / 256 + 1, sys->num_sms * 8);
  double* guard = sys->S.guard;
  if (cudaMemsetAsync(guard, 0, sizeof(double), st) != cudaSuccess) return GSR_E_CUDA;
  gsr::k_pack_ff_knot<<<bn, 256, 0, st>>>(sys->L, Y, k, KP, guard, w->U, w->Uk);
  gsr::k_zero_d<<<bm, 256, 0, st>>>(w->Z, m * KP, nullptr);
  rc = gsr::aprod2_b(sys, w, w->U, w->Uk, w->Z, guard, st);
  if (rc != GSR_OK) return rc;
  gsr::k_add_cols<<<bm, 256, 0, st>>>(w->Z, k, KP, m, sys->L.col_exp, guard, X);
  if (cudaGetLastError() != cudaSuccess) return GSR_E_CUDA;
  return gsr::launch_aprod2_f64(sys, GSR_VALUES_F64, Y, k, X, guard, st);
}

int gsr_lsqr_solve_batch(gsr_system* sys, int k, const double* B, double* X,
                         const gsr_lsqr_opts* opts, gsr_lsqr_result* res, void* stream) {
  if (!sys || !opts || !res || k < 1 || k > 32) return GSR_E_ARG;
  if ((!B && sys->L.n_rows > 0) || (!X && sys->L.n_unk > 0)) return GSR_E_ARG;
  if (opts->precond < GSR_PRECOND_NONE || opts->precond > GSR_PRECOND_USER) return GSR_E_ARG;
  if (opts->precond == GSR_PRECOND_USER && !opts->scale) return GSR_E_ARG;
  if (opts->precision != GSR_PREC_F64 && opts->precision != GSR_PREC_MIXED) return GSR_E_ARG;
  if (opts->precision == GSR_PREC_MIXED && !sys->rec_f32) return GSR_E_ARG;
  if (opts->var || opts->rnorm_hist || opts->n_cov > 0) return GSR_E_UNSUPPORTED;
  if (opts->err_hist && !opts->x_ref) return GSR_E_ARG;
  if (sys->row_scaled) return GSR_E_UNSUPPORTED;  // as for gsr_lsqr_solve
  if (sys->n_con > 0) return GSR_E_UNSUPPORTED;    // constraint rows: single-vector forms only
  gsr::DeviceGuard dg(sys->device);
  if (!dg.ok) return GSR_E_CUDA;
  if (const int se = gsr::sticky_error(sys)) return se;  // an earlier launch failed
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (sys->L.n_rows == 0 || sys->L.n_unk == 0) {
    if (X && sys->L.n_unk > 0) cudaMemsetAsync(X, 0, sys->L.n_unk * k * 8, st);
    for (int j = 0; j < k; ++j) std::memset(&res[j], 0, sizeof(res[j]));
    return gsr::cuda_status(cudaStreamSynchronize(st));
  }
  const int rc = gsr::lsqr_batch(sys, k, B, X, opts, res, st);
  return rc == GSR_OK ? gsr::sticky_error(sys) : rc;
}

int gsr_batch_tuning(const gsr_system* sys, int* threads, int* tile_rows) {
  if (!sys || !sys->batch) return GSR_E_ARG;
  const gsr::BatchWork* w = static_cast<const gsr::BatchWork*>(sys->batch);
  if (threads) *threads = w->threads;
  if (tile_rows) *tile_rows = 1 << w->csc.tile_log;
  return GSR_OK;
}

}  // extern "C"
