// aprod 1 (Eq. 2, y += A x) and aprod 2 (Eq. 3, x += A^T y) kernels for sm_103a.
//
// Both products are HBM-bound (about 0.2 flop per byte) and use no tensor
// cores. B300's FP64 pipe runs at ~1/64 of its FP32 rate, so the hot loops
// contain no double-precision arithmetic: products and sums are float pairs
// (hi, lo) with error-free transformations, and LSQR's u vector is kept as
// float pairs. A finished sum (a star's, a knot's, a histogram bin's) reaches
// FP64 memory as one L2 atomic of hi + lo, both widened exactly and added once
// in FP64.
//
// aprod 1 streams 64-row records into shared memory with TMA bulk copies
// (double-buffered per pair of warps, one row per lane) so that DRAM latency
// is off the critical path; the x gathers (L2-resident) of a row are issued at
// once and accumulated in five independent chains.
// aprod 2 is three kernels that run concurrently on two streams:
//   astro+glob  per-star sums over star-sorted records (segmented warp scan),
//   instr       per tile of up to 2048 rows, entries added into a float-pair
//               shared-memory histogram by compare-and-swap,
//   att         start-knot-ordered copy, sliding 4-knot window per axis.
#include <algorithm>

#include "gsr_system.cuh"

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

// x += hi + lo as two L2 reductions, each word widened exactly with integer
// instructions (no FP64 arithmetic on the SM).
__device__ __forceinline__ void red_ff(double* x, ff a) {
  if (a.h != 0.0f) atomicAdd(x, f2d_exact(a.h));
  if (a.l != 0.0f) atomicAdd(x, f2d_exact(a.l));
}

// ---------------------------------------------------------------------------
// Element conversions (only at the edges of the C ABI and of a solve).
// ---------------------------------------------------------------------------
// out = +-2^-cexp[j] scale[j] x[j] as float pairs (the rescaled input of a
// product); an entry outside the vector band sets *guard.
__global__ void k_to_ff(const double* __restrict__ x, const double* __restrict__ scale,
                        const int16_t* __restrict__ cexp, int neg, double* guard,
                        float2* __restrict__ out, int64_t n) {
  bool out_of_band = false;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    double v = x[j];
    if (scale) v *= scale[j];
    if (cexp) v = ldexp(v, -(int)cexp[j]);
    if (neg) v = -v;
    if (!vec_in_band(v)) out_of_band = true;
    ff f = ff_from_double(v);
    out[j] = make_float2(f.h, f.l);
  }
  if (guard && out_of_band) *guard = 1.0;
}

// y (double) -> 2^-e_i y_i as pairs in row order and in knot order; an entry
// outside the vector band sets *guard.
__global__ void k_to_ff_knot(Layout L, const double* __restrict__ y, float2* __restrict__ y_ff,
                             float2* __restrict__ y_knot, const int32_t* __restrict__ kp,
                             double* guard) {
  bool out_of_band = false;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < L.n_rows;
       r += (int64_t)gridDim.x * blockDim.x) {
    double v = y[r];
    if (L.row_exp) v = ldexp(v, -(int)L.row_exp[r]);
    if (!vec_in_band(v)) out_of_band = true;
    const ff f = ff_from_double(v);
    const float2 w = make_float2(f.h, f.l);
    y_ff[r] = w;
    y_knot[kp[r]] = w;
  }
  if (guard && out_of_band) *guard = 1.0;
}

// X3[s*12 + a*4 + j] = x[att_base + a*K + s + j]: the 12 attitude unknowns a
// row with start knot s multiplies, contiguous and 32-byte aligned per axis.
__global__ void k_att_x3(Layout L, const float2* __restrict__ x, float2* __restrict__ x3,
                         const double* stop) {
  if (stop && *stop != 0.0) return;
  const int64_t n = (L.n_knots - 3) * 12;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = i / 12;
    const int a = (int)((i % 12) >> 2), j = (int)(i & 3);
    x3[i] = __ldg(x + L.att_base + a * L.n_knots + s + j);
  }
}

__device__ __forceinline__ ff ff_lo(double d) { return ff{__int_as_float(__double2loint(d)), __int_as_float(__double2hiint(d))}; }

__device__ __forceinline__ ff ldx(const float2* __restrict__ x, int64_t j) {
  const float2 a = __ldg(x + j);
  return ff{a.x, a.y};
}

template <bool F32>
__device__ __forceinline__ ff val_mul(ff v, ff u) {
  if constexpr (F32) return f_mul(v.h, u);
  else return ff_mul(v, u);
}

// ---------------------------------------------------------------------------
// aprod 1: y[r] = coef * y[r] + (A x)[r] for every row; optionally
// y_knot[pos(r)] = y[r] (the knot-ordered copy aprod 2 reads) and a
// deterministic ||y||^2 into *norm_out. coef is *coef_dev if given. y is a
// float-pair vector (YFF, LSQR) or a double vector (the C ABI).
// One CTA per SM with NP pairs of warps. A pair owns NS record buffers in
// shared memory that TMA refills while the pair computes on the others; the
// two warps of a pair take one half of each record (lane l: row 32 h + l),
// and the warp that finishes a buffer second refills it (a counter per buffer
// in shared memory, acquire/release). The instrumental unknowns are gathered
// from the block's shared memory when they fit beside the buffers
// (instr_in_smem), otherwise through L1/L2.
// ---------------------------------------------------------------------------
constexpr int A1_PF = 1;  // records a pair keeps in flight towards L2 beyond its buffers

// Coefficient of slot t for row ri of a record in shared memory.
template <bool F32>
__device__ __forceinline__ ff rec_val1(const unsigned char* rec, int t, int ri) {
  if constexpr (F32) {
    return ff{*reinterpret_cast<const float*>(rec + slot_offset<true>(t) + ri * 4), 0.0f};
  } else {
    const float2 v = *reinterpret_cast<const float2*>(rec + slot_offset<false>(t) + ri * 8);
    return ff{v.x, v.y};
  }
}
// old value of *c before adding 1 (shared memory, acquire-release at CTA scope)
__device__ __forceinline__ uint32_t smem_add_acq_rel(uint32_t* c) {
  uint32_t old;
  asm volatile("atom.acq_rel.cta.shared::cta.add.u32 %0, [%1], 1;"
               : "=r"(old)
               : "r"(smem_u32(c))
               : "memory");
  return old;
}

template <bool F32, bool YFF, bool X3, int NP, int NS>
__global__ void __launch_bounds__(NP * 64, 1)
    k_aprod1(Layout L, const float2* __restrict__ x, const float2* __restrict__ x3,
              void* __restrict__ yv, const double* __restrict__ coef_dev, double coef_host,
              float2* __restrict__ y_knot, double* part, unsigned int* counter, double* norm_out,
              const double* stop, int instr_in_smem) {
  if (stop && *stop != 0.0) return;
  using R = Rec<F32>;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bars[NP * NS];
  __shared__ uint32_t done[NP * NS];  // halves finished with each buffer (mod 2)
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, pr = wid >> 1, half = wid & 1;
  unsigned char* stage0 = smem + (size_t)pr * NS * R::BYTES;
  float2* xi_s = reinterpret_cast<float2*>(smem + (size_t)NP * NS * R::BYTES);
  if (instr_in_smem)
    for (int i = threadIdx.x; i < L.n_instr; i += blockDim.x) xi_s[i] = __ldg(x + L.instr_base + i);
  const double4_32a* __restrict__ x3q = reinterpret_cast<const double4_32a*>(x3);
  uint64_t* bar = bars + pr * NS;
  uint32_t* dn = done + pr * NS;
  const int64_t gp = (int64_t)blockIdx.x * NP + pr, np = (int64_t)gridDim.x * NP;
  const unsigned char* recs = F32 ? L.rec_f32 : L.rec_ff;
  const double coef = coef_dev ? *coef_dev : coef_host;
  const ff coef_ff = ff_from_double(coef);
  const bool glob = L.n_glob == 1;
  const ff xg = glob ? ldx(x, L.glob_col) : ff_zero();
  const uint64_t pol = policy_evict_first();  // records are read once per product

  if (half == 0 && lane == 0) {
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      mbar_init(&bar[s], 1);
      dn[s] = 0u;
    }
    fence_proxy_async();
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      const int64_t r = gp + s * np;
      if (r < L.n_recs) {
        mbar_expect_tx(&bar[s], R::BYTES);
        tma_load_hint(stage0 + s * R::BYTES, recs + r * R::BYTES, R::BYTES, &bar[s], pol);
      }
    }
#pragma unroll
    for (int k = 0; k < A1_PF; ++k) {
      const int64_t rp = gp + (NS + k) * np;
      if (rp < L.n_recs) prefetch_l2(recs + rp * R::BYTES, R::BYTES);
    }
  }
  // the partner warp waits on barriers the first warp initialised
  __syncthreads();

  const int ri = half * 32 + lane;  // this lane's row inside a record
  ff nrm = ff_zero();
  double nrm_d = 0.0;
  uint32_t parity = 0;
  bool ok = true;
  int s = 0;
  for (int64_t r = gp; r < L.n_recs; r += np) {
    const unsigned char* rec = stage0 + s * R::BYTES;
    const int64_t row = r * REC_ROWS + ri;
    const bool live = row < L.n_rows;
    ff yo = ff_zero();
    double yd = 0.0;
    if constexpr (YFF) {
      if (live) {
        const float2 a = static_cast<const float2*>(yv)[row];
        yo = ff{a.x, a.y};
      }
    } else {
      if (live) yd = static_cast<const double*>(yv)[row];
    }
    bool got = false;
    for (int i = 0; i < WAIT_LIMIT; ++i)
      if (__all_sync(0xffffffffu, mbar_try_wait(&bar[s], (parity >> s) & 1u))) {
        got = true;
        break;
      }
    if (!got) {
      if (lane == 0) set_error(L.err, GSR_E_TIMEOUT);
      ok = false;
      break;
    }
    parity ^= 1u << s;

    const int st = reinterpret_cast<const int*>(rec + R::STAR)[ri];
    const int sk = reinterpret_cast<const int*>(rec + R::ATT_S)[ri];
    int ik[6];
#pragma unroll
    for (int k = 0; k < 6; ++k)
      ik[k] = reinterpret_cast<const unsigned short*>(rec + R::INSTR_I + k * 128)[ri];
    ff xv[NSLOT];
#pragma unroll
    for (int t = 0; t < 5; ++t) xv[t] = ldx(x, 5 * (int64_t)st + t);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if constexpr (X3) {
        const double4_32a q = x3q[(int64_t)sk * 3 + a];
        xv[5 + 4 * a + 0] = ff_lo(q.x);
        xv[5 + 4 * a + 1] = ff_lo(q.y);
        xv[5 + 4 * a + 2] = ff_lo(q.z);
        xv[5 + 4 * a + 3] = ff_lo(q.w);
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) xv[5 + 4 * a + i] = ldx(x, L.att_base + a * L.n_knots + sk + i);
      }
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      if (instr_in_smem) {
        const float2 v = xi_s[ik[k]];
        xv[17 + k] = ff{v.x, v.y};
      } else {
        xv[17 + k] = ldx(x, L.instr_base + ik[k]);
      }
    }
    xv[23] = xg;
    // five independent accumulation chains: astro, 3 attitude axes,
    // instrumental (+ global), combined by a tree at the end
    ff pa[5];
#pragma unroll
    for (int g = 0; g < 5; ++g) pa[g] = ff_zero();
#pragma unroll
    for (int t = 0; t < NSLOT; ++t) {
      if (t == 23 && !glob) continue;
      const int g = t < 5 ? 0 : t < 9 ? 1 : t < 13 ? 2 : t < 17 ? 3 : 4;
      pa[g] = ff_add(pa[g], val_mul<F32>(rec_val1<F32>(rec, t, ri), xv[t]));
    }
    const ff acc = ff_add(ff_add(ff_add(pa[0], pa[1]), ff_add(pa[2], pa[3])), pa[4]);
    const int ps = reinterpret_cast<const int*>(rec + R::POS)[ri];
    // every lane of this warp is done with the buffer
    __syncwarp();
    if (lane == 0) {
      // the second half to finish refills it with the record NS steps ahead
      if (smem_add_acq_rel(&dn[s]) & 1u) {
        const int64_t rn = r + NS * np;
        if (rn < L.n_recs) {
          fence_proxy_async();
          mbar_expect_tx(&bar[s], R::BYTES);
          tma_load_hint(stage0 + s * R::BYTES, recs + rn * R::BYTES, R::BYTES, &bar[s], pol);
        }
        const int64_t rp = rn + A1_PF * np;
        if (rp < L.n_recs) prefetch_l2(recs + rp * R::BYTES, R::BYTES);
      }
    }
    if constexpr (YFF) {
      const ff yn = ff_norm(ff_add(ff_mul(coef_ff, yo), acc));
      if (live) {
        static_cast<float2*>(yv)[row] = make_float2(yn.h, yn.l);
        nrm = ff_add(nrm, ff_mul(yn, yn));
        if (y_knot) y_knot[ps] = make_float2(yn.h, yn.l);
      }
    } else {
      double a = ff_to_double(acc);
      if (L.row_exp && live) a = ldexp(a, -(int)L.row_exp[row]);
      const double yn = __fma_rn(coef, yd, a);
      if (live) {
        static_cast<double*>(yv)[row] = yn;
        nrm_d = __fma_rn(yn, yn, nrm_d);
      }
    }
    s = (s + 1 == NS) ? 0 : s + 1;
  }
  if (!ok) {
    // give copies still in flight on the pair's buffers a bounded chance to land
    for (int q = 0; q < NS; ++q)
      for (int i = 0; i < WAIT_LIMIT / 16; ++i)
        if (mbar_try_wait(&bar[q], (parity >> q) & 1u)) break;
  }
  if (norm_out) grid_sum_store(YFF ? ff_to_double(nrm) : nrm_d, part, counter, norm_out);
}

// ---------------------------------------------------------------------------
// aprod 2, astrometric + global part. One warp per two records (grid-stride),
// the four rows of a lane are consecutive; per-star runs are summed in
// registers, joined across lanes by a segmented inclusive scan and added into
// x once per record pair (a star whose rows span pairs gets one add per pair).
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
__device__ __forceinline__ Astro astro_shfl_up(const Astro& a, int d) {
  Astro r;
#pragma unroll
  for (int t = 0; t < 5; ++t) r.c[t] = ff_shfl_up(a.c[t], d);
  return r;
}
__device__ __forceinline__ void astro_flush(double* __restrict__ x, int star, const Astro& a) {
#pragma unroll
  for (int t = 0; t < 5; ++t) red_ff(x + 5 * (int64_t)star + t, a.c[t]);
}

template <bool F32>
__global__ void __launch_bounds__(256) k_aprod2_astro(Layout L, const float2* __restrict__ y,
                                                      double* __restrict__ x, const double* stop) {
  if (stop && *stop != 0.0) return;
  using R = Rec<F32>;
  const int lane = threadIdx.x & 31, lp = lane & 15;
  const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const unsigned char* recs = F32 ? L.rec_f32 : L.rec_ff;
  const bool glob = L.n_glob == 1;
  const int64_t n_pairs = (L.n_recs + 1) / 2;
  ff gacc = ff_zero();
  // A warp takes two consecutive records (128 rows); lane l holds rows
  // 4(l%16) .. 4(l%16)+3 of record 2p + l/16, so one cross-lane scan serves
  // 128 rows. Runs are merged inside the lane first.
  for (int64_t pr = gw; pr < n_pairs; pr += nw) {
    const int64_t rl = 2 * pr + (lane >> 4);
    const bool have = rl < L.n_recs;
    const unsigned char* rec = recs + (have ? rl : 2 * pr) * R::BYTES;
    int s[4];
    ff v[6][4];
    float4 ya = make_float4(0.f, 0.f, 0.f, 0.f), yb = ya;
    if (have) {
      // y is padded to whole records (zeros), so these loads are in bounds
      const float4* yp = reinterpret_cast<const float4*>(y + rl * REC_ROWS + 4 * lp);
      ya = __ldcs(yp);
      yb = __ldcs(yp + 1);
      const int4 st = __ldcs(reinterpret_cast<const int4*>(rec + R::STAR + lp * 16));
      s[0] = st.x;
      s[1] = st.y;
      s[2] = st.z;
      s[3] = st.w;
#pragma unroll
      for (int t = 0; t < 6; ++t) {
        const int slot = t < 5 ? t : 23;
        if constexpr (F32) {
          const float4 a =
              __ldcs(reinterpret_cast<const float4*>(rec + slot_offset<true>(slot) + lp * 16));
          v[t][0] = ff{a.x, 0.0f};
          v[t][1] = ff{a.y, 0.0f};
          v[t][2] = ff{a.z, 0.0f};
          v[t][3] = ff{a.w, 0.0f};
        } else {
          const float4* q =
              reinterpret_cast<const float4*>(rec + slot_offset<false>(slot) + lp * 32);
          const float4 a = __ldcs(q), c = __ldcs(q + 1);
          v[t][0] = ff{a.x, a.y};
          v[t][1] = ff{a.z, a.w};
          v[t][2] = ff{c.x, c.y};
          v[t][3] = ff{c.z, c.w};
        }
      }
    } else {
#pragma unroll
      for (int t = 0; t < 6; ++t)
#pragma unroll
        for (int k = 0; k < 4; ++k) v[t][k] = ff_zero();
    }
    // a lane without a record continues the last star of lane 15 with zeros
    const int s_last15 = __shfl_sync(0xffffffffu, have ? s[3] : 0, 15);
    if (!have) s[0] = s[1] = s[2] = s[3] = s_last15;
    const ff u[4] = {ff{ya.x, ya.y}, ff{ya.z, ya.w}, ff{yb.x, yb.y}, ff{yb.z, yb.w}};
    Astro pk[4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int t = 0; t < 5; ++t) pk[k].c[t] = val_mul<F32>(v[t][k], u[k]);
    if (glob)
#pragma unroll
      for (int k = 0; k < 4; ++k) gacc = ff_add(gacc, val_mul<F32>(v[5][k], u[k]));

    // in-lane runs: head = run of s[0], tail = run of s[3]; a run strictly
    // between them is complete here and is flushed at once
    Astro acc = pk[0], head = pk[0];
    bool head_done = false;
#pragma unroll
    for (int k = 1; k < 4; ++k) {
      if (s[k] == s[k - 1]) {
        acc = astro_add(acc, pk[k]);
      } else {
        if (!head_done) {
          head = acc;
          head_done = true;
        } else {
          astro_flush(x, s[k - 1], acc);
        }
        acc = pk[k];
      }
    }
    const int s0 = s[0], s1 = s[3];
    const bool uniform = (s0 == s1);
    if (uniform) head = acc;
    const Astro tail = acc;
    // segmented inclusive scan of the tail runs across lanes
    const int prev_last = __shfl_up_sync(0xffffffffu, s1, 1);
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
    if (!uniform) {  // the run of the lane's first row ends inside this lane
      Astro tot = head;
      if (lane > 0 && s0 == prev_last) tot = astro_add(tot, vprev);
      astro_flush(x, s0, tot);
    }
    const int s0_next = __shfl_down_sync(0xffffffffu, s0, 1);
    if (lane == 31 || s0_next != s1) astro_flush(x, s1, V);
  }
  if (glob) {
    gacc = ff_warp_sum(gacc);
    if (lane == 0) red_ff(x + L.glob_col, gacc);
  }
}

// ---------------------------------------------------------------------------
// aprod 2, instrumental part. One block per tile of ct_rows rows (grid-stride).
// The tile's entries (coefficient, row, bin) of one column group are
// TMA-copied into shared memory together with the tile's u (two buffers: the
// block's next tile streams in while it works on the current one); each
// product is added into the block's float-pair histogram of the group's
// columns by a 64-bit compare-and-swap of the pair (lock-free: some thread
// wins every round of a conflict, and retries are bounded), so a tile needs no
// barrier between its entries. (Setup orders a tile's entries in rounds of
// distinct bins, so neighbouring threads rarely meet on one bin.) The
// histogram is added into x at the end.
// ---------------------------------------------------------------------------
constexpr int IU = 4;              // entries per thread per pass
constexpr int CAS_LIMIT = 1 << 16; // compare-and-swap attempts before giving up

// hist += p by compare-and-swap on the (hi, lo) pair; false if it gave up
__device__ __forceinline__ bool hist_add(float2* hist, ff p) {
  unsigned long long* h = reinterpret_cast<unsigned long long*>(hist);
  unsigned long long old = *reinterpret_cast<volatile unsigned long long*>(h);
  for (int i = 0; i < CAS_LIMIT; ++i) {
    const ff cur{__uint_as_float((unsigned)old), __uint_as_float((unsigned)(old >> 32))};
    const ff nh = ff_add(cur, p);
    const unsigned long long nv = (unsigned long long)__float_as_uint(nh.h) |
                                  ((unsigned long long)__float_as_uint(nh.l) << 32);
    const unsigned long long prev = atomicCAS(h, old, nv);
    if (prev == old) return true;
    old = prev;
  }
  return false;
}

template <bool F32, int NBUF, int NTH>
__global__ void __launch_bounds__(NTH, NTH == 512 ? 1 : 2)
    k_aprod2_instr(Layout L, const float2* __restrict__ y, double* __restrict__ x,
                   const double* stop) {
  if (stop && *stop != 0.0) return;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar[2];
  constexpr int VB = F32 ? 4 : 8;  // bytes per entry coefficient
  const int CT = L.ct_rows;
  // block -> (column group g, first tile); the grid is a multiple of the groups
  const int G = L.n_bgroups, g = blockIdx.x % G;
  const int64_t T = gridDim.x / G;
  const int bin_lo = g * L.bgroup_bins;
  const int nb = min(L.bgroup_bins, (int)L.n_instr - bin_lo);
  const int64_t KB = instr_keys_bytes(L.ct_max_ent), VBB = instr_vals_bytes(L.ct_max_ent, F32);
  const int64_t TB = KB + VBB + (int64_t)CT * 8;
  // [buffer 0 | buffer 1 | histogram of the group's columns], a buffer being
  // [keys | coefficients | u pairs CT], keys and coefficients of one segment
  float2* hist = reinterpret_cast<float2*>(smem + NBUF * TB);
  for (int i = threadIdx.x; i < nb; i += blockDim.x) hist[i] = make_float2(0.f, 0.f);
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_proxy_async();
  }
  __syncthreads();
  __shared__ int seg_n_s[2];  // entries of the segment in each buffer
  // (first entry, entries) of the segment of tile ct in this block's group
  auto seg_of = [&](int64_t ct) {
    return ct < L.n_ctiles ? L.iseg[ct * G + g] : make_longlong2(0, 0);
  };
  // thread 0: start the copies of segment sg (tile ct, group g) into buffer b
  auto issue = [&](int64_t ct, int b, longlong2 sg) {
    unsigned char* base = smem + b * TB;
    const int64_t e0 = sg.x, ne = sg.y;
    seg_n_s[b] = (int)ne;
    fence_proxy_async();
    // sizes rounded up to 16 bytes (segments start 16-byte aligned and the
    // entry arrays are padded); u is padded to whole tiles
    const uint32_t kb = (uint32_t)((ne * 4 + 15) & ~15LL);
    const uint32_t vb = (uint32_t)((ne * VB + 15) & ~15LL);
    const uint32_t ub = (uint32_t)CT * 8u;
    mbar_expect_tx(&bar[b], kb + vb + ub);
    tma_load(base + KB + VBB, y + ct * CT, ub, &bar[b]);
    if (ne > 0) {
      tma_load(base, L.ient_key + e0, kb, &bar[b]);
      if constexpr (F32) tma_load(base + KB, L.ient_f32 + e0, vb, &bar[b]);
      else tma_load(base + KB, L.ient_ff + e0, vb, &bar[b]);
    }
  };
  uint32_t parity = 0u, pending = 0u;  // bit q: phase / copy in flight of buffer q
  bool ok = true, cas_ok = true;
  int b = 0;
  const int64_t t0 = blockIdx.x / G;
  // thread 0 loads each segment's (first entry, entries) one copy ahead of
  // the copy that needs it, so that the load's latency stays off its path
  longlong2 nxt = make_longlong2(0, 0);
  if (threadIdx.x == 0) {
    if (NBUF == 2 && t0 < L.n_ctiles) issue(t0, 0, seg_of(t0));
    nxt = seg_of(NBUF == 2 ? t0 + T : t0);
  }
  if (NBUF == 2 && t0 < L.n_ctiles) pending = 1u;
  for (int64_t ct = t0; ct < L.n_ctiles; ct += T, b ^= (NBUF - 1)) {
    // the buffer written here was last read by the previous tile, which ended
    // in a barrier
    if (NBUF == 1) {
      if (threadIdx.x == 0) {
        issue(ct, 0, nxt);
        nxt = seg_of(ct + T);
      }
      pending = 1u;
    } else if (ct + T < L.n_ctiles) {
      if (threadIdx.x == 0) {
        issue(ct + T, b ^ 1, nxt);
        nxt = seg_of(ct + 2 * T);
      }
      pending |= 1u << (b ^ 1);
    }
    bool got = false;
    for (int i = 0; i < WAIT_LIMIT; ++i)
      if (mbar_try_wait(&bar[b], (parity >> b) & 1u)) {
        got = true;
        break;
      }
    if (!__syncthreads_and(got)) {
      if (threadIdx.x == 0) set_error(L.err, GSR_E_TIMEOUT);
      ok = false;
      break;
    }
    parity ^= 1u << b;
    pending &= ~(1u << b);
    const uint32_t* keys = reinterpret_cast<const uint32_t*>(smem + b * TB);
    const unsigned char* vals = smem + b * TB + KB;
    const float2* us = reinterpret_cast<const float2*>(smem + b * TB + KB + VBB);
    const int ne = seg_n_s[b];
    for (int e = threadIdx.x; e < ne; e += NTH * IU) {
      // IU entries per thread: their shared-memory reads issue together, then
      // each product goes into the histogram by compare-and-swap
      ff p[IU];
      int bin[IU];
#pragma unroll
      for (int j = 0; j < IU; ++j) {
        const int ej = e + j * NTH;
        bin[j] = -1;
        p[j] = ff_zero();
        if (ej < ne) {
          const uint32_t key = keys[ej];
          const int row = (int)(key >> INSTR_BIN_BITS);
          bin[j] = (int)(key & ((1u << INSTR_BIN_BITS) - 1)) - bin_lo;
          const float2 uu = us[row];
          if constexpr (F32) {
            p[j] = f_mul(reinterpret_cast<const float*>(vals)[ej], ff{uu.x, uu.y});
          } else {
            const float2 vv = reinterpret_cast<const float2*>(vals)[ej];
            p[j] = ff_mul(ff{vv.x, vv.y}, ff{uu.x, uu.y});
          }
        }
      }
#pragma unroll
      for (int j = 0; j < IU; ++j)
        if (bin[j] >= 0 && !hist_add(hist + bin[j], p[j])) cas_ok = false;
    }
    // every thread is done with buffer b before a copy into it is issued
    __syncthreads();
  }
  if (!cas_ok) set_error(L.err, GSR_E_TIMEOUT);
  if (!ok) {
    // let the copies still in flight land before the block exits (bounded)
    for (int q = 0; q < NBUF; ++q)
      if ((pending >> q) & 1u)
        for (int i = 0; i < WAIT_LIMIT / 16; ++i)
          if (mbar_try_wait(&bar[q], (parity >> q) & 1u)) break;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    const float2 h = hist[i];
    red_ff(x + L.instr_base + bin_lo + i, ff{h.x, h.y});
  }
}

// ---------------------------------------------------------------------------
// aprod 2, attitude part over the knot-ordered copies: positions with start
// knot s add into knots s..s+3 of each axis. A sliding 4-knot window per axis
// of per-lane partial sums lives in registers; knot s is final (for the warp)
// once its positions are done, and is then summed over the warp and added into
// x. Every load of a step (U positions per lane) is issued before any
// arithmetic.
// ---------------------------------------------------------------------------
// Attitude coefficient t of knot-order position p.
template <bool F32>
__device__ __forceinline__ ff att_val(const Layout& L, int t, int64_t p) {
  if constexpr (F32) {
    return ff{__ldcs(L.att_knot_f32 + (int64_t)t * L.n_rows + p), 0.0f};
  } else {
    const float2 a = __ldcs(L.att_knot_ff + (int64_t)t * L.n_rows + p);
    return ff{a.x, a.y};
  }
}

// A warp walks its range of start knots s; the rows of knot s are one run of
// the knot order, read 64 positions at a time (2 per lane): the coefficients
// in that order (coalesced). u comes from its copy in
// the same order, or (BLK) from the blocked copy, where the run of knot s is one
// segment per row block: lane b holds the bounds of block b's segment, and for
// each 64 positions the warp walks the segments that overlap them, every lane
// taking the blocked position of its own positions.
template <bool F32, bool BLK>
__global__ void __launch_bounds__(256) k_aprod2_att(Layout L, const float2* __restrict__ y_knot,
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
  const int64_t kb_w = L.n_knots - 2;
  const int nb = BLK ? L.n_kblk : 0;
  const bool own = lane < nb;
  const int32_t* kbl = BLK ? L.kb_start + (int64_t)(own ? lane : 0) * kb_w : nullptr;
  // bounds of block `lane`'s segment: the current knot's, the next loaded ahead
  int e0 = 0, e1 = 0;
  if (BLK && own) {
    e0 = kbl[s_begin];
    e1 = kbl[s_begin + 1];
  }
  // positions per lane per step: 2 keeps the float-pair kernel near 128
  // registers, so a block fits beside the instrumental kernel's block on every
  // SM; the FP32-value kernel stays at 128 registers with 3
  constexpr int U = F32 ? 3 : 2;
  for (int s = s_begin; s < s_end; ++s) {
    const int64_t p0 = L.knot_start[s], p1 = L.knot_start[s + 1];
    const int total = (int)(p1 - p0);
    // segment of block `lane`: blocked start a, length n, start c in the run
    int a = 0, n = 0, c = 0;
    if constexpr (BLK) {
      a = e0;
      n = e1 - e0;
      e0 = e1;
      if (own && s + 2 < kb_w) e1 = kbl[s + 2];
      c = n;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, c, d);
        if (lane >= d) c += y;
      }
      c -= n;
    }
    ff acc[12];
#pragma unroll
    for (int t = 0; t < 12; ++t) acc[t] = ff_zero();
    int bseg = 0;  // first segment that ends after the current step's start
    for (int qb = 0; qb < total; qb += 32 * U) {
      int64_t pu[U];
#pragma unroll
      for (int q = 0; q < U; ++q) pu[q] = p0 + qb + lane + 32 * q;
      if constexpr (BLK) {
        // skip the segments that end at or before qb (some segment ends after it)
        while (__shfl_sync(0xffffffffu, c + n, bseg) <= qb) ++bseg;
        for (int b = bseg; b < nb; ++b) {
          const int cb = __shfl_sync(0xffffffffu, c, b);
          if (cb >= qb + 32 * U) break;
          const int nbb = __shfl_sync(0xffffffffu, n, b), ab = __shfl_sync(0xffffffffu, a, b);
#pragma unroll
          for (int q = 0; q < U; ++q) {
            const int qi = qb + lane + 32 * q;
            if (qi >= cb && qi < cb + nbb) pu[q] = (int64_t)ab + (qi - cb);
          }
        }
      }
      ff u[U];
      ff v[12][U];
#pragma unroll
      for (int q = 0; q < U; ++q) {
        const int qi = qb + lane + 32 * q;
        const bool in = qi < total;
        const float2 uu = in ? __ldcs(y_knot + pu[q]) : make_float2(0.f, 0.f);
        u[q] = ff{uu.x, uu.y};
#pragma unroll
        for (int t = 0; t < 12; ++t) v[t][q] = in ? att_val<F32>(L, t, p0 + qi) : ff_zero();
      }
#pragma unroll
      for (int t = 0; t < 12; ++t) {
        ff sum = val_mul<F32>(v[t][0], u[0]);
#pragma unroll
        for (int q = 1; q < U; ++q) sum = ff_add(sum, val_mul<F32>(v[t][q], u[q]));
        acc[t] = ff_add(acc[t], sum);
      }
    }
    // the windows hold this lane's partial sums; only a finished knot is
    // reduced over the warp (3 values instead of 12 per bucket)
#pragma unroll
    for (int a3 = 0; a3 < 3; ++a3)
#pragma unroll
      for (int j = 0; j < 4; ++j) win[a3][j] = ff_add(win[a3][j], acc[4 * a3 + j]);
    {
      // knot s is complete for this warp
      const ff k0 = ff_warp_sum(win[0][0]), k1 = ff_warp_sum(win[1][0]),
               k2 = ff_warp_sum(win[2][0]);
      if (lane < 3) red_ff(x + L.att_base + lane * K + s, lane == 0 ? k0 : lane == 1 ? k1 : k2);
    }
#pragma unroll
    for (int a3 = 0; a3 < 3; ++a3) {
      win[a3][0] = win[a3][1];
      win[a3][1] = win[a3][2];
      win[a3][2] = win[a3][3];
      win[a3][3] = ff_zero();
    }
  }
  // the three knots after the last bucket also received contributions
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const ff k0 = ff_warp_sum(win[0][j]), k1 = ff_warp_sum(win[1][j]), k2 = ff_warp_sum(win[2][j]);
    if (lane < 3)
      red_ff(x + L.att_base + lane * K + s_end + j, lane == 0 ? k0 : lane == 1 ? k1 : k2);
  }
}

// ---------------------------------------------------------------------------
// FP64 products for inputs outside the float-pair band (and for systems whose
// rescaled coefficients are too spread for it). One thread per row, the
// coefficient of the stored record widened exactly and scaled back by
// 2^-(e_i + g_j), products and sums in FP64 (aprod 2 adds into x with FP64 L2
// atomics). They run only when *guard != 0 (guard null: always), so that the
// choice between them and the float-pair kernels is made on the device.
// ---------------------------------------------------------------------------
template <bool F32>
__device__ __forceinline__ int64_t rec_col(const Layout& L, const unsigned char* rec, int t,
                                           int ri) {
  using R = Rec<F32>;
  if (t < 5) return 5 * (int64_t)reinterpret_cast<const int*>(rec + R::STAR)[ri] + t;
  if (t < 17)
    return L.att_base + ((t - 5) >> 2) * L.n_knots +
           reinterpret_cast<const int*>(rec + R::ATT_S)[ri] + ((t - 5) & 3);
  if (t < 23)
    return L.instr_base +
           reinterpret_cast<const unsigned short*>(rec + R::INSTR_I + (t - 17) * 128)[ri];
  return L.glob_col;
}

// Original coefficient A_it (from the rescaled stored value) and its column.
template <bool F32>
__device__ __forceinline__ double rec_coef_f64(const Layout& L, const unsigned char* rec, int t,
                                               int ri, int e, int64_t col) {
  const ff v = rec_val1<F32>(rec, t, ri);
  double a = __dadd_rn((double)v.h, (double)v.l);
  const int sh = e + (L.col_exp ? (int)L.col_exp[col] : 0);
  return sh ? ldexp(a, -sh) : a;
}

// k right-hand sides interleaved (x[col * k + j], y[row * k + j]); k = 1 for
// the single-vector form.
template <bool F32>
__global__ void k_aprod1_f64(Layout L, const double* __restrict__ x, int k, int neg,
                             double* __restrict__ y, const double* guard) {
  if (guard && *guard == 0.0) return;
  using R = Rec<F32>;
  const unsigned char* recs = F32 ? L.rec_f32 : L.rec_ff;
  const int nt = L.n_glob == 1 ? NSLOT : NSLOT - 1;
  for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < L.n_rows;
       row += (int64_t)gridDim.x * blockDim.x) {
    const unsigned char* rec = recs + (row / REC_ROWS) * R::BYTES;
    const int ri = (int)(row % REC_ROWS);
    const int e = L.row_exp ? (int)L.row_exp[row] : 0;
    for (int j = 0; j < k; ++j) {
      double acc = 0.0;
      for (int t = 0; t < nt; ++t) {
        const int64_t col = rec_col<F32>(L, rec, t, ri);
        acc = __fma_rn(rec_coef_f64<F32>(L, rec, t, ri, e, col), x[col * k + j], acc);
      }
      y[row * k + j] += neg ? -acc : acc;
    }
  }
}

template <bool F32>
__global__ void k_aprod2_f64(Layout L, const double* __restrict__ y, int k,
                             double* __restrict__ x, const double* guard) {
  if (guard && *guard == 0.0) return;
  using R = Rec<F32>;
  const unsigned char* recs = F32 ? L.rec_f32 : L.rec_ff;
  const int nt = L.n_glob == 1 ? NSLOT : NSLOT - 1;
  for (int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; row < L.n_rows;
       row += (int64_t)gridDim.x * blockDim.x) {
    const unsigned char* rec = recs + (row / REC_ROWS) * R::BYTES;
    const int ri = (int)(row % REC_ROWS);
    const int e = L.row_exp ? (int)L.row_exp[row] : 0;
    for (int t = 0; t < nt; ++t) {
      const int64_t col = rec_col<F32>(L, rec, t, ri);
      const double a = rec_coef_f64<F32>(L, rec, t, ri, e, col);
      for (int j = 0; j < k; ++j) {
        const double yi = y[row * k + j];
        if (yi != 0.0) atomicAdd(x + col * k + j, __dmul_rn(a, yi));
      }
    }
  }
}

// x += 2^-g_j z_j (the column exponents of a rescaled aprod 2), unless *guard.
__global__ void k_add_rescaled(int64_t n, const double* __restrict__ z,
                               const int16_t* __restrict__ cexp, double* __restrict__ x,
                               const double* guard) {
  if (guard && *guard != 0.0) return;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x)
    x[j] += ldexp(z[j], -(int)cexp[j]);
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
constexpr int A1_NP = 6;                    // warp pairs per aprod 1 block (one block per SM)
constexpr int A1_NS_FF = 2, A1_NS_F32 = 3;  // record buffers per warp pair
constexpr int A1_XI_SMEM_MAX = 6144;        // instrumental unknowns staged in shared memory
// More instrumental unknowns than that: one record buffer per pair and five
// pairs, so that all of them still fit beside the buffers (up to ~20,000 with
// float-pair values; measured on 160M rows x 20,000 columns: 12.06 -> 11.74 ms,
// and with FP32 values, which gathered them through L2 before, 8.47 -> 6.31 ms)
constexpr int A1_NP1 = 5;
constexpr int A1_SMEM_MAX = 226 * 1024;  // dynamic shared memory of that configuration

int cuda_status(cudaError_t e) { return e == cudaSuccess ? GSR_OK : GSR_E_CUDA; }

int set_kernel_attributes() {
  cudaError_t e = cudaSuccess;
  auto C = [&](cudaError_t r) {
    if (e == cudaSuccess) e = r;
  };
  const int ff_bytes = A1_NP * A1_NS_FF * Rec<false>::BYTES + A1_XI_SMEM_MAX * 8;
  const int f32_bytes = A1_NP * A1_NS_F32 * Rec<true>::BYTES + A1_XI_SMEM_MAX * 8;
  C(cudaFuncSetAttribute(k_aprod1<false, true, true, A1_NP, A1_NS_FF>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, ff_bytes));
  C(cudaFuncSetAttribute(k_aprod1<false, false, true, A1_NP, A1_NS_FF>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, ff_bytes));
  C(cudaFuncSetAttribute(k_aprod1<false, false, false, A1_NP, A1_NS_FF>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, ff_bytes));
  C(cudaFuncSetAttribute(k_aprod1<true, true, true, A1_NP, A1_NS_F32>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, f32_bytes));
  C(cudaFuncSetAttribute(k_aprod1<true, false, true, A1_NP, A1_NS_F32>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, f32_bytes));
  C(cudaFuncSetAttribute(k_aprod1<true, false, false, A1_NP, A1_NS_F32>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, f32_bytes));
#define GSR_A1W_ATTR(F, YF, X3, NP)                                                       \
  C(cudaFuncSetAttribute(k_aprod1<F, YF, X3, NP, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                         A1_SMEM_MAX));
  GSR_A1W_ATTR(false, true, true, A1_NP1) GSR_A1W_ATTR(false, false, true, A1_NP1)
  GSR_A1W_ATTR(false, false, false, A1_NP1) GSR_A1W_ATTR(true, true, true, A1_NP1)
  GSR_A1W_ATTR(true, false, true, A1_NP1) GSR_A1W_ATTR(true, false, false, A1_NP1)
#undef GSR_A1W_ATTR
#define GSR_INSTR_ATTR(F, B, T)                                                             \
  C(cudaFuncSetAttribute(k_aprod2_instr<F, B, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                         INSTR_SMEM_BUDGET));
  GSR_INSTR_ATTR(false, 1, 256) GSR_INSTR_ATTR(true, 1, 256)
  GSR_INSTR_ATTR(false, 2, 512) GSR_INSTR_ATTR(true, 2, 512)
#undef GSR_INSTR_ATTR
  return cuda_status(e);
}

int launch_to_ff(const double* x, const double* scale, const int16_t* cexp, int neg,
                 double* guard, float2* out, int64_t n, cudaStream_t st) {
  if (n <= 0) return GSR_OK;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 148 * 8) blocks = 148 * 8;
  k_to_ff<<<blocks, 256, 0, st>>>(x, scale, cexp, neg, guard, out, n);
  return cuda_status(cudaGetLastError());
}

int launch_to_ff_knot(gsr_system* sys, int which_values, const double* y, float2* y_ff,
                      float2* y_knot, double* guard, cudaStream_t st) {
  if (sys->L.n_rows <= 0) return GSR_OK;
  int blocks = (int)((sys->L.n_rows + 255) / 256);
  if (blocks > sys->num_sms * 8) blocks = sys->num_sms * 8;
  k_to_ff_knot<<<blocks, 256, 0, st>>>(sys->L, y, y_ff, y_knot, knot_positions(sys->L, which_values),
                                       guard);
  return cuda_status(cudaGetLastError());
}

int launch_att_x3(gsr_system* sys, const float2* x_ff, const double* stop, cudaStream_t st) {
  const int64_t n = (sys->L.n_knots - 3) * 12;
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sys->num_sms * 4);
  k_att_x3<<<blocks, 256, 0, st>>>(sys->L, x_ff, sys->S.x3, stop);
  return cuda_status(cudaGetLastError());
}

// aprod 1 reads x_ff and its knot-interleaved attitude copy sys->S.x3 (built by
// launch_att_x3 from the same x_ff beforehand).
template <bool YFF, bool X3>
static int launch_aprod1_t(gsr_system* sys, int which_values, const float2* x_ff, void* y,
                           const double* coef_dev, double coef_host, float2* y_knot,
                           double* norm_slot, const double* stop, cudaStream_t st) {
  const Layout& L = sys->L;
  if (L.n_recs <= 0) {
    if (norm_slot) return cuda_status(cudaMemsetAsync(norm_slot, 0, sizeof(double), st));
    return GSR_OK;
  }
  const bool f32 = which_values == GSR_VALUES_F32;
  const int64_t smem1 =
      (int64_t)A1_NP1 * (f32 ? Rec<true>::BYTES : Rec<false>::BYTES) + L.n_instr * 8;
  if (L.n_instr > A1_XI_SMEM_MAX && smem1 <= A1_SMEM_MAX) {
    // A1_NP1 pairs with one buffer each, every instrumental unknown staged
    const int64_t need1 = (L.n_recs + A1_NP1 - 1) / A1_NP1;
    const int b1 = need1 < sys->num_sms ? (int)need1 : sys->num_sms;
    if (f32)
      k_aprod1<true, YFF, X3, A1_NP1, 1><<<b1, A1_NP1 * 64, (int)smem1, st>>>(
          L, x_ff, sys->S.x3, y, coef_dev, coef_host, y_knot, sys->S.red, sys->S.count,
          norm_slot, stop, 1);
    else
      k_aprod1<false, YFF, X3, A1_NP1, 1><<<b1, A1_NP1 * 64, (int)smem1, st>>>(
          L, x_ff, sys->S.x3, y, coef_dev, coef_host, y_knot, sys->S.red, sys->S.count,
          norm_slot, stop, 1);
    return cuda_status(cudaGetLastError());
  }
  int blocks = sys->num_sms;
  const int64_t need = (L.n_recs + A1_NP - 1) / A1_NP;
  if (need < blocks) blocks = (int)need;
  const int xi = L.n_instr <= A1_XI_SMEM_MAX ? 1 : 0;
  const int xib = xi ? (int)L.n_instr * 8 : 0;
  // A1_NP pairs of warps, each pair with its own record buffers
  if (f32)
    k_aprod1<true, YFF, X3, A1_NP, A1_NS_F32>
        <<<blocks, A1_NP * 64, A1_NP * A1_NS_F32 * Rec<true>::BYTES + xib, st>>>(
            L, x_ff, sys->S.x3, y, coef_dev, coef_host, y_knot, sys->S.red, sys->S.count,
            norm_slot, stop, xi);
  else
    k_aprod1<false, YFF, X3, A1_NP, A1_NS_FF>
        <<<blocks, A1_NP * 64, A1_NP * A1_NS_FF * Rec<false>::BYTES + xib, st>>>(
            L, x_ff, sys->S.x3, y, coef_dev, coef_host, y_knot, sys->S.red, sys->S.count,
            norm_slot, stop, xi);
  return cuda_status(cudaGetLastError());
}

int launch_aprod1(gsr_system* sys, int which_values, const float2* x_ff, double* y,
                  const double* coef_dev, double coef_host, double* y_knot, double* norm_slot,
                  const double* stop, cudaStream_t st) {
  if (y_knot) return GSR_E_ARG;  // the knot-order copy exists for the float-pair form only
  return launch_aprod1_t<false, false>(sys, which_values, x_ff, y, coef_dev, coef_host, nullptr,
                                       norm_slot, stop, st);
}

int launch_aprod1_x3(gsr_system* sys, int which_values, const float2* x_ff, double* y,
                     const double* stop, cudaStream_t st) {
  return launch_aprod1_t<false, true>(sys, which_values, x_ff, y, nullptr, 1.0, nullptr, nullptr,
                                      stop, st);
}

int launch_aprod1_ff(gsr_system* sys, int which_values, const float2* x_ff, float2* y,
                     const double* coef_dev, float2* y_knot, double* norm_slot,
                     const double* stop, cudaStream_t st) {
  return launch_aprod1_t<true, true>(sys, which_values, x_ff, y, coef_dev, 0.0, y_knot, norm_slot,
                                     stop, st);
}

int launch_aprod2(gsr_system* sys, int which_values, const float2* y, const float2* y_knot,
                  double* x, const double* stop, cudaStream_t st) {
  const Layout& L = sys->L;
  if (L.n_rows <= 0) return GSR_OK;
  const bool f32 = which_values == GSR_VALUES_F32;
  // The latency-bound instrumental part is launched first on the caller's
  // stream; the attitude and then the astrometric part, which stream at full
  // bandwidth, run beside it on the side stream.
  if (cudaEventRecord(sys->ev_fork, st) != cudaSuccess) return GSR_E_CUDA;
  if (cudaStreamWaitEvent(sys->side, sys->ev_fork, 0) != cudaSuccess) return GSR_E_CUDA;
  // G column groups, each over tile streams of num_sms * per_sm / G blocks
  const int64_t per_group = std::max<int64_t>(
      1, std::min<int64_t>((int64_t)sys->num_sms * L.ct_per_sm / L.n_bgroups, L.n_ctiles));
  const int ib = (int)(per_group * L.n_bgroups);
  const int ismem =
      (int)instr_smem_bytes(L.ct_rows, L.ct_max_ent, L.bgroup_bins, f32, L.ct_bufs);
  if (L.n_ctiles > 0) {
    if (L.ct_per_sm == 1) {
      if (f32) k_aprod2_instr<true, 2, 512><<<ib, 512, ismem, st>>>(L, y, x, stop);
      else k_aprod2_instr<false, 2, 512><<<ib, 512, ismem, st>>>(L, y, x, stop);
    } else {
      if (f32) k_aprod2_instr<true, 1, 256><<<ib, 256, ismem, st>>>(L, y, x, stop);
      else k_aprod2_instr<false, 1, 256><<<ib, 256, ismem, st>>>(L, y, x, stop);
    }
    if (cudaGetLastError() != cudaSuccess) return GSR_E_CUDA;
  }
  const int att_blocks = (L.n_att_warps + 7) / 8;
  if (att_blocks > 0) {
    // the float-pair copy of u is blocked when n_kblk > 1; the FP32 one never
    if (f32) k_aprod2_att<true, false><<<att_blocks, 256, 0, sys->side>>>(L, y_knot, x, stop);
    else if (L.n_kblk > 1)
      k_aprod2_att<false, true><<<att_blocks, 256, 0, sys->side>>>(L, y_knot, x, stop);
    else k_aprod2_att<false, false><<<att_blocks, 256, 0, sys->side>>>(L, y_knot, x, stop);
    if (cudaGetLastError() != cudaSuccess) return GSR_E_CUDA;
  }
  const int ab = (int)std::min<int64_t>((int64_t)sys->num_sms * 8, ((L.n_recs + 1) / 2 + 7) / 8);
  if (f32) k_aprod2_astro<true><<<ab, 256, 0, sys->side>>>(L, y, x, stop);
  else k_aprod2_astro<false><<<ab, 256, 0, sys->side>>>(L, y, x, stop);
  if (cudaGetLastError() != cudaSuccess) return GSR_E_CUDA;
  if (cudaEventRecord(sys->ev_join, sys->side) != cudaSuccess) return GSR_E_CUDA;
  if (cudaStreamWaitEvent(st, sys->ev_join, 0) != cudaSuccess) return GSR_E_CUDA;
  return GSR_OK;
}

int launch_aprod1_f64(gsr_system* sys, int which_values, const double* x, int k, int neg,
                      double* y, const double* guard, cudaStream_t st) {
  const Layout& L = sys->L;
  if (L.n_rows <= 0) return GSR_OK;
  const int blocks = (int)std::min<int64_t>((L.n_rows + 255) / 256, (int64_t)sys->num_sms * 8);
  if (which_values == GSR_VALUES_F32)
    k_aprod1_f64<true><<<blocks, 256, 0, st>>>(L, x, k, neg, y, guard);
  else
    k_aprod1_f64<false><<<blocks, 256, 0, st>>>(L, x, k, neg, y, guard);
  return cuda_status(cudaGetLastError());
}

int launch_aprod2_f64(gsr_system* sys, int which_values, const double* y, int k, double* x,
                      const double* guard, cudaStream_t st) {
  const Layout& L = sys->L;
  if (L.n_rows <= 0) return GSR_OK;
  const int blocks = (int)std::min<int64_t>((L.n_rows + 255) / 256, (int64_t)sys->num_sms * 8);
  if (which_values == GSR_VALUES_F32)
    k_aprod2_f64<true><<<blocks, 256, 0, st>>>(L, y, k, x, guard);
  else
    k_aprod2_f64<false><<<blocks, 256, 0, st>>>(L, y, k, x, guard);
  return cuda_status(cudaGetLastError());
}

// The observation rows of a direct aprod 1 (float-pair kernels or FP64).
static int aprod1_direct_obs(gsr_system* sys, int which_values, const double* x, int neg,
                             double* y, cudaStream_t st) {
  const Layout& L = sys->L;
  if (L.n_rows <= 0) return GSR_OK;
  if (sys->wide) return launch_aprod1_f64(sys, which_values, x, 1, neg, y, nullptr, st);
  double* guard = sys->S.guard;
  if (cudaMemsetAsync(guard, 0, sizeof(double), st) != cudaSuccess) return GSR_E_CUDA;
  int rc = launch_to_ff(x, nullptr, L.col_exp, neg, guard, sys->S.x_ff, L.n_unk, st);
  if (rc != GSR_OK) return rc;
  rc = launch_att_x3(sys, sys->S.x_ff, guard, st);
  if (rc != GSR_OK) return rc;
  rc = launch_aprod1_x3(sys, which_values, sys->S.x_ff, y, guard, st);
  if (rc != GSR_OK) return rc;
  return launch_aprod1_f64(sys, which_values, x, 1, neg, y, guard, st);
}

int aprod1_direct(gsr_system* sys, int which_values, const double* x, int neg, double* y,
                  cudaStream_t st) {
  const int rc = aprod1_direct_obs(sys, which_values, x, neg, y, st);
  if (rc != GSR_OK) return rc;
  return con_aprod1_direct(sys, x, neg, y, st);  // the constraint rows (FP64)
}

// The observation rows of a direct aprod 2.
static int aprod2_direct_obs(gsr_system* sys, int which_values, const double* y, double* x,
                             cudaStream_t st) {
  const Layout& L = sys->L;
  if (L.n_rows <= 0) return GSR_OK;
  if (sys->wide) return launch_aprod2_f64(sys, which_values, y, 1, x, nullptr, st);
  double* guard = sys->S.guard;
  if (cudaMemsetAsync(guard, 0, sizeof(double), st) != cudaSuccess) return GSR_E_CUDA;
  int rc = launch_to_ff_knot(sys, which_values, y, sys->S.y_ff, sys->S.y_knot, guard, st);
  if (rc != GSR_OK) return rc;
  double* acc = L.col_exp ? sys->S.zx : x;
  if (L.col_exp &&
      cudaMemsetAsync(sys->S.zx, 0, (size_t)L.n_unk * sizeof(double), st) != cudaSuccess)
    return GSR_E_CUDA;
  rc = launch_aprod2(sys, which_values, sys->S.y_ff, sys->S.y_knot, acc, guard, st);
  if (rc != GSR_OK) return rc;
  if (L.col_exp) {
    const int blocks = (int)std::min<int64_t>((L.n_unk + 255) / 256, (int64_t)sys->num_sms * 8);
    k_add_rescaled<<<blocks, 256, 0, st>>>(L.n_unk, sys->S.zx, L.col_exp, x, guard);
    if (cudaGetLastError() != cudaSuccess) return GSR_E_CUDA;
  }
  return launch_aprod2_f64(sys, which_values, y, 1, x, guard, st);
}

int aprod2_direct(gsr_system* sys, int which_values, const double* y, double* x,
                  cudaStream_t st) {
  const int rc = aprod2_direct_obs(sys, which_values, y, x, st);
  if (rc != GSR_OK) return rc;
  return con_aprod2_direct(sys, y, x, st);
}

}  // namespace gsr
