// Learned column preconditioner: per-column features of the attitude and
// instrumental blocks, a small MLP (8 -> 64 -> 64 -> 1) that maps them to a
// log multiplier of the column scaling, its training (MSE gradient + Adam) and
// the scaling d_j = exp(m_j) / ||A_:,j|| handed to LSQR.
//
// The paper preconditions by column scaling only (Sec. 2); the learned part
// changes how the attitude / instrumental columns are weighted and therefore
// only the iteration count, never the least-squares solution.
//
// Arithmetic: weights and activations (and the activation gradients) are
// BF16, every product runs on the tensor cores as mma.sync m16n8k16 BF16 with
// FP32 accumulation; biases, the output, the loss and Adam are FP32.
#include <cuda_bf16.h>

#include <cmath>
#include <cstdint>

#include "gsr_system.cuh"

namespace gsr {

namespace {

constexpr int NF = GSR_MLP_NFEAT;    // 8
constexpr int NH = GSR_MLP_HIDDEN;   // 64
constexpr int NP = GSR_MLP_NPARAM;   // 4801
constexpr int O_W1 = 0, O_B1 = O_W1 + NH * NF, O_W2 = O_B1 + NH, O_B2 = O_W2 + NH * NH,
              O_W3 = O_B2 + NH, O_B3 = O_W3 + NH;
static_assert(O_B3 + 1 == NP, "parameter layout");
constexpr int WS = NH + 8;           // padded bf16 row stride of the smem weight tiles

// ---------------------------------------------------------------------------
// Features of column q (q < 3K: attitude axis q / K, knot q % K; else
// instrumental column q - 3K), computed in FP64 and stored as float:
//   f0 log ||A_:,j||              f4 position in the block (knot or instrument index, 0..1)
//   f1 log(1 + n_j)               f5 log of the block's mean observation count
//   f2 1 for instrumental         f6 f1 - log(1 + mean count)  (relative density)
//   f3 axis / 2 (attitude)        f7 log(||A_:,j|| / sqrt(max(n_j, 1)))  (rms coefficient)
// n_j is the number of rows with a coefficient slot in column j.
// ---------------------------------------------------------------------------
__global__ void k_instr_count(Layout L, int* __restrict__ cnt) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < L.n_rows;
       r += (int64_t)gridDim.x * blockDim.x) {
    const unsigned short* ins =
        reinterpret_cast<const unsigned short*>(L.rec_ff + (r >> 6) * Rec<false>::BYTES +
                                                Rec<false>::INSTR_I) + (r & 63);
#pragma unroll
    for (int k = 0; k < 6; ++k) atomicAdd(cnt + ins[k * 64], 1);
  }
}

__global__ void k_features(Layout L, const double* __restrict__ colnorm,
                           const int* __restrict__ icnt, float* __restrict__ feats) {
  const int64_t K = L.n_knots, nq = 3 * K + L.n_instr;
  const double mean_att = K > 0 ? 4.0 * (double)L.n_rows / (double)K : 0.0;
  const double mean_ins = L.n_instr > 0 ? 6.0 * (double)L.n_rows / (double)L.n_instr : 0.0;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nq;
       q += (int64_t)gridDim.x * blockDim.x) {
    const bool ins = q >= 3 * K;
    double n, pos, axis, mean;
    if (!ins) {
      const int64_t a = q / K, kn = q % K;
      // rows whose 4-knot window [s, s+3] covers knot kn
      const int64_t s0 = kn - 3 > 0 ? kn - 3 : 0, s1 = kn < K - 4 ? kn : K - 4;
      n = s1 >= s0 ? (double)(L.knot_start[s1 + 1] - L.knot_start[s0]) : 0.0;
      pos = K > 1 ? (double)kn / (double)(K - 1) : 0.0;
      axis = 0.5 * (double)a;
      mean = mean_att;
    } else {
      const int64_t i = q - 3 * K;
      n = (double)icnt[i];
      pos = L.n_instr > 1 ? (double)i / (double)(L.n_instr - 1) : 0.0;
      axis = 0.0;
      mean = mean_ins;
    }
    const double c = colnorm[L.att_base + q];
    const double lc = c > 0.0 ? log(c) : 0.0;
    const double l1n = log1p(n);
    const double lm = mean > 0.0 ? log(mean) : 0.0;
    float* f = feats + q * NF;
    f[0] = (float)lc;
    f[1] = (float)l1n;
    f[2] = ins ? 1.0f : 0.0f;
    f[3] = (float)axis;
    f[4] = (float)pos;
    f[5] = (float)lm;
    f[6] = (float)(l1n - log1p(mean));
    f[7] = (float)(lc - 0.5 * log(n > 1.0 ? n : 1.0));
  }
}

// Running sums of f and f^2 over n feature rows (for the standardisation).
__global__ void k_feature_moments(const float* __restrict__ f, int64_t n, double* __restrict__ acc) {
  double s[2 * NF];
#pragma unroll
  for (int k = 0; k < 2 * NF; ++k) s[k] = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
#pragma unroll
    for (int k = 0; k < NF; ++k) {
      const double v = f[i * NF + k];
      s[k] += v;
      s[NF + k] += v * v;
    }
#pragma unroll
  for (int k = 0; k < 2 * NF; ++k) {
    double v = s[k];
    for (int m = 16; m >= 1; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
    if ((threadIdx.x & 31) == 0) atomicAdd(acc + k, v);
  }
}

// ---------------------------------------------------------------------------
// Tensor-core helpers (mma.sync m16n8k16, BF16 inputs, FP32 accumulate).
// Fragment ownership (g = lane / 4, t = lane % 4):
//   A 16x16: {a0,a1} (g, 2t..2t+1), {a2,a3} (g+8, 2t..), {a4,a5} (g, 2t+8..), {a6,a7} (g+8, 2t+8..)
//   B 16x8 : {b0,b1} (k 2t..2t+1, n g), {b2,b3} (k 2t+8.., n g)
//   C 16x8 : c0,c1 (g, 2t..2t+1), c2,c3 (g+8, 2t..2t+1)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
// two floats -> bf16x2 (lo in the low half), round to nearest even
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}
__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }
__device__ __forceinline__ float lo_f(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float hi_f(uint32_t v) { return __uint_as_float(v & 0xffff0000u); }
__device__ __forceinline__ uint32_t ld_pair(const __nv_bfloat16* p) {
  return *reinterpret_cast<const uint32_t*>(p);
}
__device__ __forceinline__ uint32_t ld2(const __nv_bfloat16* p0, const __nv_bfloat16* p1) {
  return (uint32_t)__bfloat16_as_ushort(*p0) | ((uint32_t)__bfloat16_as_ushort(*p1) << 16);
}

struct MlpSmem {
  __nv_bfloat16 W1[NH][16];   // [hidden][input], inputs 8..15 zero
  __nv_bfloat16 W2[NH][WS];   // [out][in]
  float b1[NH], b2[NH], w3[NH];  // w3 holds its BF16-rounded value
  float b3;
  float mean[NF], istd[NF];
};

__device__ void load_weights(MlpSmem& s, const float* __restrict__ th,
                             const float* __restrict__ nrm) {
  for (int i = threadIdx.x; i < NH * 16; i += blockDim.x) {
    const int h = i / 16, k = i % 16;
    s.W1[h][k] = __float2bfloat16_rn(k < NF ? th[O_W1 + h * NF + k] : 0.0f);
  }
  for (int i = threadIdx.x; i < NH * NH; i += blockDim.x) {
    const int o = i / NH, k = i % NH;
    s.W2[o][k] = __float2bfloat16_rn(th[O_W2 + i]);
  }
  for (int i = threadIdx.x; i < NH; i += blockDim.x) {
    s.b1[i] = th[O_B1 + i];
    s.b2[i] = th[O_B2 + i];
    s.w3[i] = bf16r(th[O_W3 + i]);
  }
  if (threadIdx.x < NF) {
    s.mean[threadIdx.x] = nrm[threadIdx.x];
    s.istd[threadIdx.x] = nrm[NF + threadIdx.x];
  }
  if (threadIdx.x == 0) s.b3 = th[O_B3];
  __syncthreads();
}

// standardised feature k of sample row (0 outside [0, n))
__device__ __forceinline__ float feat(const MlpSmem& s, const float* __restrict__ f, int64_t row,
                                      int64_t n, int k) {
  if (row >= n) return 0.0f;
  return __fmul_rn(__fsub_rn(__ldg(f + row * NF + k), s.mean[k]), s.istd[k]);
}

// Forward pass of one 16-sample tile held by one warp. Outputs: the layer-1
// activations as A fragments (h1a[kc], hidden units kc*16..kc*16+15), the
// layer-2 activations in C layout (h2[nt][*], units nt*8 + 2t + {0,1}), and
// the network output of rows g and g+8 (m[0], m[1], in all 4 lanes of the group).
__device__ __forceinline__ void mlp_tile_fwd(const MlpSmem& s, const float* __restrict__ f,
                                             int64_t r0, int64_t n, uint32_t (&h1a)[4][4],
                                             float (&h2)[8][4], float (&m)[2]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  uint32_t a1[4];
  a1[0] = pack_bf16(feat(s, f, r0 + g, n, 2 * t), feat(s, f, r0 + g, n, 2 * t + 1));
  a1[1] = pack_bf16(feat(s, f, r0 + g + 8, n, 2 * t), feat(s, f, r0 + g + 8, n, 2 * t + 1));
  a1[2] = 0u;
  a1[3] = 0u;
  float c1[8][4];
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const float bb0 = s.b1[nt * 8 + 2 * t], bb1 = s.b1[nt * 8 + 2 * t + 1];
    c1[nt][0] = bb0;
    c1[nt][1] = bb1;
    c1[nt][2] = bb0;
    c1[nt][3] = bb1;
    mma16816(c1[nt], a1, ld_pair(&s.W1[nt * 8 + g][2 * t]), 0u);
  }
#pragma unroll
  for (int kc = 0; kc < 4; ++kc) {
    h1a[kc][0] = pack_bf16(fmaxf(c1[2 * kc][0], 0.f), fmaxf(c1[2 * kc][1], 0.f));
    h1a[kc][1] = pack_bf16(fmaxf(c1[2 * kc][2], 0.f), fmaxf(c1[2 * kc][3], 0.f));
    h1a[kc][2] = pack_bf16(fmaxf(c1[2 * kc + 1][0], 0.f), fmaxf(c1[2 * kc + 1][1], 0.f));
    h1a[kc][3] = pack_bf16(fmaxf(c1[2 * kc + 1][2], 0.f), fmaxf(c1[2 * kc + 1][3], 0.f));
  }
  float p0 = 0.f, p1 = 0.f;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const float bb0 = s.b2[nt * 8 + 2 * t], bb1 = s.b2[nt * 8 + 2 * t + 1];
    float c[4] = {bb0, bb1, bb0, bb1};
#pragma unroll
    for (int kc = 0; kc < 4; ++kc)
      mma16816(c, h1a[kc], ld_pair(&s.W2[nt * 8 + g][kc * 16 + 2 * t]),
               ld_pair(&s.W2[nt * 8 + g][kc * 16 + 8 + 2 * t]));
#pragma unroll
    for (int e = 0; e < 4; ++e) h2[nt][e] = bf16r(fmaxf(c[e], 0.f));
    const float w0 = s.w3[nt * 8 + 2 * t], w1 = s.w3[nt * 8 + 2 * t + 1];
    p0 = __fmaf_rn(h2[nt][0], w0, __fmaf_rn(h2[nt][1], w1, p0));
    p1 = __fmaf_rn(h2[nt][2], w0, __fmaf_rn(h2[nt][3], w1, p1));
  }
  p0 += __shfl_xor_sync(0xffffffffu, p0, 1);
  p0 += __shfl_xor_sync(0xffffffffu, p0, 2);
  p1 += __shfl_xor_sync(0xffffffffu, p1, 1);
  p1 += __shfl_xor_sync(0xffffffffu, p1, 2);
  m[0] = p0 + s.b3;
  m[1] = p1 + s.b3;
}

__global__ void __launch_bounds__(128) k_mlp_fwd(const float* __restrict__ f, int64_t n,
                                                 const float* __restrict__ nrm,
                                                 const float* __restrict__ theta,
                                                 float* __restrict__ out) {
  __shared__ MlpSmem s;
  load_weights(s, theta, nrm);
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int64_t nt16 = (n + 15) / 16;
  const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t tile = w0; tile < nt16; tile += nw) {
    uint32_t h1a[4][4];
    float h2[8][4], m[2];
    const int64_t r0 = tile * 16;
    mlp_tile_fwd(s, f, r0, n, h1a, h2, m);
    if (t == 0) {
      if (r0 + g < n) out[r0 + g] = m[0];
      if (r0 + g + 8 < n) out[r0 + g + 8] = m[1];
    }
  }
}

// ---------------------------------------------------------------------------
// Gradient of L = (1/n) sum (m_i - t_i)^2. A block of 4 warps takes 64 samples
// per step: each warp recomputes the forward pass of its 16 rows and forms
// dz2 = g w3 [h2 > 0] and dz1 = (dz2 W2) [h1 > 0] (BF16); the tiles go to
// shared memory, and warp w then accumulates rows 16w..16w+15 of
// dW2 = dz2^T h1 and dW1 = dz1^T f (plus db1 through a column of ones in f)
// over the 64 samples on the tensor cores. Every block writes its partial
// gradient; k_mlp_reduce adds the partials in block order (deterministic).
// ---------------------------------------------------------------------------
struct GradTiles {
  __nv_bfloat16 dz2[64][WS];
  __nv_bfloat16 h1[64][WS];
  __nv_bfloat16 dz1[64][WS];
  __nv_bfloat16 f[64][24];  // standardised inputs, column 8 = 1 (bias), 9..15 = 0
  float red[4][2 * NH + 2];
};

__global__ void __launch_bounds__(128) k_mlp_grad(const float* __restrict__ f,
                                                  const float* __restrict__ target, int64_t n,
                                                  const float* __restrict__ nrm,
                                                  const float* __restrict__ theta,
                                                  float* __restrict__ part) {
  __shared__ MlpSmem s;
  __shared__ GradTiles T;
  load_weights(s, theta, nrm);
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3, w = threadIdx.x >> 5;
  const float inv_n = 2.0f / (float)n;
  float dW2[8][4], dW1[2][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int e = 0; e < 4; ++e) dW2[i][e] = 0.f;
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int e = 0; e < 4; ++e) dW1[i][e] = 0.f;
  float dw3[16], db2[16], db3 = 0.f, lsum = 0.f;
#pragma unroll
  for (int i = 0; i < 16; ++i) dw3[i] = db2[i] = 0.f;

  const int64_t nsteps = (n + 63) / 64;
  for (int64_t step = blockIdx.x; step < nsteps; step += gridDim.x) {
    const int64_t r0 = step * 64 + 16 * w;
    uint32_t h1a[4][4];
    float h2[8][4], m[2];
    mlp_tile_fwd(s, f, r0, n, h1a, h2, m);
    float gr[2];
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      const int64_t row = r0 + g + 8 * hh;
      const float d = row < n ? m[hh] - __ldg(target + row) : 0.0f;
      gr[hh] = d * inv_n;
      if (t == 0) {
        lsum = __fmaf_rn(d, d, lsum);
        db3 += gr[hh];
      }
    }
    // dz2 in C layout, BF16; partial sums of dw3 and db2
    float dz2[8][4];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float gg = gr[e >> 1];
        const float w3v = s.w3[nt * 8 + 2 * t + (e & 1)];
        dz2[nt][e] = h2[nt][e] > 0.f ? bf16r(gg * w3v) : 0.f;
        dw3[nt * 2 + (e & 1)] = __fmaf_rn(h2[nt][e], gg, dw3[nt * 2 + (e & 1)]);
        db2[nt * 2 + (e & 1)] += dz2[nt][e];
      }
    }
    // tiles for the weight gradients
    const int ra = 16 * w + g, rb = ra + 8;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const int c = nt * 8 + 2 * t;
      *reinterpret_cast<uint32_t*>(&T.dz2[ra][c]) = pack_bf16(dz2[nt][0], dz2[nt][1]);
      *reinterpret_cast<uint32_t*>(&T.dz2[rb][c]) = pack_bf16(dz2[nt][2], dz2[nt][3]);
    }
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
      const int c = kc * 16 + 2 * t;
      *reinterpret_cast<uint32_t*>(&T.h1[ra][c]) = h1a[kc][0];
      *reinterpret_cast<uint32_t*>(&T.h1[rb][c]) = h1a[kc][1];
      *reinterpret_cast<uint32_t*>(&T.h1[ra][c + 8]) = h1a[kc][2];
      *reinterpret_cast<uint32_t*>(&T.h1[rb][c + 8]) = h1a[kc][3];
    }
    {
      // inputs 2t, 2t+1 of rows ra, rb; column 8 = 1 and 9..15 = 0 from lanes t = 0..3
      const int64_t rowa = r0 + g, rowb = r0 + g + 8;
      *reinterpret_cast<uint32_t*>(&T.f[ra][2 * t]) =
          pack_bf16(feat(s, f, rowa, n, 2 * t), feat(s, f, rowa, n, 2 * t + 1));
      *reinterpret_cast<uint32_t*>(&T.f[rb][2 * t]) =
          pack_bf16(feat(s, f, rowb, n, 2 * t), feat(s, f, rowb, n, 2 * t + 1));
      const uint32_t ones = t == 0 ? pack_bf16(1.0f, 0.0f) : 0u;
      *reinterpret_cast<uint32_t*>(&T.f[ra][8 + 2 * t]) = ones;
      *reinterpret_cast<uint32_t*>(&T.f[rb][8 + 2 * t]) = ones;
    }
    // dh1 = dz2 W2 (A = dz2 as fragments, B[k = out][n = in] = W2[out][in])
    uint32_t dza[4][4];
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
      dza[kc][0] = pack_bf16(dz2[2 * kc][0], dz2[2 * kc][1]);
      dza[kc][1] = pack_bf16(dz2[2 * kc][2], dz2[2 * kc][3]);
      dza[kc][2] = pack_bf16(dz2[2 * kc + 1][0], dz2[2 * kc + 1][1]);
      dza[kc][3] = pack_bf16(dz2[2 * kc + 1][2], dz2[2 * kc + 1][3]);
    }
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int kc = 0; kc < 4; ++kc)
        mma16816(c, dza[kc],
                 ld2(&s.W2[kc * 16 + 2 * t][nt * 8 + g], &s.W2[kc * 16 + 2 * t + 1][nt * 8 + g]),
                 ld2(&s.W2[kc * 16 + 8 + 2 * t][nt * 8 + g],
                     &s.W2[kc * 16 + 9 + 2 * t][nt * 8 + g]));
      // mask by h1 > 0: h1 of units nt*8 + 2t + {0,1} is in h1a[nt/2][(nt&1)*2 + {0: row g, 1: row g+8}]
      const uint32_t hA = h1a[nt >> 1][(nt & 1) * 2], hB = h1a[nt >> 1][(nt & 1) * 2 + 1];
      const float d0 = lo_f(hA) > 0.f ? c[0] : 0.f, d1 = hi_f(hA) > 0.f ? c[1] : 0.f;
      const float d2 = lo_f(hB) > 0.f ? c[2] : 0.f, d3 = hi_f(hB) > 0.f ? c[3] : 0.f;
      const int cc = nt * 8 + 2 * t;
      *reinterpret_cast<uint32_t*>(&T.dz1[ra][cc]) = pack_bf16(d0, d1);
      *reinterpret_cast<uint32_t*>(&T.dz1[rb][cc]) = pack_bf16(d2, d3);
    }
    __syncthreads();
    // weight gradients of rows (output units) 16w..16w+15 over the 64 samples
    const int u0 = 16 * w + g, u1 = u0 + 8;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
      const int s0 = kk * 16 + 2 * t, s8 = s0 + 8;
      uint32_t a2[4], a1[4];
      a2[0] = ld2(&T.dz2[s0][u0], &T.dz2[s0 + 1][u0]);
      a2[1] = ld2(&T.dz2[s0][u1], &T.dz2[s0 + 1][u1]);
      a2[2] = ld2(&T.dz2[s8][u0], &T.dz2[s8 + 1][u0]);
      a2[3] = ld2(&T.dz2[s8][u1], &T.dz2[s8 + 1][u1]);
      a1[0] = ld2(&T.dz1[s0][u0], &T.dz1[s0 + 1][u0]);
      a1[1] = ld2(&T.dz1[s0][u1], &T.dz1[s0 + 1][u1]);
      a1[2] = ld2(&T.dz1[s8][u0], &T.dz1[s8 + 1][u0]);
      a1[3] = ld2(&T.dz1[s8][u1], &T.dz1[s8 + 1][u1]);
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        const int k = nt * 8 + g;
        mma16816(dW2[nt], a2, ld2(&T.h1[s0][k], &T.h1[s0 + 1][k]),
                 ld2(&T.h1[s8][k], &T.h1[s8 + 1][k]));
      }
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        const int k = nt * 8 + g;
        mma16816(dW1[nt], a1, ld2(&T.f[s0][k], &T.f[s0 + 1][k]),
                 ld2(&T.f[s8][k], &T.f[s8 + 1][k]));
      }
    }
    __syncthreads();
  }

  // ---- write this block's partial gradient ----
  float* P = part + (int64_t)blockIdx.x * (NP + 1);
  const int u0 = 16 * w + g, u1 = u0 + 8;
#pragma unroll
  for (int nt = 0; nt < 8; ++nt) {
    const int k = nt * 8 + 2 * t;
    P[O_W2 + u0 * NH + k] = dW2[nt][0];
    P[O_W2 + u0 * NH + k + 1] = dW2[nt][1];
    P[O_W2 + u1 * NH + k] = dW2[nt][2];
    P[O_W2 + u1 * NH + k + 1] = dW2[nt][3];
  }
  P[O_W1 + u0 * NF + 2 * t] = dW1[0][0];
  P[O_W1 + u0 * NF + 2 * t + 1] = dW1[0][1];
  P[O_W1 + u1 * NF + 2 * t] = dW1[0][2];
  P[O_W1 + u1 * NF + 2 * t + 1] = dW1[0][3];
  if (t == 0) {  // column 8 of the second n-tile: sum of dz1 = db1
    P[O_B1 + u0] = dW1[1][0];
    P[O_B1 + u1] = dW1[1][2];
  }
  // dw3, db2, db3 and the loss: lanes with equal t hold the same columns
#pragma unroll
  for (int i = 0; i < 16; ++i)
#pragma unroll
    for (int msk = 4; msk <= 16; msk <<= 1) {
      dw3[i] += __shfl_xor_sync(0xffffffffu, dw3[i], msk);
      db2[i] += __shfl_xor_sync(0xffffffffu, db2[i], msk);
    }
#pragma unroll
  for (int msk = 1; msk <= 16; msk <<= 1) {
    db3 += __shfl_xor_sync(0xffffffffu, db3, msk);
    lsum += __shfl_xor_sync(0xffffffffu, lsum, msk);
  }
  if (g == 0) {
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        T.red[w][nt * 8 + 2 * t + e] = dw3[nt * 2 + e];
        T.red[w][NH + nt * 8 + 2 * t + e] = db2[nt * 2 + e];
      }
  }
  if (lane == 0) {
    T.red[w][2 * NH] = db3;
    T.red[w][2 * NH + 1] = lsum;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 2 * NH + 2; i += blockDim.x) {
    const float v = ((T.red[0][i] + T.red[1][i]) + T.red[2][i]) + T.red[3][i];
    if (i < NH) P[O_W3 + i] = v;
    else if (i < 2 * NH) P[O_B2 + i - NH] = v;
    else if (i == 2 * NH) P[O_B3] = v;
    else P[NP] = v;  // sum of squared errors
  }
}

__global__ void k_mlp_reduce(const float* __restrict__ part, int nblocks, float* __restrict__ grad,
                             float* __restrict__ loss, int64_t n) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p <= NP; p += gridDim.x * blockDim.x) {
    float v = 0.f;
    for (int b = 0; b < nblocks; ++b) v += part[(int64_t)b * (NP + 1) + p];
    if (p < NP) grad[p] = v;
    else if (loss) *loss = v / (float)n;
  }
}

__global__ void k_adam(float* __restrict__ th, const float* __restrict__ gr, float* __restrict__ mo,
                       float* __restrict__ ve, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < NP; p += gridDim.x * blockDim.x) {
    const float gg = gr[p];
    const float m = b1 * mo[p] + (1.0f - b1) * gg;
    const float v = b2 * ve[p] + (1.0f - b2) * gg * gg;
    mo[p] = m;
    ve[p] = v;
    th[p] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
  }
}

// d_j = exp(clamp(m_q)) / ||A_:,j|| on the attitude + instrumental columns,
// 1 / ||A_:,j|| elsewhere (1 for an empty column).
__global__ void k_learned_scaling(Layout L, const double* __restrict__ colnorm,
                                  const float* __restrict__ m, float clamp,
                                  double* __restrict__ d) {
  const int64_t q0 = L.att_base, q1 = L.att_base + 3 * L.n_knots + L.n_instr;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < L.n_unk;
       j += (int64_t)gridDim.x * blockDim.x) {
    const double c = colnorm[j];
    double mult = 1.0;
    if (j >= q0 && j < q1 && m) {
      const float mq = fminf(fmaxf(m[j - q0], -clamp), clamp);
      mult = exp((double)mq);
    }
    d[j] = c > 0.0 ? mult / c : 1.0;
  }
}

int grid_for(int64_t work, int threads, int cap) {
  const int64_t b = (work + threads - 1) / threads;
  return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace
}  // namespace gsr

using namespace gsr;

extern "C" int64_t gsr_n_learned_cols(const gsr_system* s) {
  return s ? 3 * s->L.n_knots + s->L.n_instr : 0;
}

extern "C" int gsr_column_features(gsr_system* s, float* feats, void* stream) {
  if (!s || !feats) return GSR_E_ARG;
  gsr::DeviceGuard dg(s->device);
  if (!dg.ok) return GSR_E_CUDA;
  if (const int se = gsr::sticky_error(s)) return se;  // an earlier launch failed
  cudaStream_t st = (cudaStream_t)stream;
  const Layout& L = s->L;
  if (!s->instr_count) {
    if (cudaMalloc((void**)&s->instr_count, (L.n_instr > 0 ? L.n_instr : 1) * sizeof(int)) !=
        cudaSuccess) {
      cudaGetLastError();
      return GSR_E_OOM;
    }
    if (cudaMemsetAsync(s->instr_count, 0, L.n_instr * sizeof(int), st) != cudaSuccess)
      return GSR_E_CUDA;
    if (L.n_rows > 0)
      k_instr_count<<<grid_for(L.n_rows, 256, s->num_sms * 8), 256, 0, st>>>(L, s->instr_count);
    if (cudaGetLastError() != cudaSuccess) return GSR_E_CUDA;
  }
  const int64_t nq = 3 * L.n_knots + L.n_instr;
  if (nq > 0)
    k_features<<<grid_for(nq, 256, s->num_sms * 8), 256, 0, st>>>(L, s->colnorm, s->instr_count,
                                                                  feats);
  return cudaGetLastError() == cudaSuccess ? GSR_OK : GSR_E_CUDA;
}

extern "C" int gsr_feature_moments(const float* feats, int64_t n, double* acc, void* stream) {
  if ((!feats && n > 0) || !acc || n < 0) return GSR_E_ARG;
  if (n == 0) return GSR_OK;
  k_feature_moments<<<grid_for(n, 256, 148 * 4), 256, 0, (cudaStream_t)stream>>>(feats, n, acc);
  return cudaGetLastError() == cudaSuccess ? GSR_OK : GSR_E_CUDA;
}

// norm[0..7] = mean, norm[8..15] = 1/std (1 for a constant feature) from the
// moments acc (sums and sums of squares over n rows).
__global__ void k_feature_norm(const double* __restrict__ acc, int64_t n, float* __restrict__ norm) {
  const int k = threadIdx.x;
  if (k >= NF) return;
  const double mean = acc[k] / (double)n;
  const double var = fmax(acc[NF + k] / (double)n - mean * mean, 0.0);
  norm[k] = (float)mean;
  norm[NF + k] = var > 1e-12 ? (float)(1.0 / sqrt(var)) : 1.0f;
}

extern "C" int gsr_feature_standardisation(const double* acc, int64_t n, float* norm,
                                           void* stream) {
  if (!acc || !norm || n <= 0) return GSR_E_ARG;
  k_feature_norm<<<1, 32, 0, (cudaStream_t)stream>>>(acc, n, norm);
  return cudaGetLastError() == cudaSuccess ? GSR_OK : GSR_E_CUDA;
}

extern "C" int gsr_mlp_forward(const float* feats, int64_t n, const float* norm,
                               const float* theta, float* m, void* stream) {
  if (n < 0 || (n > 0 && (!feats || !norm || !theta || !m))) return GSR_E_ARG;
  if (n == 0) return GSR_OK;
  const int64_t warps = (n + 15) / 16;
  k_mlp_fwd<<<grid_for(warps * 32, 128, 148 * 16), 128, 0, (cudaStream_t)stream>>>(feats, n, norm,
                                                                                  theta, m);
  return cudaGetLastError() == cudaSuccess ? GSR_OK : GSR_E_CUDA;
}

extern "C" int gsr_mlp_grad(const float* feats, const float* target, int64_t n, const float* norm,
                            const float* theta, float* work, float* grad, float* loss,
                            void* stream) {
  if (n <= 0 || !feats || !target || !norm || !theta || !work || !grad) return GSR_E_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int blocks = grid_for((n + 63) / 64, 1, GSR_MLP_GRID);
  k_mlp_grad<<<blocks, 128, 0, st>>>(feats, target, n, norm, theta, work);
  if (cudaGetLastError() != cudaSuccess) return GSR_E_CUDA;
  k_mlp_reduce<<<(NP + 1 + 255) / 256, 256, 0, st>>>(work, blocks, grad, loss, n);
  return cudaGetLastError() == cudaSuccess ? GSR_OK : GSR_E_CUDA;
}

extern "C" int gsr_mlp_adam(float* theta, const float* grad, float* mom, float* vel, int64_t step,
                            float lr, float beta1, float beta2, float eps, void* stream) {
  if (!theta || !grad || !mom || !vel || step < 1 || !(lr > 0.0f) || !(beta1 >= 0.0f) ||
      !(beta1 < 1.0f) || !(beta2 >= 0.0f) || !(beta2 < 1.0f) || !(eps > 0.0f))
    return GSR_E_ARG;
  const float c1 = (float)(1.0 - std::pow((double)beta1, (double)step));
  const float c2 = (float)(1.0 - std::pow((double)beta2, (double)step));
  k_adam<<<(NP + 255) / 256, 256, 0, (cudaStream_t)stream>>>(theta, grad, mom, vel, lr, beta1,
                                                             beta2, eps, c1, c2);
  return cudaGetLastError() == cudaSuccess ? GSR_OK : GSR_E_CUDA;
}

extern "C" int gsr_learned_scaling(gsr_system* s, const float* m, float clamp, double* d,
                                   void* stream) {
  if (!s || !d || !(clamp >= 0.0f)) return GSR_E_ARG;
  gsr::DeviceGuard dg(s->device);
  if (!dg.ok) return GSR_E_CUDA;
  if (const int se = gsr::sticky_error(s)) return se;  // an earlier launch failed
  if (s->L.n_unk > 0)
    k_learned_scaling<<<grid_for(s->L.n_unk, 256, s->num_sms * 8), 256, 0,
                        (cudaStream_t)stream>>>(s->L, s->colnorm, m, clamp, d);
  return cudaGetLastError() == cudaSuccess ? GSR_OK : GSR_E_CUDA;
}
