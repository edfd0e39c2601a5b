// gsr_create / gsr_destroy and the plain aprod entry points.
//
// gsr_create validates the packed rows of Sec. 2 on the host (one pass,
// several threads), builds the index structures (the stable counting sort of
// rows by attitude start knot, the attitude warp ranges, and the instrumental
// entries of every tile ordered into rounds of distinct bins), uploads the
// values in chunks and lays them out on the device as 64-row records of float
// pairs (plus an optional FP32 copy) and a knot-ordered copy of the attitude
// block. The column norms ||A_:,j|| (used by the column-scaling preconditioner,
// Sec. 2 solver step 2) are computed on the device.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

#include "gsr_system.cuh"

namespace gsr {

namespace {

constexpr int64_t CHUNK_ROWS = 1 << 22;  // rows per upload chunk (768 MB of values)

template <bool F32>
__device__ __forceinline__ void put_indices(unsigned char* rec, int l, int c, int star, int s,
                                            int p, const int32_t* ins) {
  using R = Rec<F32>;
  reinterpret_cast<int32_t*>(rec + R::STAR)[2 * l + c] = star;
  reinterpret_cast<int32_t*>(rec + R::ATT_S)[2 * l + c] = s;
  reinterpret_cast<int32_t*>(rec + R::POS)[2 * l + c] = p;
  for (int k = 0; k < 6; ++k)
    reinterpret_cast<uint16_t*>(rec + R::INSTR_I + k * 128)[2 * l + c] = (uint16_t)ins[k];
}

// Lay out rows [r0, r0+n) of the raw upload into the records and the
// knot-ordered attitude copy (row r at L.gpos[r]; the FP32 records carry that
// position, the float-pair ones L.pos[r]), each value rescaled to 2^(e_i + g_j) A_ij when
// the system has exponents; accumulate the squared column norms of 2^g_j A_ij.
__global__ void k_layout(Layout L, unsigned char* __restrict__ rec_ff,
                         unsigned char* __restrict__ rec_f32, float2* __restrict__ att_ff,
                         float* __restrict__ att_f32, const double* __restrict__ raw,
                         const int32_t* __restrict__ raw_instr, const int32_t* __restrict__ star,
                         const int32_t* __restrict__ s_knot, double* __restrict__ c2, int64_t r0,
                         int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = r0 + i;
    const int64_t rec = r / REC_ROWS;
    const int l = (int)((r % REC_ROWS) >> 1), c = (int)(r & 1);
    const int st = star[r], sk = s_knot[r], p = L.pos[r], gp = L.gpos[r];
    const int er = L.row_exp ? (int)L.row_exp[r] : 0;
    unsigned char* rf = rec_ff + rec * Rec<false>::BYTES;
    unsigned char* r32 = rec_f32 ? rec_f32 + rec * Rec<true>::BYTES : nullptr;
    put_indices<false>(rf, l, c, st, sk, p, raw_instr + i * 6);
    if (r32) put_indices<true>(r32, l, c, st, sk, gp, raw_instr + i * 6);
    for (int t = 0; t < NSLOT; ++t) {
      double v = raw[i * NSLOT + t];
      int64_t col = -1;
      if (t < 5) {
        col = 5 * (int64_t)st + t;
      } else if (t < 17) {
        const int a = (t - 5) >> 2, jj = (t - 5) & 3;
        col = L.att_base + a * L.n_knots + sk + jj;
      } else if (t < 23) {
        col = L.instr_base + raw_instr[i * 6 + (t - 17)];
      } else if (L.n_glob == 1) {
        col = L.glob_col;
      } else {
        v = 0.0;
      }
      const int ec = (col >= 0 && L.col_exp) ? (int)L.col_exp[col] : 0;
      const double vs = (er + ec) ? ldexp(v, er + ec) : v;  // exact power-of-two rescaling
      const float h = __double2float_rn(vs);
      const float lo = __double2float_rn(vs - (double)h);
      float* pf = reinterpret_cast<float*>(rf + slot_offset<false>(t) + l * 16);
      pf[2 * c] = h;
      pf[2 * c + 1] = lo;
      if (r32) reinterpret_cast<float*>(r32 + slot_offset<true>(t) + l * 8)[c] = h;
      if (t >= 5 && t < 17) {
        att_ff[(int64_t)(t - 5) * L.n_rows + gp] = make_float2(h, lo);
        if (att_f32) att_f32[(int64_t)(t - 5) * L.n_rows + gp] = h;
      }
      if (col < 0) continue;
      const double vc = ec ? ldexp(v, ec) : v;
      atomicAdd(c2 + col, vc * vc);
    }
  }
}

// Padding rows of the last record: the last real star, knot 0, zero values.
__global__ void k_pad_records(Layout L, unsigned char* rec_ff, unsigned char* rec_f32, int star) {
  const int64_t r = L.n_rows + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= L.n_recs * REC_ROWS) return;
  const int64_t rec = r / REC_ROWS;
  const int l = (int)((r % REC_ROWS) >> 1), c = (int)(r & 1);
  const int32_t zeros[6] = {0, 1, 2, 3, 4, 5};
  put_indices<false>(rec_ff + rec * Rec<false>::BYTES, l, c, star, 0, 0, zeros);
  if (rec_f32) put_indices<true>(rec_f32 + rec * Rec<true>::BYTES, l, c, star, 0, 0, zeros);
}

// ||A_:,j|| = 2^-g_j ||2^g_j A_:,j||.
__global__ void k_sqrt(double* __restrict__ a, const int16_t* __restrict__ cexp, int64_t n) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x) {
    const double c = sqrt(a[j]);
    a[j] = cexp ? ldexp(c, -(int)cexp[j]) : c;
  }
}

template <typename T>
int dalloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return e == cudaErrorMemoryAllocation ? GSR_E_OOM : GSR_E_CUDA;
  }
  return GSR_OK;
}

void free_system(gsr_system* s) {
  if (!s) return;
  destroy_batch(s);
  free_constraints(s);
  delete[] s->colnorm_obs;
  void* ptrs[] = {s->rec_ff, s->rec_f32, s->pos, s->att_knot_ff, s->att_knot_f32, s->knot_start,
                  s->kb_start, s->gpos, s->att_warp_knot, s->iseg, s->ient_ff, s->ient_f32,
                  s->ient_key, s->colnorm, s->u, s->u_knot, s->v, s->w, s->xz, s->z,
                  s->dscale, s->dscale_ff, s->v_ff, s->mx_x1, s->mx_d, s->mx_r, s->scal, s->S.red,
                  s->S.count, s->S.x_ff, s->S.x3,
                  s->S.y_ff, s->S.y_knot, s->instr_count, s->row_exp, s->col_exp,
                  s->S.guard, s->S.iexp, s->S.zx};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (s->host_scal) cudaFreeHost(s->host_scal);
  if (s->err_host) cudaFreeHost(s->err_host);
  if (s->side) cudaStreamDestroy(s->side);
  if (s->ev_fork) cudaEventDestroy(s->ev_fork);
  if (s->ev_join) cudaEventDestroy(s->ev_join);
  delete s;
}

// Host validation of rows [a, b). Returns GSR_OK or the first error kind found.
int validate_rows(const gsr_dims& d, const double* vals, const int64_t* astro_off,
                  const int64_t* att_off, const int32_t* instr, int64_t a, int64_t b,
                  int32_t* star, int32_t* s_knot) {
  const int64_t K = d.n_knots, astro_end = 5 * d.n_stars;
  for (int64_t i = a; i < b; ++i) {
    const int64_t ao = astro_off[i];
    if (ao < 0 || ao >= astro_end || ao % 5 != 0) return GSR_E_INDEX;
    if (i > 0 && astro_off[i - 1] > ao) return GSR_E_UNSORTED;
    const int64_t s = att_off[i] - astro_end;
    if (s < 0 || s > K - 4) return GSR_E_INDEX;
    const int32_t* ir = instr + i * 6;
    for (int k = 0; k < 6; ++k) {
      if (ir[k] < 0 || ir[k] >= d.n_instr) return GSR_E_INDEX;
      for (int m = 0; m < k; ++m)
        if (ir[m] == ir[k]) return GSR_E_INDEX;
    }
    const double* vr = vals + i * NSLOT;
    const int nv = d.n_glob == 1 ? NSLOT : NSLOT - 1;
    for (int t = 0; t < nv; ++t)
      if (!std::isfinite(vr[t])) return GSR_E_NONFINITE;
    star[i] = (int32_t)(ao / 5);
    s_knot[i] = (int32_t)s;
  }
  return GSR_OK;
}

template <typename F>
void parallel_for(int64_t n, unsigned nt, F f) {
  if (nt <= 1 || n < 2) {
    for (int64_t i = 0; i < n; ++i) f(i, 0u);
    return;
  }
  std::vector<std::thread> th;
  for (unsigned k = 0; k < nt; ++k)
    th.emplace_back([&, k] {
      for (int64_t i = k; i < n; i += nt) f(i, k);
    });
  for (auto& t : th) t.join();
}

// ---------------------------------------------------------------------------
// Exact power-of-two rescaling of the coefficients (host, at creation). The
// float-pair kernels carry FP32's exponent range; FP64 input may span far more.
// Scaling row i by 2^e_i and column j by 2^g_j is exact and is undone exactly
// at the edges (vector conversions, FP64 outputs, the column preconditioner),
// so it changes no result. Chosen in this order:
//   1. every nonzero |A_ij| in [2^-40, 2^40): no rescaling at all;
//   2. column exponents only (column maxima to [1, 2)), if that leaves every
//      coefficient >= 2^-100;
//   3. otherwise row and column exponents that fit the binary exponents of the
//      coefficients in the least-squares sense (alternately subtract each
//      row's and each column's mean exponent, rounded, until nothing moves;
//      for A = R A0 C this recovers R and C up to the spread of A0), then
//      column maxima to [1, 2).
// A coefficient still below 2^-100 of the largest of its column after that
// has a spread no diagonal scaling removes (a 2 x 2 minor decides it):
// GSR_E_UNSUPPORTED. Below 2^-40 the system is "wide": its direct products run
// the FP64 kernels.
// ---------------------------------------------------------------------------
struct Rescale {
  std::vector<int16_t> row, col;  // empty: all exponents 0
  bool row_scaled = false, wide = false;
};

constexpr int NO_EXP = INT32_MIN / 2;

// Column of slot t of row i (or -1 for the absent global slot).
inline int64_t slot_col(const gsr_dims& d, const int32_t* star, const int32_t* s_knot,
                        const int32_t* instr, int64_t i, int t) {
  const int64_t att_base = 5 * d.n_stars, instr_base = att_base + 3 * d.n_knots;
  if (t < 5) return 5 * (int64_t)star[i] + t;
  if (t < 17) return att_base + ((t - 5) >> 2) * d.n_knots + s_knot[i] + ((t - 5) & 3);
  if (t < 23) return instr_base + instr[i * 6 + (t - 17)];
  return d.n_glob == 1 ? instr_base + d.n_instr : -1;
}

// Row chunks for nt threads that never split a star (the astrometric columns
// of a star are then touched by one thread only).
std::vector<int64_t> star_chunks(const int32_t* star, int64_t n, unsigned nt) {
  std::vector<int64_t> b(1, 0);
  for (unsigned k = 1; k < nt; ++k) {
    int64_t r = std::max(b.back(), (n * (int64_t)k) / nt);
    while (r > 0 && r < n && star[r] == star[r - 1]) ++r;
    b.push_back(std::min(r, n));
  }
  b.push_back(n);
  return b;
}

// Statistics of x_ij = ilogb|A_ij| + e_i + g_j over the nonzero coefficients:
// per row the sum and count (rsum, rcnt), per column the largest (cmax) or the
// sum and count (csum, ccnt); returns the smallest x_ij. Null outputs are
// skipped.
struct ExpStats {
  std::vector<int64_t> rsum, csum;
  std::vector<int32_t> rcnt, ccnt, cmax;
};
int scan_exponents(const gsr_dims& d, const double* vals, const int32_t* star,
                   const int32_t* s_knot, const int32_t* instr, const std::vector<int>& e,
                   const std::vector<int>& g, unsigned nt, bool rows, bool col_sums,
                   bool col_max, ExpStats& out) {
  const int64_t n = d.n_rows, n_unk = (int64_t)g.size();
  const int64_t sh0 = 5 * d.n_stars, n_sh = n_unk - sh0;  // columns shared between stars
  const std::vector<int64_t> ch = star_chunks(star, n, nt);
  const unsigned nc = (unsigned)ch.size() - 1;
  if (rows) {
    out.rsum.assign(n, 0);
    out.rcnt.assign(n, 0);
  }
  if (col_sums) {
    out.csum.assign(n_unk, 0);
    out.ccnt.assign(n_unk, 0);
  }
  if (col_max) out.cmax.assign(n_unk, NO_EXP);
  std::vector<std::vector<int64_t>> lsum(nc);
  std::vector<std::vector<int32_t>> lcnt(nc), lmax(nc);
  std::vector<int> mins(nc, INT32_MAX);
  std::vector<std::thread> th;
  for (unsigned k = 0; k < nc; ++k)
    th.emplace_back([&, k] {
      if (col_sums) {
        lsum[k].assign(n_sh, 0);
        lcnt[k].assign(n_sh, 0);
      }
      if (col_max) lmax[k].assign(n_sh, NO_EXP);
      int mn = INT32_MAX;
      for (int64_t i = ch[k]; i < ch[k + 1]; ++i) {
        int64_t rs = 0;
        int32_t rc = 0;
        for (int t = 0; t < NSLOT; ++t) {
          const double v = vals[i * NSLOT + t];
          if (v == 0.0) continue;
          const int64_t c = slot_col(d, star, s_knot, instr, i, t);
          if (c < 0) continue;
          const int x = std::ilogb(v) + e[i] + g[c];
          mn = std::min(mn, x);
          rs += x;
          ++rc;
          const bool own = c < sh0;  // an astrometric column: this thread's alone
          if (col_sums) {
            (own ? out.csum[c] : lsum[k][c - sh0]) += x;
            ++(own ? out.ccnt[c] : lcnt[k][c - sh0]);
          }
          if (col_max) {
            int32_t& m = own ? out.cmax[c] : lmax[k][c - sh0];
            m = std::max(m, (int32_t)x);
          }
        }
        if (rows) {
          out.rsum[i] = rs;
          out.rcnt[i] = rc;
        }
      }
      mins[k] = mn;
    });
  for (auto& t : th) t.join();
  for (unsigned k = 0; k < nc; ++k)
    for (int64_t c = 0; c < n_sh; ++c) {
      if (col_sums) {
        out.csum[sh0 + c] += lsum[k][c];
        out.ccnt[sh0 + c] += lcnt[k][c];
      }
      if (col_max) out.cmax[sh0 + c] = std::max(out.cmax[sh0 + c], lmax[k][c]);
    }
  int mn = INT32_MAX;
  for (int m : mins) mn = std::min(mn, m);
  return mn;
}

// round(sum / count) for count > 0
inline int mean_exp(int64_t sum, int32_t cnt) {
  return (int)std::llround((double)sum / (double)cnt);
}

int choose_rescaling(const gsr_dims& d, const double* vals, const int32_t* star,
                     const int32_t* s_knot, const int32_t* instr, unsigned nt, Rescale& out) {
  const int64_t n = d.n_rows;
  const int64_t n_unk = 5 * d.n_stars + 3 * d.n_knots + d.n_instr + d.n_glob;
  out = Rescale();
  if (n == 0) return GSR_OK;
  std::vector<int> e(n, 0), g(n_unk, 0);
  ExpStats st;
  const int mn0 = scan_exponents(d, vals, star, s_knot, instr, e, g, nt, false, false, true, st);
  int mx0 = NO_EXP;
  for (int v : st.cmax) mx0 = std::max(mx0, v);
  if (mx0 == NO_EXP || (mn0 >= MAT_BAND_LO && mx0 < MAT_BAND_HI)) return GSR_OK;  // step 1
  // step 2: column maxima to [1, 2)
  for (int64_t c = 0; c < n_unk; ++c) g[c] = st.cmax[c] == NO_EXP ? 0 : -st.cmax[c];
  int mn = scan_exponents(d, vals, star, s_knot, instr, e, g, nt, false, false, false, st);
  if (mn < MAT_WIDE_LO) {
    // step 3: least-squares fit of row and column exponents
    std::fill(g.begin(), g.end(), 0);
    for (int it = 0; it < 64; ++it) {
      bool moved = false;
      scan_exponents(d, vals, star, s_knot, instr, e, g, nt, true, false, false, st);
      for (int64_t i = 0; i < n; ++i)
        if (st.rcnt[i] > 0) {
          const int m = mean_exp(st.rsum[i], st.rcnt[i]);
          if (m != 0) {
            e[i] -= m;
            moved = true;
          }
        }
      scan_exponents(d, vals, star, s_knot, instr, e, g, nt, false, true, false, st);
      for (int64_t c = 0; c < n_unk; ++c)
        if (st.ccnt[c] > 0) {
          const int m = mean_exp(st.csum[c], st.ccnt[c]);
          if (m != 0) {
            g[c] -= m;
            moved = true;
          }
        }
      if (!moved) break;
    }
    // a common row exponent is a column one
    const int e0 = e[0];
    bool same = true;
    for (int64_t i = 1; i < n && same; ++i) same = e[i] == e0;
    if (same) {
      std::fill(e.begin(), e.end(), 0);
      for (int& v : g) v += e0;
    }
    scan_exponents(d, vals, star, s_knot, instr, e, g, nt, false, false, true, st);
    for (int64_t c = 0; c < n_unk; ++c)
      if (st.cmax[c] != NO_EXP) g[c] -= st.cmax[c];
    mn = scan_exponents(d, vals, star, s_knot, instr, e, g, nt, false, false, false, st);
    if (mn < MAT_WIDE_LO) return GSR_E_UNSUPPORTED;
    out.row_scaled = !same;
  }
  for (int v : e)
    if (v < INT16_MIN || v > INT16_MAX) return GSR_E_UNSUPPORTED;
  for (int v : g)
    if (v < INT16_MIN || v > INT16_MAX) return GSR_E_UNSUPPORTED;
  out.wide = mn < MAT_BAND_LO;
  if (out.row_scaled) out.row.assign(e.begin(), e.end());
  out.col.assign(g.begin(), g.end());
  return GSR_OK;
}

// Instrumental entries of every tile of ct rows, split by column group (G
// groups of bpg consecutive columns), each (tile, group) segment ordered into
// rounds in which every column occurs at most once (round = earlier
// occurrences of the column in the tile) and by column inside a round.
// Segments are stored tile-major, each starting at a multiple of 4 entries;
// seg[c] = (first entry, entries) of segment c (the padding after a segment
// belongs to none).
struct InstrRounds {
  std::vector<longlong2> seg;
  std::vector<uint32_t> key;
  std::vector<float2> vff;
  std::vector<float> vf32;
  int64_t max_ent = 0;
};

void build_instr_rounds(const gsr_dims& d, const double* vals, const int32_t* instr, int ct,
                        int G, int bpg, bool want_f32, unsigned nt, const Rescale& rs,
                        InstrRounds& out) {
  const int64_t instr_base = 5 * d.n_stars + 3 * d.n_knots;
  const int64_t n = d.n_rows;
  const int64_t n_ct = (n + ct - 1) / ct;
  const int64_t n_seg = n_ct * G;
  std::vector<int64_t> seg_n(n_seg, 0);
  std::vector<std::vector<int32_t>> occ(nt, std::vector<int32_t>(d.n_instr, 0));
  parallel_for(n_ct, nt, [&](int64_t t, unsigned w) {
    auto& o = occ[w];
    const int64_t a = t * ct, b = std::min<int64_t>(n, a + ct);
    for (int64_t i = a; i < b; ++i)
      for (int k = 0; k < 6; ++k) ++seg_n[t * G + instr[i * 6 + k] / bpg];
  });
  std::vector<int64_t> seg_start(n_seg + 1, 0);
  out.seg.resize(n_seg);
  out.max_ent = 0;
  for (int64_t c = 0; c < n_seg; ++c) {
    seg_start[c + 1] = (seg_start[c] + seg_n[c] + 3) & ~3LL;  // next segment 16-B aligned
    out.seg[c] = make_longlong2(seg_start[c], seg_n[c]);
    out.max_ent = std::max(out.max_ent, seg_n[c]);
  }
  const int64_t n_ent = seg_start[n_seg];
  out.key.assign(n_ent + 4, 0u);  // +4: TMA copies are rounded up to 16 bytes
  out.vff.assign(n_ent + 4, make_float2(0.f, 0.f));
  if (want_f32) out.vf32.assign(n_ent + 4, 0.f);
  parallel_for(n_ct, nt, [&](int64_t t, unsigned w) {
    auto& o = occ[w];
    const int64_t a = t * ct, b = std::min<int64_t>(n, a + ct);
    std::vector<uint64_t> order;
    order.reserve(6 * (b - a));
    for (int64_t i = a; i < b; ++i)
      for (int k = 0; k < 6; ++k) {
        const int bin = instr[i * 6 + k];
        const uint64_t g = (uint64_t)(bin / bpg);
        const uint64_t rnd = (uint64_t)o[bin]++;
        order.push_back((g << 58) | (rnd << 40) | ((uint64_t)bin << 24) |
                        ((uint64_t)(i - a) << 3) | (uint64_t)k);
      }
    for (int64_t i = a; i < b; ++i)
      for (int k = 0; k < 6; ++k) o[instr[i * 6 + k]] = 0;
    std::sort(order.begin(), order.end());
    int64_t cur_g = -1, e = 0;
    for (uint64_t v : order) {
      const int64_t g = (int64_t)(v >> 58);
      const uint32_t bin = (uint32_t)((v >> 24) & 0xffff);
      const int64_t row = (int64_t)((v >> 3) & 0x1fffff);
      const int k = (int)(v & 7);
      if (g != cur_g) {
        e = seg_start[t * G + g];
        cur_g = g;
      }
      out.key[e] = ((uint32_t)row << INSTR_BIN_BITS) | bin;
      double x = vals[(a + row) * NSLOT + 17 + k];
      const int ex = (rs.row.empty() ? 0 : rs.row[a + row]) +
                     (rs.col.empty() ? 0 : rs.col[instr_base + bin]);
      if (ex) x = std::ldexp(x, ex);
      const float h = (float)x;
      out.vff[e] = make_float2(h, (float)(x - (double)h));
      if (want_f32) out.vf32[e] = h;
      ++e;
    }
  });
}

// Entries a (tile, group) segment is sized for before the exact count is known:
// all 6 ct with one group, else the mean plus six standard deviations.
int64_t est_seg_entries(int ct, int G) {
  if (G == 1) return 6LL * ct;
  const double m = 6.0 * ct / G;
  return (int64_t)(m + 6.0 * std::sqrt(m)) + 8;
}

}  // namespace

int build_system(const gsr_dims* dims, const double* vals, const int64_t* astro_off,
                 const int64_t* att_off, const int32_t* instr, int device, cudaStream_t st,
                 gsr_system** out) {
  const gsr_dims d = *dims;
  if (d.n_rows < 0 || d.n_stars < 0 || d.n_knots < 4 || d.n_instr < 6 ||
      (d.n_glob != 0 && d.n_glob != 1) ||
      (d.storage != GSR_STORE_F64 && d.storage != GSR_STORE_F32_PLUS_F64))
    return GSR_E_ARG;
  if (d.n_rows > 0 && (!vals || !astro_off || !att_off || !instr || d.n_stars < 1))
    return GSR_E_ARG;
  const int64_t n_unk = 5 * d.n_stars + 3 * d.n_knots + d.n_instr + d.n_glob;
  if (d.n_rows >= (int64_t(1) << 31) || n_unk >= (int64_t(1) << 31) ||
      d.n_instr > MAX_HIST_INSTR)
    return GSR_E_UNSUPPORTED;
  const bool want_f32 = d.storage == GSR_STORE_F32_PLUS_F64;

  const int64_t n = d.n_rows;
  const int64_t n_recs = (n + REC_ROWS - 1) / REC_ROWS;
  unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  if (n < 100000) nt = 1;

  // ---- host validation and per-row indices (multi-threaded) ----
  std::vector<int32_t> star(std::max<int64_t>(n, 1)), s_knot(std::max<int64_t>(n, 1)),
      pos(std::max<int64_t>(n, 1));
  {
    std::vector<int> rc(nt, GSR_OK);
    std::vector<std::thread> th;
    const int64_t per = (n + nt - 1) / nt;
    for (unsigned k = 0; k < nt; ++k) {
      const int64_t a = std::min<int64_t>(n, k * per), b = std::min<int64_t>(n, a + per);
      th.emplace_back([&, k, a, b] {
        rc[k] = validate_rows(d, vals, astro_off, att_off, instr, a, b, star.data(),
                              s_knot.data());
      });
    }
    for (auto& t : th) t.join();
    for (int r : rc)
      if (r != GSR_OK) return r;
  }
  // ---- exact power-of-two rescaling into the float-pair range ----
  Rescale rs;
  {
    const int r = choose_rescaling(d, vals, star.data(), s_knot.data(), instr, nt, rs);
    if (r != GSR_OK) return r;
  }
  // ---- knot order: counting sort of rows by start knot (stable), and the
  // blocked order of the float-pair copy of u ----
  const int64_t n_buckets = d.n_knots - 3;
  std::vector<int64_t> knot_start(n_buckets + 1, 0);  // first position of start knot s
  for (int64_t r = 0; r < n; ++r) knot_start[s_knot[r] + 1]++;
  for (int64_t b = 0; b < n_buckets; ++b) knot_start[b + 1] += knot_start[b];
  std::vector<int32_t> gpos(n);  // position of each row in the knot order
  {
    std::vector<int64_t> next(knot_start.begin(), knot_start.end() - 1);
    for (int64_t r = 0; r < n; ++r) gpos[r] = (int32_t)(next[s_knot[r]]++);
  }
  // blocked copy of u (see KBLK_MAX): n_kblk blocks of kblk_rows rows
  int64_t n_kblk = std::min<int64_t>(KBLK_MAX, n / (KBLK_MIN_PER_KNOT *
                                                    std::max<int64_t>(1, n_buckets)));
  int64_t kblk_rows = n;
  if (n_kblk >= 2) {
    kblk_rows = ((n + n_kblk - 1) / n_kblk + REC_ROWS - 1) / REC_ROWS * REC_ROWS;
    n_kblk = (n + kblk_rows - 1) / kblk_rows;
  }
  if (n_kblk < 2 || kblk_rows > KBLK_MAX_ROWS) {
    n_kblk = 1;
    kblk_rows = n;
  }
  const int64_t kb_w = n_buckets + 1;
  std::vector<int32_t> kb_start;
  if (n_kblk > 1) {
    kb_start.assign((size_t)n_kblk * kb_w, 0);
    for (int64_t b = 0; b < n_kblk; ++b) {
      const int64_t r0 = b * kblk_rows, r1 = std::min<int64_t>(n, r0 + kblk_rows);
      int32_t* ks = kb_start.data() + b * kb_w;
      for (int64_t r = r0; r < r1; ++r) ks[s_knot[r] + 1]++;
      ks[0] = (int32_t)r0;
      for (int64_t k = 0; k < n_buckets; ++k) ks[k + 1] += ks[k];
      std::vector<int32_t> next(ks, ks + n_buckets);
      for (int64_t r = r0; r < r1; ++r) pos[r] = next[s_knot[r]]++;
    }
  } else {
    std::copy(gpos.begin(), gpos.end(), pos.begin());
  }
  // ---- instrumental tiles and column groups ----
  // Larger tiles mean fewer tile switches per entry. The columns are split
  // into the fewest groups (each block holds one group's histogram) that still
  // allow tiles of at least 1024 rows; then the largest tile wins, and between
  // equal tiles two single-buffered 256-thread blocks per SM (one block's
  // copy waits overlap the other's work) beat one double-buffered
  // 512-thread block. The sizes are checked against the exact segment counts.
  InstrRounds ir;
  int ct = 0, G = 1, bpg = (int)d.n_instr, ct_bufs = 2, ct_per_sm = 1;
  for (int g = 1; g <= 4; ++g) {
    const int b = (int)((d.n_instr + g - 1) / g);
    int c2 = 0, c1 = 0;
    for (int c = CT_ROWS_MAX; c >= 256 && c2 == 0; c >>= 1)
      if (instr_smem_bytes(c, est_seg_entries(c, g), b, false, 1) <= INSTR_SMEM_HALF) c2 = c;
    for (int c = CT_ROWS_MAX; c >= REC_ROWS && c1 == 0; c >>= 1)
      if (instr_smem_bytes(c, est_seg_entries(c, g), b, false, 2) <= INSTR_SMEM_BUDGET) c1 = c;
    if (c1 == 0 && c2 == 0) continue;
    const bool two = c2 > 0 && c2 >= c1;
    ct = two ? c2 : c1;
    G = g;
    bpg = b;
    ct_bufs = two ? 1 : 2;
    ct_per_sm = two ? 2 : 1;
    if (ct >= 1024) break;
  }
  if (ct == 0) return GSR_E_UNSUPPORTED;
  for (;;) {
    build_instr_rounds(d, vals, instr, ct, G, bpg, want_f32, nt, rs, ir);
    const int64_t lim = ct_per_sm == 2 ? INSTR_SMEM_HALF : INSTR_SMEM_BUDGET;
    if (instr_smem_bytes(ct, ir.max_ent, bpg, false, ct_bufs) <= lim || ct <= REC_ROWS) break;
    ct >>= 1;  // an unusually full segment: retry with shorter tiles
  }
  if (instr_smem_bytes(ct, ir.max_ent, bpg, false, ct_bufs) >
      (ct_per_sm == 2 ? INSTR_SMEM_HALF : INSTR_SMEM_BUDGET))
    return GSR_E_UNSUPPORTED;

  // host validation is done; everything below needs the device
  if (cudaSetDevice(device) != cudaSuccess) return GSR_E_CUDA;
  gsr_system* sys = new (std::nothrow) gsr_system();
  if (!sys) return GSR_E_OOM;
  std::memset(sys, 0, sizeof(*sys));
  sys->device = device;
  sys->dims = d;
  sys->row_scaled = rs.row_scaled;
  sys->wide = rs.wide;
  cudaDeviceGetAttribute(&sys->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (sys->num_sms <= 0) sys->num_sms = NUM_SMS_B300;

  Layout& L = sys->L;
  L.n_rows = n;
  L.n_stars = d.n_stars;
  L.n_knots = d.n_knots;
  L.n_instr = d.n_instr;
  L.n_glob = d.n_glob;
  L.n_unk = n_unk;
  L.n_recs = n_recs;
  L.att_base = 5 * d.n_stars;
  L.instr_base = L.att_base + 3 * d.n_knots;
  L.glob_col = L.instr_base + d.n_instr;
  L.ct_rows = ct;
  L.n_bgroups = G;
  L.bgroup_bins = bpg;
  L.ct_max_ent = (int32_t)ir.max_ent;
  L.ct_bufs = ct_bufs;
  L.ct_per_sm = ct_per_sm;
  L.n_ctiles = (int64_t)ir.seg.size() / G;

  L.n_att_warps = sys->num_sms * 8;  // one 8-warp block per SM (the kernel holds ~180 registers)
  std::vector<int32_t> att_warp_knot(L.n_att_warps + 1);
  {
    int64_t b = 0;
    att_warp_knot[0] = 0;
    for (int w = 1; w < L.n_att_warps; ++w) {
      const int64_t target = (n * (int64_t)w) / L.n_att_warps;
      while (b < n_buckets && knot_start[b + 1] <= target) ++b;
      att_warp_knot[w] = (int32_t)std::max<int64_t>(b, att_warp_knot[w - 1]);
    }
    att_warp_knot[L.n_att_warps] = (int32_t)n_buckets;
  }

  // ---- device allocations ----
  const size_t n_ent = ir.key.size();
  int rc = GSR_OK;
  auto A = [&](int r) {
    if (rc == GSR_OK) rc = r;
  };
  A(dalloc(&sys->rec_ff, (size_t)n_recs * Rec<false>::BYTES));
  if (want_f32) A(dalloc(&sys->rec_f32, (size_t)n_recs * Rec<true>::BYTES));
  A(dalloc(&sys->pos, (size_t)n));
  A(dalloc(&sys->att_knot_ff, (size_t)n * 12));
  if (want_f32) A(dalloc(&sys->att_knot_f32, (size_t)n * 12));
  A(dalloc(&sys->knot_start, (size_t)n_buckets + 1));
  if (n_kblk > 1) {
    A(dalloc(&sys->kb_start, kb_start.size()));
    A(dalloc(&sys->gpos, (size_t)n));
  }
  A(dalloc(&sys->att_warp_knot, (size_t)L.n_att_warps + 1));
  A(dalloc(&sys->iseg, ir.seg.size()));
  A(dalloc(&sys->ient_key, n_ent));
  A(dalloc(&sys->ient_ff, n_ent));
  if (want_f32) A(dalloc(&sys->ient_f32, n_ent));
  if (rc == GSR_OK) {
    if (cudaHostAlloc(reinterpret_cast<void**>(&sys->err_host), sizeof(int),
                      cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer(reinterpret_cast<void**>(&sys->err), sys->err_host, 0) !=
            cudaSuccess) {
      cudaGetLastError();
      rc = GSR_E_CUDA;
    } else {
      *sys->err_host = GSR_OK;
    }
  }
  A(dalloc(&sys->colnorm, (size_t)n_unk));
  A(dalloc(&sys->S.red, 65536));
  A(dalloc(&sys->S.count, 64));
  A(dalloc(&sys->S.x_ff, (size_t)n_unk));
  A(dalloc(&sys->S.x3, (size_t)n_buckets * 12));
  A(dalloc(&sys->S.y_ff, (size_t)padded_rows(L)));
  A(dalloc(&sys->S.y_knot, (size_t)n));
  A(dalloc(&sys->S.guard, 4));
  A(dalloc(&sys->S.iexp, 32));
  if (!rs.row.empty()) A(dalloc(&sys->row_exp, rs.row.size()));
  if (!rs.col.empty()) {
    A(dalloc(&sys->col_exp, rs.col.size()));
    A(dalloc(&sys->S.zx, (size_t)n_unk));
  }
  if (rc != GSR_OK) {
    free_system(sys);
    return rc;
  }
  if (cudaStreamCreateWithFlags(&sys->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&sys->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&sys->ev_join, cudaEventDisableTiming) != cudaSuccess) {
    free_system(sys);
    return GSR_E_CUDA;
  }

  auto fail = [&](int code) {
    cudaStreamSynchronize(st);
    free_system(sys);
    return code;
  };
  cudaError_t e = cudaSuccess;
  auto C = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
  };
  C(cudaMemsetAsync(sys->rec_ff, 0, (size_t)n_recs * Rec<false>::BYTES, st));
  if (want_f32) C(cudaMemsetAsync(sys->rec_f32, 0, (size_t)n_recs * Rec<true>::BYTES, st));
  C(cudaMemsetAsync(sys->S.count, 0, 64 * sizeof(unsigned int), st));
  C(cudaMemsetAsync(sys->colnorm, 0, (size_t)n_unk * sizeof(double), st));
  C(cudaMemsetAsync(sys->S.y_ff, 0, (size_t)padded_rows(L) * sizeof(float2), st));
  C(cudaMemsetAsync(sys->S.guard, 0, 4 * sizeof(double), st));
  if (sys->row_exp)
    C(cudaMemcpyAsync(sys->row_exp, rs.row.data(), rs.row.size() * sizeof(int16_t),
                      cudaMemcpyHostToDevice, st));
  if (sys->col_exp)
    C(cudaMemcpyAsync(sys->col_exp, rs.col.data(), rs.col.size() * sizeof(int16_t),
                      cudaMemcpyHostToDevice, st));
  C(cudaMemcpyAsync(sys->pos, pos.data(), (size_t)n * 4, cudaMemcpyHostToDevice, st));
  C(cudaMemcpyAsync(sys->knot_start, knot_start.data(), (size_t)(n_buckets + 1) * 8,
                    cudaMemcpyHostToDevice, st));
  if (n_kblk > 1) {
    C(cudaMemcpyAsync(sys->kb_start, kb_start.data(), kb_start.size() * 4,
                      cudaMemcpyHostToDevice, st));
    C(cudaMemcpyAsync(sys->gpos, gpos.data(), (size_t)n * 4, cudaMemcpyHostToDevice, st));
  }
  C(cudaMemcpyAsync(sys->att_warp_knot, att_warp_knot.data(), (size_t)(L.n_att_warps + 1) * 4,
                    cudaMemcpyHostToDevice, st));
  C(cudaMemcpyAsync(sys->iseg, ir.seg.data(), ir.seg.size() * sizeof(longlong2),
                    cudaMemcpyHostToDevice, st));
  C(cudaMemcpyAsync(sys->ient_key, ir.key.data(), n_ent * 4, cudaMemcpyHostToDevice, st));
  C(cudaMemcpyAsync(sys->ient_ff, ir.vff.data(), n_ent * 8, cudaMemcpyHostToDevice, st));
  if (want_f32)
    C(cudaMemcpyAsync(sys->ient_f32, ir.vf32.data(), n_ent * 4, cudaMemcpyHostToDevice, st));
  if (e != cudaSuccess) return fail(GSR_E_CUDA);

  L.rec_ff = sys->rec_ff;
  L.rec_f32 = sys->rec_f32;
  L.pos = sys->pos;
  L.att_knot_ff = sys->att_knot_ff;
  L.att_knot_f32 = sys->att_knot_f32;
  L.knot_start = sys->knot_start;
  L.kb_start = sys->kb_start;
  L.gpos = n_kblk > 1 ? sys->gpos : sys->pos;
  L.n_kblk = (int32_t)n_kblk;
  L.kblk_rows = kblk_rows;
  L.att_warp_knot = sys->att_warp_knot;
  L.iseg = sys->iseg;
  L.ient_ff = sys->ient_ff;
  L.ient_f32 = sys->ient_f32;
  L.ient_key = sys->ient_key;
  L.err = sys->err;
  L.row_exp = sys->row_exp;
  L.col_exp = sys->col_exp;

  // ---- chunked upload of the values and indices, laid out on the device ----
  if (n > 0) {
    const int64_t ch = std::min<int64_t>(CHUNK_ROWS, n);
    double* raw = nullptr;
    int32_t* raw_instr = nullptr;
    int32_t* d_star = nullptr;
    int32_t* d_sk = nullptr;
    int r1 = dalloc(&raw, (size_t)ch * NSLOT);
    int r2 = dalloc(&raw_instr, (size_t)ch * 6);
    int r3 = dalloc(&d_star, (size_t)n);
    int r4 = dalloc(&d_sk, (size_t)n);
    if (r1 != GSR_OK || r2 != GSR_OK || r3 != GSR_OK || r4 != GSR_OK) {
      if (raw) cudaFree(raw);
      if (raw_instr) cudaFree(raw_instr);
      if (d_star) cudaFree(d_star);
      if (d_sk) cudaFree(d_sk);
      return fail(r1 != GSR_OK ? r1 : r2 != GSR_OK ? r2 : r3 != GSR_OK ? r3 : r4);
    }
    C(cudaMemcpyAsync(d_star, star.data(), (size_t)n * 4, cudaMemcpyHostToDevice, st));
    C(cudaMemcpyAsync(d_sk, s_knot.data(), (size_t)n * 4, cudaMemcpyHostToDevice, st));
    for (int64_t r0 = 0; r0 < n && e == cudaSuccess; r0 += ch) {
      const int64_t m = std::min(ch, n - r0);
      C(cudaMemcpyAsync(raw, vals + r0 * NSLOT, (size_t)m * NSLOT * 8, cudaMemcpyHostToDevice, st));
      C(cudaMemcpyAsync(raw_instr, instr + r0 * 6, (size_t)m * 6 * 4, cudaMemcpyHostToDevice, st));
      const int blocks = (int)std::min<int64_t>((m + 255) / 256, sys->num_sms * 16);
      k_layout<<<blocks, 256, 0, st>>>(L, sys->rec_ff, sys->rec_f32, sys->att_knot_ff,
                                       sys->att_knot_f32, raw, raw_instr, d_star, d_sk,
                                       sys->colnorm, r0, m);
      C(cudaGetLastError());
    }
    const int64_t n_pad = n_recs * REC_ROWS - n;
    if (n_pad > 0) {
      k_pad_records<<<(int)((n_pad + 255) / 256), 256, 0, st>>>(L, sys->rec_ff, sys->rec_f32,
                                                                star[n - 1]);
      C(cudaGetLastError());
    }
    C(cudaStreamSynchronize(st));
    cudaFree(raw);
    cudaFree(raw_instr);
    cudaFree(d_star);
    cudaFree(d_sk);
  }
  k_sqrt<<<sys->num_sms * 4, 256, 0, st>>>(sys->colnorm, sys->col_exp, n_unk);
  C(cudaGetLastError());
  C(cudaStreamSynchronize(st));
  if (e != cudaSuccess) return fail(GSR_E_CUDA);
  if (set_kernel_attributes() != GSR_OK) return fail(GSR_E_CUDA);
  *out = sys;
  return GSR_OK;
}

void destroy_system(gsr_system* s) {
  if (!s) return;
  DeviceGuard dg(s->device);
  cudaDeviceSynchronize();
  free_system(s);
}

}  // namespace gsr

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

int gsr_create(const gsr_dims* dims, const double* vals, const int64_t* astro_off,
               const int64_t* att_off, const int32_t* instr, int device, void* stream,
               gsr_system** out) {
  if (!dims || !out) return GSR_E_ARG;
  *out = nullptr;
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) {
    cudaGetLastError();
    prev = -1;
  }
  const int rc = gsr::build_system(dims, vals, astro_off, att_off, instr, device,
                           static_cast<cudaStream_t>(stream), out);
  if (prev >= 0) cudaSetDevice(prev);  // leave the caller's current device as it was
  return rc;
}

void gsr_destroy(gsr_system* sys) { gsr::destroy_system(sys); }

const char* gsr_strerror(int status) {
  switch (status) {
    case GSR_OK: return "ok";
    case GSR_E_ARG: return "invalid argument";
    case GSR_E_INDEX: return "row index outside its block (astro/attitude/instrumental)";
    case GSR_E_UNSORTED: return "rows are not sorted by star";
    case GSR_E_NONFINITE: return "NaN or Inf in the input";
    case GSR_E_OOM: return "device memory allocation failed";
    case GSR_E_CUDA: return "CUDA runtime error";
    case GSR_E_TIMEOUT: return "bounded device wait ran out";
    case GSR_E_UNSUPPORTED: return "size beyond this build's limits";
    default: return "unknown status";
  }
}

int64_t gsr_n_unknowns(const gsr_system* sys) { return sys ? sys->L.n_unk : -1; }
int64_t gsr_n_rows(const gsr_system* sys) { return sys ? sys->L.n_rows : -1; }

int gsr_aprod1_values(gsr_system* sys, int which_values, const double* x, double* y,
                      void* stream) {
  if (!sys || (!x && sys->L.n_unk > 0) || (!y && sys->L.n_rows > 0)) return GSR_E_ARG;
  if (which_values != GSR_VALUES_F64 && which_values != GSR_VALUES_F32) return GSR_E_ARG;
  if (which_values == GSR_VALUES_F32 && !sys->rec_f32) return GSR_E_ARG;
  gsr::DeviceGuard dg(sys->device);
  if (!dg.ok) return GSR_E_CUDA;
  if (const int se = gsr::sticky_error(sys)) return se;  // an earlier launch failed
  return gsr::aprod1_direct(sys, which_values, x, 0, y, static_cast<cudaStream_t>(stream));
}

int gsr_aprod2_values(gsr_system* sys, int which_values, const double* y, double* x,
                      void* stream) {
  if (!sys || (!x && sys->L.n_unk > 0) || (!y && sys->L.n_rows > 0)) return GSR_E_ARG;
  if (which_values != GSR_VALUES_F64 && which_values != GSR_VALUES_F32) return GSR_E_ARG;
  if (which_values == GSR_VALUES_F32 && !sys->rec_f32) return GSR_E_ARG;
  gsr::DeviceGuard dg(sys->device);
  if (!dg.ok) return GSR_E_CUDA;
  if (const int se = gsr::sticky_error(sys)) return se;  // an earlier launch failed
  return gsr::aprod2_direct(sys, which_values, y, x, static_cast<cudaStream_t>(stream));
}

int gsr_aprod1(gsr_system* sys, const double* x, double* y, void* stream) {
  return gsr_aprod1_values(sys, GSR_VALUES_F64, x, y, stream);
}

int gsr_aprod2(gsr_system* sys, const double* y, double* x, void* stream) {
  return gsr_aprod2_values(sys, GSR_VALUES_F64, y, x, stream);
}

int gsr_column_norms(gsr_system* sys, double* c, void* stream) {
  if (!sys || !c) return GSR_E_ARG;
  gsr::DeviceGuard dg(sys->device);
  if (!dg.ok) return GSR_E_CUDA;
  if (const int se = gsr::sticky_error(sys)) return se;  // an earlier launch failed
  return gsr::cuda_status(cudaMemcpyAsync(c, sys->colnorm, (size_t)sys->L.n_unk * sizeof(double),
                                          cudaMemcpyDeviceToDevice,
                                          static_cast<cudaStream_t>(stream)));
}

}  // extern "C"
