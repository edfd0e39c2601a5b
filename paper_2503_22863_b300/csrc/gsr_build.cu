// gsr_create / gsr_destroy and the plain aprod entry points.
//
// gsr_create validates the packed rows of Sec. 2 on the host (one pass,
// several threads), builds the small index structures (star-sorted warp
// ranges, the counting sort of rows by attitude start knot), uploads the
// values in chunks and lays them out on the device as float pairs in
// coalesced warp tiles, plus a knot-ordered copy of the attitude block. The
// column norms ||A_:,j|| (used by the column-scaling preconditioner, Sec. 2
// solver step 2) are computed on the device.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

#include "gsr_internal.cuh"

namespace gsr {

namespace {

constexpr int64_t CHUNK_ROWS = 1 << 22;  // rows per upload chunk (768 MB of values)
constexpr int MAX_HIST_INSTR = 28672;    // instrumental bins that fit a block's shared memory

__global__ void k_layout(Layout L, float* __restrict__ vals_ff, float* __restrict__ vals_f32,
                         float2* __restrict__ att_ff, float* __restrict__ att_f32,
                         uint16_t* __restrict__ instr_t, const double* __restrict__ raw,
                         const int32_t* __restrict__ raw_instr, const int32_t* __restrict__ star,
                         const int32_t* __restrict__ s_knot, const int32_t* __restrict__ pos,
                         double* __restrict__ c2, int64_t r0, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = r0 + i;
    const int64_t tile = r / TILE_ROWS;
    const int l = (int)((r % TILE_ROWS) / ROWS_PER_LANE);
    const int j = (int)(r % ROWS_PER_LANE);
    const int q = j >> 1, c = j & 1;
    const int64_t st = star[r], sk = s_knot[r], p = pos[r];
    for (int t = 0; t < NSLOT; ++t) {
      double v = raw[i * NSLOT + t];
      if (t == 23 && L.n_glob == 0) v = 0.0;
      const float h = __double2float_rn(v);
      const float lo = __double2float_rn(v - (double)h);
      const int64_t e = ((tile * NSLOT + t) * 2 + q) * 32 + l;
      vals_ff[e * 4 + 2 * c] = h;
      vals_ff[e * 4 + 2 * c + 1] = lo;
      if (vals_f32) vals_f32[e * 2 + c] = h;
      int64_t col;
      if (t < 5) {
        col = 5 * st + t;
      } else if (t < 17) {
        const int a = (t - 5) >> 2, jj = (t - 5) & 3;
        col = L.att_base + a * L.n_knots + sk + jj;
        att_ff[(int64_t)(t - 5) * L.n_rows + p] = make_float2(h, lo);
        if (att_f32) att_f32[(int64_t)(t - 5) * L.n_rows + p] = h;
      } else if (t < 23) {
        const int idx = raw_instr[i * 6 + (t - 17)];
        col = L.instr_base + idx;
        instr_t[((tile * 6 + (t - 17)) * 32 + l) * 4 + j] = (uint16_t)idx;
      } else {
        if (L.n_glob == 0) continue;
        col = L.glob_col;
      }
      atomicAdd(c2 + col, v * v);
    }
  }
}

__global__ void k_sqrt(double* __restrict__ a, int64_t n) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n;
       j += (int64_t)gridDim.x * blockDim.x)
    a[j] = sqrt(a[j]);
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
  void* ptrs[] = {s->vals_ff, s->vals_f32, s->star, s->att_s, s->att_pos, s->instr,
                  s->att_knot_ff, s->att_knot_f32, s->knot_start, s->att_warp_knot,
                  s->row_tile_warp, s->colnorm, s->u, s->u_knot, s->v, s->w, s->xz, s->z,
                  s->dscale, s->v_ff, s->scal, s->S.red, s->S.count, s->S.x_ff, s->S.y_knot};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (s->host_scal) cudaFreeHost(s->host_scal);
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
  const int64_t n = d.n_rows;
  const int64_t n_tiles = (n + TILE_ROWS - 1) / TILE_ROWS;
  const int64_t n_pad = n_tiles * TILE_ROWS;

  // ---- host validation and per-row indices (multi-threaded) ----
  std::vector<int32_t> star(n_pad), s_knot(n_pad), pos(n_pad);
  {
    unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    if (n < 100000) nt = 1;
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
  // padded rows: same star as the last row, knot 0, zero values
  for (int64_t r = n; r < n_pad; ++r) {
    star[r] = n > 0 ? star[n - 1] : 0;
    s_knot[r] = 0;
    pos[r] = 0;
  }
  // ---- counting sort of rows by start knot (stable) ----
  const int64_t n_buckets = d.n_knots - 3;
  std::vector<int64_t> knot_start(n_buckets + 1, 0);
  for (int64_t r = 0; r < n; ++r) knot_start[s_knot[r] + 1]++;
  for (int64_t b = 0; b < n_buckets; ++b) knot_start[b + 1] += knot_start[b];
  {
    std::vector<int64_t> next(knot_start.begin(), knot_start.end() - 1);
    for (int64_t r = 0; r < n; ++r) pos[r] = (int32_t)(next[s_knot[r]]++);
  }

  // host validation is done; everything below needs the device
  if (cudaSetDevice(device) != cudaSuccess) return GSR_E_CUDA;
  gsr_system* sys = new (std::nothrow) gsr_system();
  if (!sys) return GSR_E_OOM;
  std::memset(sys, 0, sizeof(*sys));
  sys->device = device;
  sys->dims = d;
  cudaDeviceGetAttribute(&sys->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (sys->num_sms <= 0) sys->num_sms = NUM_SMS_B300;

  Layout& L = sys->L;
  L.n_rows = n;
  L.n_stars = d.n_stars;
  L.n_knots = d.n_knots;
  L.n_instr = d.n_instr;
  L.n_glob = d.n_glob;
  L.n_unk = n_unk;
  L.n_tiles = n_tiles;
  L.att_base = 5 * d.n_stars;
  L.instr_base = L.att_base + 3 * d.n_knots;
  L.glob_col = L.instr_base + d.n_instr;

  // ---- launch shapes and warp partitions ----
  sys->hist_bytes = (int)(d.n_instr * sizeof(double));
  sys->main_block = 512;
  // one 512-thread block per SM: the kernel needs ~110 registers per thread
  const int per_sm = 1;
  sys->main_ctas = sys->num_sms * per_sm;
  L.n_main_warps = sys->main_ctas * (sys->main_block / 32);
  std::vector<int64_t> row_tile_warp(L.n_main_warps + 1);
  for (int w = 0; w <= L.n_main_warps; ++w)
    row_tile_warp[w] = (n_tiles * (int64_t)w) / L.n_main_warps;
  L.n_att_warps = sys->num_sms * 16;
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
  int rc = GSR_OK;
  auto A = [&](int r) {
    if (rc == GSR_OK) rc = r;
  };
  A(dalloc(&sys->vals_ff, (size_t)n_pad * NSLOT / 2));  // float4 per 2 rows per slot
  if (d.storage == GSR_STORE_F32_PLUS_F64) A(dalloc(&sys->vals_f32, (size_t)n_pad * NSLOT / 2 + 1));
  A(dalloc(&sys->star, (size_t)n_pad / 4 + 1));
  A(dalloc(&sys->att_s, (size_t)n_pad / 4 + 1));
  A(dalloc(&sys->att_pos, (size_t)n_pad / 4 + 1));
  A(dalloc(&sys->instr, (size_t)n_pad * 6 / 4 + 1));
  A(dalloc(&sys->att_knot_ff, (size_t)n * 12));
  if (d.storage == GSR_STORE_F32_PLUS_F64) A(dalloc(&sys->att_knot_f32, (size_t)n * 12));
  A(dalloc(&sys->knot_start, (size_t)n_buckets + 1));
  A(dalloc(&sys->att_warp_knot, (size_t)L.n_att_warps + 1));
  A(dalloc(&sys->row_tile_warp, (size_t)L.n_main_warps + 1));
  A(dalloc(&sys->colnorm, (size_t)n_unk));
  A(dalloc(&sys->S.red, 65536));
  A(dalloc(&sys->S.count, 64));
  A(dalloc(&sys->S.x_ff, (size_t)n_unk));
  A(dalloc(&sys->S.y_knot, (size_t)n));
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
  C(cudaMemsetAsync(sys->vals_ff, 0, (size_t)n_pad * NSLOT * sizeof(float4) / 2, st));
  if (sys->vals_f32) C(cudaMemsetAsync(sys->vals_f32, 0, (size_t)n_pad * NSLOT * sizeof(float), st));
  C(cudaMemsetAsync(sys->instr, 0, (size_t)n_pad * 6 * sizeof(uint16_t), st));
  C(cudaMemsetAsync(sys->S.count, 0, 64 * sizeof(unsigned int), st));
  C(cudaMemsetAsync(sys->colnorm, 0, (size_t)n_unk * sizeof(double), st));
  C(cudaMemcpyAsync(sys->star, star.data(), (size_t)n_pad * 4, cudaMemcpyHostToDevice, st));
  C(cudaMemcpyAsync(sys->att_s, s_knot.data(), (size_t)n_pad * 4, cudaMemcpyHostToDevice, st));
  C(cudaMemcpyAsync(sys->att_pos, pos.data(), (size_t)n_pad * 4, cudaMemcpyHostToDevice, st));
  C(cudaMemcpyAsync(sys->knot_start, knot_start.data(), (size_t)(n_buckets + 1) * 8,
                    cudaMemcpyHostToDevice, st));
  C(cudaMemcpyAsync(sys->att_warp_knot, att_warp_knot.data(), (size_t)(L.n_att_warps + 1) * 4,
                    cudaMemcpyHostToDevice, st));
  C(cudaMemcpyAsync(sys->row_tile_warp, row_tile_warp.data(), (size_t)(L.n_main_warps + 1) * 8,
                    cudaMemcpyHostToDevice, st));
  if (e != cudaSuccess) return fail(GSR_E_CUDA);

  L.vals_ff = sys->vals_ff;
  L.vals_f32 = sys->vals_f32;
  L.star = sys->star;
  L.att_s = sys->att_s;
  L.att_pos = sys->att_pos;
  L.instr = sys->instr;
  L.att_knot_ff = sys->att_knot_ff;
  L.att_knot_f32 = sys->att_knot_f32;
  L.knot_start = sys->knot_start;
  L.att_warp_knot = sys->att_warp_knot;
  L.row_tile_warp = sys->row_tile_warp;

  // ---- chunked upload of the values and instrumental indices ----
  if (n > 0) {
    const int64_t ch = std::min<int64_t>(CHUNK_ROWS, n);
    double* raw = nullptr;
    int32_t* raw_instr = nullptr;
    int r1 = dalloc(&raw, (size_t)ch * NSLOT);
    int r2 = dalloc(&raw_instr, (size_t)ch * 6);
    if (r1 != GSR_OK || r2 != GSR_OK) {
      if (raw) cudaFree(raw);
      if (raw_instr) cudaFree(raw_instr);
      return fail(r1 != GSR_OK ? r1 : r2);
    }
    for (int64_t r0 = 0; r0 < n && e == cudaSuccess; r0 += ch) {
      const int64_t m = std::min(ch, n - r0);
      C(cudaMemcpyAsync(raw, vals + r0 * NSLOT, (size_t)m * NSLOT * 8, cudaMemcpyHostToDevice, st));
      C(cudaMemcpyAsync(raw_instr, instr + r0 * 6, (size_t)m * 6 * 4, cudaMemcpyHostToDevice, st));
      int blocks = (int)std::min<int64_t>((m + 255) / 256, sys->num_sms * 16);
      k_layout<<<blocks, 256, 0, st>>>(L, reinterpret_cast<float*>(sys->vals_ff),
                                       reinterpret_cast<float*>(sys->vals_f32), sys->att_knot_ff,
                                       sys->att_knot_f32, reinterpret_cast<uint16_t*>(sys->instr),
                                       raw, raw_instr, reinterpret_cast<const int32_t*>(sys->star),
                                       reinterpret_cast<const int32_t*>(sys->att_s),
                                       reinterpret_cast<const int32_t*>(sys->att_pos),
                                       sys->colnorm, r0, m);
      C(cudaGetLastError());
    }
    C(cudaStreamSynchronize(st));
    cudaFree(raw);
    cudaFree(raw_instr);
  }
  k_sqrt<<<sys->num_sms * 4, 256, 0, st>>>(sys->colnorm, n_unk);
  C(cudaGetLastError());
  C(cudaStreamSynchronize(st));
  if (e != cudaSuccess) return fail(GSR_E_CUDA);
  if (set_kernel_attributes(MAX_HIST_INSTR * (int)sizeof(double)) != GSR_OK) return fail(GSR_E_CUDA);

  *out = sys;
  return GSR_OK;
}

void destroy_system(gsr_system* s) {
  if (!s) return;
  cudaSetDevice(s->device);
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
  return gsr::build_system(dims, vals, astro_off, att_off, instr, device,
                           static_cast<cudaStream_t>(stream), out);
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
  if (which_values == GSR_VALUES_F32 && !sys->vals_f32) return GSR_E_ARG;
  if (cudaSetDevice(sys->device) != cudaSuccess) return GSR_E_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc = gsr::launch_to_ff(x, nullptr, sys->S.x_ff, sys->L.n_unk, st);
  if (rc != GSR_OK) return rc;
  return gsr::launch_aprod1(sys, which_values, sys->S.x_ff, y, nullptr, 1.0, nullptr, nullptr,
                            nullptr, st);
}

int gsr_aprod2_values(gsr_system* sys, int which_values, const double* y, double* x,
                      void* stream) {
  if (!sys || (!x && sys->L.n_unk > 0) || (!y && sys->L.n_rows > 0)) return GSR_E_ARG;
  if (which_values != GSR_VALUES_F64 && which_values != GSR_VALUES_F32) return GSR_E_ARG;
  if (which_values == GSR_VALUES_F32 && !sys->vals_f32) return GSR_E_ARG;
  if (cudaSetDevice(sys->device) != cudaSuccess) return GSR_E_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int rc = gsr::launch_scatter_knot(sys, y, sys->S.y_knot, st);
  if (rc != GSR_OK) return rc;
  return gsr::launch_aprod2(sys, which_values, y, sys->S.y_knot, x, nullptr, st);
}

int gsr_aprod1(gsr_system* sys, const double* x, double* y, void* stream) {
  return gsr_aprod1_values(sys, GSR_VALUES_F64, x, y, stream);
}

int gsr_aprod2(gsr_system* sys, const double* y, double* x, void* stream) {
  return gsr_aprod2_values(sys, GSR_VALUES_F64, y, x, stream);
}

int gsr_column_norms(gsr_system* sys, double* c, void* stream) {
  if (!sys || !c) return GSR_E_ARG;
  if (cudaSetDevice(sys->device) != cudaSuccess) return GSR_E_CUDA;
  return gsr::cuda_status(cudaMemcpyAsync(c, sys->colnorm, (size_t)sys->L.n_unk * sizeof(double),
                                          cudaMemcpyDeviceToDevice,
                                          static_cast<cudaStream_t>(stream)));
}

}  // extern "C"
