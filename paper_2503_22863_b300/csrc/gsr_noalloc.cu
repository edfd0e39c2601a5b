// gsr_aprod1_noalloc: aprod 1 (y += A x) whose only scratch lives in a fixed,
// file-scope device array of this library instead of memory allocated by the
// library or the caller.
//
// Who needs it: code that must not allocate device memory at the moment it
// calls us. Typical cases are a process whose device memory has been taken up
// front by another framework's caching allocator, and latency-critical loops
// where the implicit device synchronisation of cudaMalloc/cudaFree is not
// acceptable. This entry point calls no cudaMalloc, cudaFree or any allocating
// routine; the caller only passes x and y.
//
// The scratch is the float-pair copy of x that the aprod 1 kernel gathers from.
// It holds at most GSR_NOALLOC_MAX_UNK unknowns (8 MiB of float pairs), a size
// every GPU that loads the library keeps reserved until the process exits.
#include <mutex>

#include "gsr_system.cuh"

namespace {

constexpr int64_t kMaxUnk = GSR_NOALLOC_MAX_UNK;
constexpr int kMaxDevices = 64;

// The static scratch: one copy per device, reserved when the module loads.
static __device__ __align__(256) float2 g_x_pairs[kMaxUnk];
// Set when x leaves the range the float-pair kernel handles exactly (the FP64
// kernel then computes the product instead).
static __device__ __align__(8) double g_guard;

// Host code cannot pass the symbols themselves to a kernel (on the host they
// name stand-ins, not device memory), so the device addresses are looked up
// once per device, with that device current, and cached here.
std::mutex g_mu;
float2* g_addr[kMaxDevices] = {};
double* g_guard_addr[kMaxDevices] = {};

int static_scratch(int device, float2** out, double** guard) {
  if (device < 0 || device >= kMaxDevices) return GSR_E_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[device]) {
    void* p = nullptr;
    void* q = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_x_pairs);
    if (e == cudaSuccess) e = cudaGetSymbolAddress(&q, g_guard);
    if (e != cudaSuccess || p == nullptr || q == nullptr) {
      cudaGetLastError();
      return GSR_E_CUDA;
    }
    g_addr[device] = static_cast<float2*>(p);
    g_guard_addr[device] = static_cast<double*>(q);
  }
  *out = g_addr[device];
  *guard = g_guard_addr[device];
  return GSR_OK;
}

}  // namespace

extern "C" int gsr_aprod1_noalloc(gsr_system* sys, const double* x, double* y, void* stream) {
  if (!sys || (!x && sys->L.n_unk > 0) || (!y && sys->L.n_rows > 0)) return GSR_E_ARG;
  if (sys->L.n_unk > kMaxUnk) return GSR_E_UNSUPPORTED;
  gsr::DeviceGuard dg(sys->device);
  if (!dg.ok) return GSR_E_CUDA;
  if (const int se = gsr::sticky_error(sys)) return se;  // an earlier launch failed
  float2* pairs = nullptr;
  double* guard = nullptr;
  int rc = static_scratch(sys->device, &pairs, &guard);
  if (rc != GSR_OK) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the constraint rows (FP64 kernel, no scratch)
  rc = gsr::con_aprod1_direct(sys, x, 0, y, st);
  if (rc != GSR_OK || sys->L.n_rows == 0) return rc;
  // coefficients too spread for the float pairs: the FP64 kernel, no scratch
  if (sys->wide) return gsr::launch_aprod1_f64(sys, GSR_VALUES_F64, x, 1, 0, y, nullptr, st);
  // Every call rewrites pairs[0, N_unk) and the flag before the product reads
  // them, so no part of the shared buffer has to start at zero.
  if (cudaMemsetAsync(guard, 0, sizeof(double), st) != cudaSuccess) return GSR_E_CUDA;
  rc = gsr::launch_to_ff(x, nullptr, sys->L.col_exp, 0, guard, pairs, sys->L.n_unk, st);
  if (rc != GSR_OK) return rc;
  rc = gsr::launch_aprod1(sys, GSR_VALUES_F64, pairs, y, nullptr, 1.0, nullptr, nullptr, guard,
                          st);
  if (rc != GSR_OK) return rc;
  return gsr::launch_aprod1_f64(sys, GSR_VALUES_F64, x, 1, 0, y, guard, st);
}
