// Mean bins of gridded data for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code running under an allocator that
// owns all device memory (a framework's caching pool or a fixed arena), code
// inside a region that must not allocate (for instance while other work
// holds the memory budget), or a plugin host that forbids allocations behind
// its back.  fpca_bin_mean_static gives them the mean binning of dense data
// with no allocation at all: the per-subject scratch (N_i) lives in a
// file-scope __device__ array of fixed size.
#include <cuda.h>

#include <mutex>

#include "fpca_internal.cuh"

namespace {

// Per-subject observation counts, at most kMaxSubjects subjects (4 MiB).
// Every GPU that loads the library holds this array until the process exits.
constexpr int kMaxSubjects = 1 << 20;
static __device__ __align__(256) int32_t g_subject_scratch[kMaxSubjects];

constexpr int kMaxDevices = 64;
// The device address of the array, looked up per device and remembered with
// the unique id of the context it was looked up in: after a cudaDeviceReset
// the device gets a new primary context (and the module, with the array, may
// load elsewhere), so a changed id triggers a new lookup.
int32_t* g_scratch_addr[kMaxDevices] = {};
unsigned long long g_scratch_ctx_id[kMaxDevices] = {};
std::mutex g_scratch_mutex;

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

template <typename Fn>
Fn driver_fn(const char* name) {
  void* p = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion(name, &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return reinterpret_cast<Fn>(p);
}

// Unique id of the calling thread's current context (0 if there is none or the
// driver does not report one).
unsigned long long current_ctx_id() {
  static CtxGetCurrentFn get_cur = driver_fn<CtxGetCurrentFn>("cuCtxGetCurrent");
  static CtxGetIdFn get_id = driver_fn<CtxGetIdFn>("cuCtxGetId");
  if (!get_cur || !get_id) return 0;
  CUcontext c = nullptr;
  if (get_cur(&c) != CUDA_SUCCESS || !c) return 0;
  unsigned long long id = 0;
  if (get_id(c, &id) != CUDA_SUCCESS) return 0;
  return id;
}

__device__ __forceinline__ double load_y(const void* y, int prec, size_t idx) {
  return prec == FPCA_F64 ? static_cast<const double*>(y)[idx]
                          : static_cast<double>(static_cast<const float*>(y)[idx]);
}

// N_i into the static scratch: one block per subject.
__global__ void k_subject_counts_static(int P, const uint8_t* __restrict__ mask,
                                        int32_t* __restrict__ Ni) {
  const int i = blockIdx.x;
  int c = 0;
  for (int p = threadIdx.x; p < P; p += blockDim.x)
    c += mask ? (mask[(size_t)i * P + p] != 0) : 1;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  __shared__ int part[32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x < 32) {
    int s = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) Ni[i] = s;
  }
}

// Dense mean bins (weights 1/N_i) reading N_i from the static scratch.
__global__ void k_bin_mean_dense_static(int n, int P, const void* __restrict__ y, int y_prec,
                                        const uint8_t* __restrict__ mask,
                                        const int32_t* __restrict__ Ni, int32_t* __restrict__ cnt,
                                        double* __restrict__ w, double* __restrict__ v,
                                        double* __restrict__ v2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  int c = 0;
  double sw = 0.0, sv = 0.0, sv2 = 0.0;
  for (int i = 0; i < n; ++i) {
    const size_t idx = (size_t)i * P + p;
    if (mask && !mask[idx]) continue;
    const int N = Ni[i];
    if (N <= 0) continue;
    const double wi = 1.0 / (double)N;
    const double yy = load_y(y, y_prec, idx);
    c += 1;
    sw = __dadd_rn(sw, wi);
    sv = __dadd_rn(sv, __dmul_rn(wi, yy));
    sv2 = __dadd_rn(sv2, __dmul_rn(wi, __dmul_rn(yy, yy)));
  }
  cnt[p] = c;
  w[p] = sw;
  v[p] = sv;
  if (v2) v2[p] = sv2;
}

}  // namespace

extern "C" fpca_status fpca_bin_mean_static(void* cuda_stream, int n, int P, const void* y,
                                            int y_prec, const uint8_t* mask, int32_t* cnt,
                                            double* w, double* v, double* v2) {
  if (n < 1 || P < 1 || !y || !cnt || !w || !v) return FPCA_E_INVALID_ARG;
  if (y_prec != FPCA_F64 && y_prec != FPCA_F32) return FPCA_E_INVALID_ARG;
  if (n > kMaxSubjects) return FPCA_E_UNSUPPORTED;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return FPCA_E_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return FPCA_E_UNSUPPORTED;
  int32_t* scratch = nullptr;
  {
    // set-up, once per device (and again if the device's context was replaced)
    // with that device current: the device address of the static array (its
    // name in host code is only a host-side stand-in)
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    const unsigned long long id = current_ctx_id();
    if (!g_scratch_addr[dev] || id == 0 || id != g_scratch_ctx_id[dev]) {
      void* addr = nullptr;
      if (cudaGetSymbolAddress(&addr, g_subject_scratch) != cudaSuccess) {
        cudaGetLastError();
        return FPCA_E_CUDA;
      }
      g_scratch_addr[dev] = static_cast<int32_t*>(addr);
      // the lookup makes the primary context current if nothing was yet
      g_scratch_ctx_id[dev] = current_ctx_id();
    }
    scratch = g_scratch_addr[dev];
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  k_subject_counts_static<<<n, 256, 0, s>>>(P, mask, scratch);
  if (cudaGetLastError() != cudaSuccess) return FPCA_E_CUDA;
  k_bin_mean_dense_static<<<(P + 127) / 128, 128, 0, s>>>(n, P, y, y_prec, mask, scratch, cnt, w,
                                                           v, v2);
  if (cudaGetLastError() != cudaSuccess) return FPCA_E_CUDA;
  return FPCA_OK;
}
