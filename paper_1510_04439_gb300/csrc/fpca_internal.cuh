// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <array>
#include <cstdint>
#include <cstddef>
#include <map>
#include <string>
#include <vector>

#include "fpca.h"

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
struct fpca_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string err;
  void* ws = nullptr;        // workspace, grown on demand
  size_t ws_bytes = 0;
  int* d_err = nullptr;      // device error word (DERR_*)
  uint64_t launches = 0;     // kernels queued by this context
  int num_sms = 0;
  size_t smem_optin = 0;
  // opt-in kernel timing: an event after every launch, durations between
  // consecutive events (the first one is marked at the top of each call)
  int prof = 0;
  cudaEvent_t prof_last = nullptr;
  struct ProfRec {
    std::string name;
    cudaEvent_t a, b;
  };
  std::vector<ProfRec> prof_pending;
  std::vector<cudaEvent_t> prof_pool;
  std::map<std::string, std::pair<double, uint64_t>> prof_totals;
  std::vector<std::string> prof_names;  // stable storage for fpca_profile_entry
  // d = 3 fused smoother: tile-pair work lists for the last grid / taps seen
  void* f3_lists = nullptr;
  size_t f3_lists_bytes = 0;
  int f3_key[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int f3_ncta = 0, f3_nitems = 0, f3_npairs = 0;
  // t-side sweep kernel of the FP32 d = 2 covariance smoother: 0 = automatic,
  // 1 = the scalar sweep (k_hsolve2), 2 = the packed-pair sweep where built;
  // the automatic choice per (M1, M2, T1, T2, compensated, half) once timed:
  // 1 or 2 as above
  int tside_kernel = 0;
  std::map<std::array<int, 6>, int> tside_choice;
  // schedule of the K-fold CV grid of the FP32 d = 2 smoother: 0 item by item,
  // 1 batched (one persistent t-side launch), 2 automatic; the automatic choice
  // per (M1, M2, folds, compensated, taps of every bandwidth) once timed: 0 or 1
  int cv_batch = 2;
  std::map<std::vector<int>, int> cv_choice;
  // CUDA-graph capture of the context's stream (fpca_graph_begin / _end): set while
  // capturing; a call that cannot be captured (a host read-back, a workspace growth,
  // an autotuner's timing, a copy from host memory) refuses and marks the capture
  int capturing = 0;
  int capture_failed = 0;
  uint64_t capture_launches = 0;  // ctx->launches when the capture began
};

// Device error codes written by kernels into ctx->d_err.
enum { DERR_NONE = 0, DERR_TIMEOUT = 1, DERR_BOUNDS = 2, DERR_NUMERIC = 3 };

// Bounded waits give up after this many nanoseconds of %globaltimer.
#define FPCA_WAIT_LIMIT_NS 2000000000ull

fpca_status fpca_fail(fpca_ctx* ctx, fpca_status st, const char* fmt, ...);
// FPCA_OK outside a graph capture; inside one, marks the capture as failed and
// returns FPCA_E_UNSUPPORTED naming `what` (work that cannot be captured).
fpca_status fpca_no_capture(fpca_ctx* ctx, const char* what);
// Checks the last launch; records the CUDA error text on failure.
fpca_status fpca_check_launch(fpca_ctx* ctx, const char* what);
// Returns a device buffer of at least `bytes`, growing the workspace (which
// synchronises the stream first). nullptr on allocation failure.
void* fpca_workspace(fpca_ctx* ctx, size_t bytes);

// Marks the start of an API call's work on the stream (kernel timing).
void fpca_prof_mark(fpca_ctx* ctx);
// Records the end of the kernel just launched (kernel timing).
void fpca_prof_end(fpca_ctx* ctx, const char* name);

#define FPCA_LAUNCHED(ctx, name)                                   \
  do {                                                             \
    (ctx)->launches++;                                             \
    fpca_status _s = fpca_check_launch((ctx), (name));             \
    if (_s != FPCA_OK) return _s;                                  \
    if ((ctx)->prof) fpca_prof_end((ctx), (name));                 \
  } while (0)

// Bump allocator over one workspace block (256-byte aligned pieces).
struct WsCarve {
  char* base;
  size_t off = 0;
  explicit WsCarve(void* b) : base(static_cast<char*>(b)) {}
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = reinterpret_cast<T*>(base + off);
    off += count * sizeof(T);
    return p;
  }
  static size_t round(size_t bytes) { return (bytes + 255) & ~size_t(255); }
};

inline int grid_P(const fpca_grid* g) {
  int P = 1;
  for (int k = 0; k < g->d; ++k) P *= g->m[k];
  return P;
}

// ---------------------------------------------------------------------------
// launchers implemented in the .cu files (all queue on ctx->stream)
// ---------------------------------------------------------------------------
// bin.cu
fpca_status launch_subject_counts_dense(fpca_ctx* ctx, int n, int P, const uint8_t* mask,
                                        int32_t* Ni);
fpca_status launch_bin_mean_dense(fpca_ctx* ctx, int n, int P, const void* y, int y_prec,
                                  const uint8_t* mask, const int32_t* Ni, int32_t* cnt,
                                  double* w, double* v, double* v2);
fpca_status launch_bin_mean_sparse(fpca_ctx* ctx, int n, const fpca_grid* g, const int64_t* offs,
                                   const double* t, const double* y, int32_t* cnt, double* w,
                                   double* v, double* v2);
fpca_status launch_cov_operands_bf16(fpca_ctx* ctx, int n, int P, int Kpad, const void* y,
                                     int y_prec, const uint8_t* mask, const int32_t* Ni,
                                     const double* mu, int mode, uint16_t* ops);
fpca_status launch_cov_dense_f64(fpca_ctx* ctx, int n, int P, const void* y, int y_prec,
                                 const uint8_t* mask, const int32_t* Ni, const double* mu,
                                 int mode, int32_t* cnt, double* w, double* v);
// FP32 bins of gridded data split by folds (q may be NULL; nfold 0 = one slice)
fpca_status launch_cov_dense_folds(fpca_ctx* ctx, int n, int P, const void* y, int y_prec,
                                   const uint8_t* mask, const double* mu, int mode,
                                   const int32_t* fold, int nfold, int32_t* cnt, float* w,
                                   float* v, float* q);
fpca_status launch_cov_sparse(fpca_ctx* ctx, int n, const fpca_grid* g, const int64_t* offs,
                              const double* t, const double* y, const double* mu, int mode,
                              const int32_t* fold, int nfold, int prec, int32_t* cnt, void* w,
                              void* v, void* q);
// gemm_tc.cu: C = X'X for the three operand planes (mask, sqrt(w) mask, sqrt(w) R)
fpca_status launch_gram_tc(fpca_ctx* ctx, int P, int Kpad, const uint16_t* ops, int32_t* cnt,
                           float* w, float* v);
// smooth.cu
// scratch: NULL (the context's workspace) or smooth_mean_scratch_bytes(P) bytes of
// device memory the call may use (256-byte aligned)
size_t smooth_mean_scratch_bytes(int P);
fpca_status launch_smooth_mean(fpca_ctx* ctx, const fpca_grid* g, const int32_t* cnt,
                               const double* w, const double* v, const double* h, double* mu,
                               uint8_t* status, void* scratch = nullptr);
// mean-smoother CV of scattered data (smooth.cu)
fpca_status mean_cv_run(fpca_ctx* ctx, const fpca_grid* g, int n, const int64_t* offs,
                        const double* t, const double* y, const int32_t* fold, int nfold,
                        const double* h, int nh, double* cv);
fpca_status launch_sigma2(fpca_ctx* ctx, const fpca_grid* g, const int32_t* cnt, const double* w,
                          const double* v2, const double* h, const double* mu, const void* gdiag,
                          int gprec, long long gstride, const int32_t* domain, double* sig_t,
                          uint8_t* status, double* sigma2);
fpca_status smooth_cov_run(fpca_ctx* ctx, const fpca_grid* g, const fpca_covbins* bins,
                           const double* h, int nh, int prec, const double* mu_raw,
                           const float* omega, int l, void* gamma, uint8_t* status, float* y,
                           double* cv);
// eig.cu
struct RprojOp {
  fpca_status (*apply)(void* self, const float* X, float* Y);  // Y = Sigma X, P x l
  void* self;
};
struct RprojWs {
  float *Y, *Q, *Z;
  double *G, *Rinv, *A, *V, *trace;
  int* order;
  double* part;  // per-block partial Gram products
  double* rr;    // Rayleigh-Ritz eigensolver scratch (5 l^2 + l)
};
size_t rproj_ws_bytes(const fpca_ctx* ctx, int P, int l);
void rproj_ws_carve(const fpca_ctx* ctx, WsCarve& c, int P, int l, RprojWs& w);
fpca_status rproj_operator(fpca_ctx* ctx, int P, int l, int k, int power_iters, double dv,
                           const float* omega, RprojOp op, const RprojWs& w, double* evals,
                           double* evecs, double* fve);
fpca_status rproj_eig_run(fpca_ctx* ctx, const fpca_grid* g, const void* gamma, int gamma_prec,
                          const int32_t* domain, const float* omega, int l, int k,
                          int power_iters, int full, double* evals, double* evecs,
                          double* fve);
