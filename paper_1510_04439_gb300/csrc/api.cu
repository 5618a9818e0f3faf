// C ABI entry points: context, argument checks and dispatch to the kernels.
#include <cstdarg>
#include <cstdio>
#include <cmath>
#include <new>

#include "fpca_internal.cuh"
#include "ptx.cuh"

fpca_status fpca_fail(fpca_ctx* ctx, fpca_status st, const char* fmt, ...) {
  if (ctx && ctx->capturing && ctx->capture_failed) {
    // a refusal inside a graph capture (fpca_no_capture) already set the text; the
    // caller's own failure on top of it (e.g. a workspace it could not grow) keeps it
    return FPCA_E_UNSUPPORTED;
  }
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    ctx->err = buf;
  }
  return st;
}

fpca_status fpca_check_launch(fpca_ctx* ctx, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return fpca_fail(ctx, FPCA_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
  return FPCA_OK;
}

static cudaEvent_t prof_event(fpca_ctx* ctx) {
  cudaEvent_t e = nullptr;
  if (!ctx->prof_pool.empty()) {
    e = ctx->prof_pool.back();
    ctx->prof_pool.pop_back();
  } else if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (cudaEventRecord(e, ctx->stream) != cudaSuccess) {
    cudaGetLastError();
    ctx->prof_pool.push_back(e);
    return nullptr;
  }
  return e;
}

void fpca_prof_mark(fpca_ctx* ctx) {
  if (!ctx->prof) return;
  cudaEvent_t e = prof_event(ctx);
  if (e) {
    // an unpaired previous mark is recycled once resolved
    if (ctx->prof_last) ctx->prof_pending.push_back({std::string(), ctx->prof_last, nullptr});
    ctx->prof_last = e;
  }
}

void fpca_prof_end(fpca_ctx* ctx, const char* name) {
  cudaEvent_t e = prof_event(ctx);
  if (!e) return;
  if (ctx->prof_last) ctx->prof_pending.push_back({std::string(name), ctx->prof_last, e});
  ctx->prof_last = e;
}

static void prof_resolve(fpca_ctx* ctx) {
  if (ctx->prof_pending.empty()) return;
  cudaStreamSynchronize(ctx->stream);
  std::vector<cudaEvent_t> done;
  for (auto& r : ctx->prof_pending) {
    if (r.b && !r.name.empty()) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
        auto& t = ctx->prof_totals[r.name];
        t.first += ms;
        t.second += 1;
      } else {
        cudaGetLastError();
      }
    }
    done.push_back(r.a);
  }
  ctx->prof_pending.clear();
  // every start event is some record's `a`; the current last mark stays live
  for (cudaEvent_t e : done)
    if (e != ctx->prof_last) ctx->prof_pool.push_back(e);
}

fpca_status fpca_no_capture(fpca_ctx* ctx, const char* what) {
  if (!ctx->capturing) return FPCA_OK;
  if (!ctx->capture_failed)
    fpca_fail(ctx, FPCA_E_UNSUPPORTED,
              "%s cannot run inside a graph capture (run the calls once before capturing)", what);
  ctx->capture_failed = 1;
  return FPCA_E_UNSUPPORTED;
}

void* fpca_workspace(fpca_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->ws_bytes) return ctx->ws;
  // growing synchronises the stream and reallocates: not inside a capture
  if (fpca_no_capture(ctx, "growing the workspace") != FPCA_OK) return nullptr;
  // Growing: the old block may still be in use by queued work.
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return nullptr;
  if (ctx->ws) cudaFree(ctx->ws);
  ctx->ws = nullptr;
  ctx->ws_bytes = 0;
  size_t want = bytes + bytes / 4;
  if (cudaMalloc(&ctx->ws, want) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  ctx->ws_bytes = want;
  return ctx->ws;
}

static bool valid_grid(fpca_ctx* ctx, const fpca_grid* g, int max_m) {
  if (!g) return false;
  if (g->d < 1 || g->d > 3) {
    fpca_fail(ctx, FPCA_E_INVALID_ARG, "grid.d must be 1..3 (got %d)", g->d);
    return false;
  }
  for (int k = 0; k < g->d; ++k) {
    if (g->m[k] < 1 || g->m[k] > max_m) {
      fpca_fail(ctx, FPCA_E_INVALID_ARG, "grid.m[%d] = %d outside 1..%d", k, g->m[k], max_m);
      return false;
    }
  }
  return true;
}

static bool valid_h(fpca_ctx* ctx, const double* h, int count) {
  if (!h) {
    fpca_fail(ctx, FPCA_E_INVALID_ARG, "bandwidth pointer is NULL");
    return false;
  }
  for (int i = 0; i < count; ++i) {
    if (!(h[i] > 0.0) || !std::isfinite(h[i])) {
      fpca_fail(ctx, FPCA_E_INVALID_ARG, "bandwidth h[%d] = %g must be finite and > 0", i, h[i]);
      return false;
    }
  }
  return true;
}

static bool valid_data(fpca_ctx* ctx, const fpca_data* data) {
  if (!data) {
    fpca_fail(ctx, FPCA_E_INVALID_ARG, "data is NULL");
    return false;
  }
  if (data->n < 1) {
    fpca_fail(ctx, FPCA_E_INVALID_ARG, "data.n must be >= 1 (got %d)", data->n);
    return false;
  }
  if (data->layout == FPCA_DENSE) {
    if (!data->y || (data->y_prec != FPCA_F64 && data->y_prec != FPCA_F32)) {
      fpca_fail(ctx, FPCA_E_INVALID_ARG, "dense data needs y with y_prec FPCA_F64 or FPCA_F32");
      return false;
    }
    return true;
  }
  if (data->layout == FPCA_SPARSE) {
    if (!data->y || !data->offs || !data->t || data->y_prec != FPCA_F64) {
      fpca_fail(ctx, FPCA_E_INVALID_ARG, "sparse data needs offs, t and FP64 y");
      return false;
    }
    return true;
  }
  fpca_fail(ctx, FPCA_E_INVALID_ARG, "data.layout must be FPCA_DENSE or FPCA_SPARSE");
  return false;
}

extern "C" {

fpca_status fpca_create(fpca_ctx** out, int device, void* cuda_stream) {
  if (!out) return FPCA_E_INVALID_ARG;
  *out = nullptr;
  fpca_ctx* ctx = new (std::nothrow) fpca_ctx();
  if (!ctx) return FPCA_E_OOM;
  ctx->device = device;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    delete ctx;
    return FPCA_E_CUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) {
    delete ctx;
    return FPCA_E_CUDA;
  }
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
    delete ctx;
    return FPCA_E_CUDA;
  }
  if (prop.major != 10 || prop.minor != 3) {
    delete ctx;
    return FPCA_E_UNSUPPORTED;
  }
  ctx->num_sms = prop.multiProcessorCount;
  ctx->smem_optin = prop.sharedMemPerBlockOptin;
  if (cudaMalloc(&ctx->d_err, sizeof(int)) != cudaSuccess) {
    delete ctx;
    return FPCA_E_OOM;
  }
  if (cudaMemset(ctx->d_err, 0, sizeof(int)) != cudaSuccess) {
    cudaFree(ctx->d_err);
    delete ctx;
    return FPCA_E_CUDA;
  }
  *out = ctx;
  return FPCA_OK;
}

void fpca_destroy(fpca_ctx* ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  prof_resolve(ctx);
  for (cudaEvent_t e : ctx->prof_pool) cudaEventDestroy(e);
  if (ctx->prof_last) cudaEventDestroy(ctx->prof_last);
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->d_err) cudaFree(ctx->d_err);
  if (ctx->f3_lists) cudaFree(ctx->f3_lists);
  delete ctx;
}

fpca_status fpca_set_stream(fpca_ctx* ctx, void* cuda_stream) {
  if (!ctx) return FPCA_E_INVALID_ARG;
  ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  return FPCA_OK;
}

const char* fpca_last_error(const fpca_ctx* ctx) { return ctx ? ctx->err.c_str() : "no context"; }

uint64_t fpca_launch_count(const fpca_ctx* ctx) { return ctx ? ctx->launches : 0; }

// Self-check of the failure detection: one thread waits on a shared-memory
// mbarrier that expects one arrival, through the same bounded wait the tensor-
// core and bulk-copy kernels use; with `arrive` set a thread arrives first.
__global__ void k_wait_probe(int arrive, int* err) {
  __shared__ __align__(8) uint64_t bar;
  const uint32_t b = ptx::smem_u32(&bar);
  if (threadIdx.x == 0) {
    ptx::mbar_init(b, 1);
    ptx::fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (arrive) ptx::mbar_arrive(b);
    ptx::mbar_wait(b, 0, err);  // gives up after FPCA_WAIT_LIMIT_NS, records DERR_TIMEOUT
  }
}

fpca_status fpca_set_sweep_kernel(fpca_ctx* ctx, int kernel) {
  if (!ctx) return FPCA_E_INVALID_ARG;
  if (kernel < 0 || kernel > 2)
    return fpca_fail(ctx, FPCA_E_INVALID_ARG, "sweep kernel must be 0 (automatic), 1 or 2");
  ctx->tside_kernel = kernel;
  return FPCA_OK;
}

fpca_status fpca_set_cv_batch(fpca_ctx* ctx, int batch) {
  if (!ctx) return FPCA_E_INVALID_ARG;
  if (batch < 0 || batch > 2)
    return fpca_fail(ctx, FPCA_E_INVALID_ARG, "CV schedule must be 0, 1 or 2 (automatic)");
  ctx->cv_batch = batch;
  return FPCA_OK;
}

fpca_status fpca_check_wait(fpca_ctx* ctx, int arrive) {
  if (!ctx) return FPCA_E_INVALID_ARG;
  fpca_prof_mark(ctx);
  k_wait_probe<<<1, 32, 0, ctx->stream>>>(arrive ? 1 : 0, ctx->d_err);
  FPCA_LAUNCHED(ctx, "wait_probe");
  return FPCA_OK;
}

fpca_status fpca_profile_enable(fpca_ctx* ctx, int enable) {
  if (!ctx) return FPCA_E_INVALID_ARG;
  if (fpca_no_capture(ctx, "fpca_profile_enable") != FPCA_OK) return FPCA_E_UNSUPPORTED;
  prof_resolve(ctx);
  ctx->prof_totals.clear();
  ctx->prof = enable ? 1 : 0;
  return FPCA_OK;
}

int fpca_profile_count(fpca_ctx* ctx) {
  if (!ctx) return 0;
  prof_resolve(ctx);
  ctx->prof_names.clear();
  for (auto& kv : ctx->prof_totals) ctx->prof_names.push_back(kv.first);
  return (int)ctx->prof_names.size();
}

fpca_status fpca_profile_entry(fpca_ctx* ctx, int i, const char** name, double* total_ms,
                               uint64_t* launches) {
  if (!ctx || i < 0 || i >= (int)ctx->prof_names.size())
    return fpca_fail(ctx, FPCA_E_INVALID_ARG, "profile entry %d out of range", i);
  const auto& t = ctx->prof_totals[ctx->prof_names[i]];
  if (name) *name = ctx->prof_names[i].c_str();
  if (total_ms) *total_ms = t.first;
  if (launches) *launches = t.second;
  return FPCA_OK;
}

// ---------------------------------------------------------------------------
// CUDA graphs of call sequences
// ---------------------------------------------------------------------------
struct fpca_graph {
  cudaGraphExec_t exec = nullptr;
  uint64_t launches = 0;  // kernels in the graph
};

fpca_status fpca_graph_begin(fpca_ctx* ctx) {
  if (!ctx) return FPCA_E_INVALID_ARG;
  if (ctx->capturing) return fpca_fail(ctx, FPCA_E_INVALID_ARG, "a capture is already open");
  if (!ctx->stream)
    return fpca_fail(ctx, FPCA_E_UNSUPPORTED,
                     "graph capture needs a context on a created stream, not the legacy default");
  if (ctx->prof) return fpca_fail(ctx, FPCA_E_UNSUPPORTED, "kernel timing is on");
  cudaError_t e = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return fpca_fail(ctx, FPCA_E_CUDA, "begin capture: %s", cudaGetErrorString(e));
  ctx->capturing = 1;
  ctx->capture_failed = 0;
  ctx->capture_launches = ctx->launches;
  return FPCA_OK;
}

fpca_status fpca_graph_end(fpca_ctx* ctx, fpca_graph** graph) {
  if (!ctx || !graph) return FPCA_E_INVALID_ARG;
  *graph = nullptr;
  if (!ctx->capturing) return fpca_fail(ctx, FPCA_E_INVALID_ARG, "no capture is open");
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
  ctx->capturing = 0;
  const uint64_t n = ctx->launches - ctx->capture_launches;
  ctx->launches = ctx->capture_launches;  // captured, not yet run
  if (e != cudaSuccess || ctx->capture_failed || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    if (ctx->capture_failed) return FPCA_E_UNSUPPORTED;  // the refusing call set the text
    return fpca_fail(ctx, FPCA_E_CUDA, "end capture: %s", cudaGetErrorString(e));
  }
  fpca_graph* out = new fpca_graph;
  out->launches = n;
  e = cudaGraphInstantiate(&out->exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    delete out;
    return fpca_fail(ctx, FPCA_E_CUDA, "instantiate: %s", cudaGetErrorString(e));
  }
  *graph = out;
  return FPCA_OK;
}

fpca_status fpca_graph_launch(fpca_ctx* ctx, const fpca_graph* graph) {
  if (!ctx || !graph) return FPCA_E_INVALID_ARG;
  if (ctx->capturing) return fpca_fail(ctx, FPCA_E_INVALID_ARG, "a capture is open");
  fpca_prof_mark(ctx);
  const cudaError_t e = cudaGraphLaunch(graph->exec, ctx->stream);
  if (e != cudaSuccess) return fpca_fail(ctx, FPCA_E_CUDA, "graph launch: %s", cudaGetErrorString(e));
  ctx->launches += graph->launches;
  if (ctx->prof) fpca_prof_end(ctx, "graph");
  return FPCA_OK;
}

uint64_t fpca_graph_launches(const fpca_graph* graph) { return graph ? graph->launches : 0; }

void fpca_graph_destroy(fpca_graph* graph) {
  if (!graph) return;
  if (graph->exec) cudaGraphExecDestroy(graph->exec);
  delete graph;
}

fpca_status fpca_sync(fpca_ctx* ctx) {
  if (!ctx) return FPCA_E_INVALID_ARG;
  if (fpca_no_capture(ctx, "fpca_sync") != FPCA_OK) return FPCA_E_UNSUPPORTED;
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return fpca_fail(ctx, FPCA_E_CUDA, "stream: %s", cudaGetErrorString(e));
  int herr = 0;
  e = cudaMemcpy(&herr, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fpca_fail(ctx, FPCA_E_CUDA, "error word: %s", cudaGetErrorString(e));
  if (herr != DERR_NONE) {
    cudaMemset(ctx->d_err, 0, sizeof(int));
    if (herr == DERR_TIMEOUT)
      return fpca_fail(ctx, FPCA_E_TIMEOUT, "a device-side bounded wait ran out");
    if (herr == DERR_NUMERIC)
      return fpca_fail(ctx, FPCA_E_NUMERIC, "an ill-conditioned local system (fused d = 3 smoother) or a non-positive pivot (PACE scores)");
    return fpca_fail(ctx, FPCA_E_CUDA, "device-side check failed (code %d)", herr);
  }
  return FPCA_OK;
}

fpca_status fpca_bin_mean(fpca_ctx* ctx, const fpca_data* data, const fpca_grid* grid,
                          int32_t* cnt, double* w, double* v, double* v2) {
  if (!ctx) return FPCA_E_INVALID_ARG;
  fpca_prof_mark(ctx);
  if (!valid_grid(ctx, grid, 1 << 20) || !valid_data(ctx, data)) return FPCA_E_INVALID_ARG;
  if (!cnt || !w || !v) return fpca_fail(ctx, FPCA_E_INVALID_ARG, "cnt, w and v are required");
  long long P = 1;
  for (int k = 0; k < grid->d; ++k) P *= grid->m[k];
  if (P > (1 << 24)) return fpca_fail(ctx, FPCA_E_INVALID_ARG, "grid has more than 2^24 bins");
  if (data->layout == FPCA_DENSE) {
    int32_t* Ni = static_cast<int32_t*>(fpca_workspace(ctx, sizeof(int32_t) * data->n));
    if (!Ni) return fpca_fail(ctx, FPCA_E_OOM, "workspace");
    fpca_status s = launch_subject_counts_dense(ctx, data->n, (int)P, data->mask, Ni);
    if (s != FPCA_OK) return s;
    return launch_bin_mean_dense(ctx, data->n, (int)P, data->y, data->y_prec, data->mask, Ni, cnt,
                                 w, v, v2);
  }
  return launch_bin_mean_sparse(ctx, data->n, grid, data->offs, data->t,
                                static_cast<const double*>(data->y), cnt, w, v, v2);
}

fpca_status fpca_smooth_mean(fpca_ctx* ctx, const fpca_grid* grid, const int32_t* cnt,
                             const double* w, const double* v, const double* h, double* mu,
                             uint8_t* status) {
  if (!ctx) return FPCA_E_INVALID_ARG;
  fpca_prof_mark(ctx);
  if (!valid_grid(ctx, grid, 1 << 20)) return FPCA_E_INVALID_ARG;
  if (!valid_h(ctx, h, grid->d)) return FPCA_E_INVALID_ARG;
  if (!cnt || !w || !v || !mu)
    return fpca_fail(ctx, FPCA_E_INVALID_ARG, "cnt, w, v and mu are required");
  return launch_smooth_mean(ctx, grid, cnt, w, v, h, mu, status);
}

fpca_status fpca_smooth_mean_cv(fpca_ctx* ctx, const fpca_data* data, const fpca_grid* grid,
                                const int32_t* fold, int nfold, const double* h, int nh,
                                double* cv) {
  if (!ctx) return FPCA_E_INVALID_ARG;
  fpca_prof_mark(ctx);
  if (!valid_grid(ctx, grid, 1 << 20) || !valid_data(ctx, data)) return FPCA_E_INVALID_ARG;
  if (data->layout != FPCA_SPARSE)
    return fpca_fail(ctx, FPCA_E_UNSUPPORTED,
                     "mean CV is built for scattered data (list gridded observations as points)");
  if (!fold || nfold < 2 || nfold > 64)
    return fpca_fail(ctx, FPCA_E_INVALID_ARG, "fold and 2 <= nfold <= 64 are required");
  if (nh < 1 || !cv) return fpca_fail(ctx, FPCA_E_INVALID_ARG, "nh >= 1 and cv are required");
  if (!valid_h(ctx, h, nh * grid->d)) return FPCA_E_INVALID_ARG;
  return mean_cv_run(ctx, grid, data->n, data->offs, data->t, static_cast<const double*>(data->y),
                     fold, nfold, h, nh, cv);
}

fpca_status fpca_bin_cov(fpca_ctx* ctx, const fpca_data* data, const fpca_grid* grid,
                         const double* mu, int prec, int mode, const int32_t* fold, int nfold,
                         int32_t* cnt, void* w, void* v, void* q) {
  if (!ctx) return FPCA_E_INVALID_ARG;
  fpca_prof_mark(ctx);
  if (!valid_grid(ctx, grid, 4096) || !valid_data(ctx, data)) return FPCA_E_INVALID_ARG;
  if (!cnt || !w || !v) return fpca_fail(ctx, FPCA_E_INVALID_ARG, "cnt, w and v are required");
  if (mode != FPCA_COV_RESIDUAL && mode != FPCA_COV_RAW)
    return fpca_fail(ctx, FPCA_E_INVALID_ARG, "mode must be FPCA_COV_RESIDUAL or FPCA_COV_RAW");
  if (mode == FPCA_COV_RESIDUAL && !mu)
    return fpca_fail(ctx, FPCA_E_INVALID_ARG, "residual mode needs mu");
  const int P = grid_P(grid);
  if ((long long)P * P > (1ll << 31))
    return fpca_fail(ctx, FPCA_E_UNSUPPORTED,
                     "P*P = %lld exceeds the materialised-covariance limit 2^31", (long long)P * P);
  if (nfold < 0 || nfold > 64 || (nfold > 0 && !fold))
    return fpca_fail(ctx, FPCA_E_INVALID_ARG, "nfold must be 0..64 with fold ids when > 0");
  if (data->layout == FPCA_DENSE) {
    if (prec == FPCA_F32) {
      if (data->n >= (1 << 24))
        return fpca_fail(ctx, FPCA_E_UNSUPPORTED, "n >= 2^24 breaks exact FP32 pair counts");
      return launch_cov_dense_folds(ctx, data->n, P, data->y, data->y_prec, data->mask, mu, mode,
                                    fold, nfold, cnt, static_cast<float*>(w),
                                    static_cast<float*>(v), static_cast<float*>(q));
    }
    if (fold || nfold > 0 || q)
      return fpca_fail(ctx, FPCA_E_UNSUPPORTED,
                       "folds and q of gridded data are built for FPCA_F32 only");
    int32_t* Ni = nullptr;
    if (prec == FPCA_F64) {
      Ni = static_cast<int32_t*>(fpca_workspace(ctx, sizeof(int32_t) * data->n));
      if (!Ni) return fpca_fail(ctx, FPCA_E_OOM, "workspace");
      fpca_status s = launch_subject_counts_dense(ctx, data->n, P, data->mask, Ni);
      if (s != FPCA_OK) return s;
      return launch_cov_dense_f64(ctx, data->n, P, data->y, data->y_prec, data->mask, Ni, mu,
                                  mode, cnt, static_cast<double*>(w), static_cast<double*>(v));
    }
    if (prec == FPCA_BF16) {
      if (P % 128 != 0)
        return fpca_fail(ctx, FPCA_E_UNSUPPORTED,
                         "the tensor-core binning needs P a multiple of 128 (P = %d)", P);
      if (data->n >= (1 << 24))
        return fpca_fail(ctx, FPCA_E_UNSUPPORTED, "n >= 2^24 breaks exact FP32 pair counts");
      const int Kpad = ((data->n + 63) / 64) * 64;
      size_t b_ni = WsCarve::round(sizeof(int32_t) * data->n);
      size_t b_ops = WsCarve::round(sizeof(uint16_t) * 3ull * P * Kpad);
      void* ws = fpca_workspace(ctx, b_ni + b_ops + 512);
      if (!ws) return fpca_fail(ctx, FPCA_E_OOM, "workspace (%zu bytes)", b_ni + b_ops);
      WsCarve carve(ws);
      Ni = carve.take<int32_t>(data->n);
      uint16_t* ops = carve.take<uint16_t>(3ull * P * Kpad);
      fpca_status s = launch_subject_counts_dense(ctx, data->n, P, data->mask, Ni);
      if (s != FPCA_OK) return s;
      s = launch_cov_operands_bf16(ctx, data->n, P, Kpad, data->y, data->y_prec, data->mask, Ni,
                                   mu, mode, ops);
      if (s != FPCA_OK) return s;
      return launch_gram_tc(ctx, P, Kpad, ops, cnt, static_cast<float*>(w),
                            static_cast<float*>(v));
    }
    return fpca_fail(ctx, FPCA_E_UNSUPPORTED, "dense binning precision must be F64, F32 or BF16");
  }
  if (prec != FPCA_F64 && prec != FPCA_F32)
    return fpca_fail(ctx, FPCA_E_UNSUPPORTED, "sparse binning precision must be F64 or F32");
  return launch_cov_sparse(ctx, data->n, grid, data->offs, data->t,
                           static_cast<const double*>(data->y), mu, mode, fold, nfold, prec, cnt,
                           w, v, q);
}

fpca_status fpca_smooth_cov_project(fpca_ctx* ctx, const fpca_grid* grid,
                                    const fpca_covbins* bins, const double* h, int nh, int prec,
                                    const double* mu_raw, const float* omega, int l,
                                    void* gamma, uint8_t* status, float* y, double* cv) {
  if (!ctx) return FPCA_E_INVALID_ARG;
  fpca_prof_mark(ctx);
  if (!valid_grid(ctx, grid, 4096)) return FPCA_E_INVALID_ARG;
  if (!bins || !bins->cnt || !bins->w || !bins->v)
    return fpca_fail(ctx, FPCA_E_INVALID_ARG, "bins need cnt, w and v");
  if (nh < 1) return fpca_fail(ctx, FPCA_E_INVALID_ARG, "nh must be >= 1");
  if (!valid_h(ctx, h, nh * grid->d)) return FPCA_E_INVALID_ARG;
  if (prec != FPCA_F64 && prec != FPCA_F32 && prec != FPCA_F32C)
    return fpca_fail(ctx, FPCA_E_INVALID_ARG, "prec must be FPCA_F64, FPCA_F32 or FPCA_F32C");
  if ((prec == FPCA_F64) != (bins->prec == FPCA_F64))
    return fpca_fail(ctx, FPCA_E_UNSUPPORTED,
                     "FP64 smoothing needs FP64 bins and FP32 smoothing FP32 bins");
  if ((omega == nullptr) != (y == nullptr) || (omega && l < 1))
    return fpca_fail(ctx, FPCA_E_INVALID_ARG, "omega, l and y go together");
  if (cv && bins->nfold < 2)
    return fpca_fail(ctx, FPCA_E_INVALID_ARG, "cv needs bins with nfold >= 2");
  if (cv && !bins->q) return fpca_fail(ctx, FPCA_E_INVALID_ARG, "cv needs bins.q");
  if (cv && mu_raw)
    return fpca_fail(ctx, FPCA_E_UNSUPPORTED, "cv is built for residual-mode bins");
  if (!gamma && !status && !y && !cv)
    return fpca_fail(ctx, FPCA_E_INVALID_ARG, "no output requested");
  if (grid->d > 2)
    return fpca_fail(ctx, FPCA_E_UNSUPPORTED, "materialised covariance smoothing is built for d <= 2");
  const int P = grid_P(grid);
  if ((long long)P * P > (1ll << 31))
    return fpca_fail(ctx, FPCA_E_UNSUPPORTED, "P*P exceeds 2^31");
  for (int k = 0; k < grid->d; ++k)
    if (grid->m[k] > 64)
      return fpca_fail(ctx, FPCA_E_UNSUPPORTED, "covariance smoothing is built for m <= 64 per axis");
  return smooth_cov_run(ctx, grid, bins, h, nh, prec, mu_raw, omega, l, gamma, status, y, cv);
}

fpca_status fpca_rproj_eig(fpca_ctx* ctx, const fpca_grid* grid, const void* gamma,
                           int gamma_prec, const int32_t* domain, const float* omega, int l,
                           int k, int power_iters, int full, double* evals, double* evecs,
                           double* fve) {
  if (!ctx) return FPCA_E_INVALID_ARG;
  fpca_prof_mark(ctx);
  if (!valid_grid(ctx, grid, 1 << 20)) return FPCA_E_INVALID_ARG;
  if (!gamma || !evals || !evecs)
    return fpca_fail(ctx, FPCA_E_INVALID_ARG, "gamma, evals and evecs are required");
  if (gamma_prec != FPCA_F64 && gamma_prec != FPCA_F32)
    return fpca_fail(ctx, FPCA_E_INVALID_ARG, "gamma_prec must be FPCA_F64 or FPCA_F32");
  const int P = grid_P(grid);
  if (k < 1 || k > P) return fpca_fail(ctx, FPCA_E_INVALID_ARG, "k must be 1..P");
  if (full) {
    if (P > 1024) return fpca_fail(ctx, FPCA_E_UNSUPPORTED, "dense eigensolver built for P <= 1024");
  } else {
    if (!omega || l <= k || l > 64)
      return fpca_fail(ctx, FPCA_E_INVALID_ARG, "random projection needs omega and k < l <= 64");
    if (power_iters < 0 || power_iters > 16)
      return fpca_fail(ctx, FPCA_E_INVALID_ARG, "power_iters must be 0..16");
  }
  return rproj_eig_run(ctx, grid, gamma, gamma_prec, domain, omega, l, k, power_iters, full,
                       evals, evecs, fve);
}

fpca_status fpca_sigma2(fpca_ctx* ctx, const fpca_grid* grid, const int32_t* cnt, const double* w,
                        const double* v2, const double* h, const double* mu, const void* gdiag,
                        int gdiag_prec, long long gdiag_stride, const int32_t* domain,
                        double* sigma2_t, uint8_t* status, double* sigma2) {
  if (!ctx) return FPCA_E_INVALID_ARG;
  fpca_prof_mark(ctx);
  if (!valid_grid(ctx, grid, 1 << 20)) return FPCA_E_INVALID_ARG;
  if (!cnt || !w || !v2 || !h || !mu || !gdiag || !sigma2_t)
    return fpca_fail(ctx, FPCA_E_INVALID_ARG, "cnt, w, v2, h, mu, gdiag and sigma2_t are required");
  if (gdiag_prec != FPCA_F64 && gdiag_prec != FPCA_F32)
    return fpca_fail(ctx, FPCA_E_INVALID_ARG, "gdiag_prec must be FPCA_F64 or FPCA_F32");
  if (gdiag_stride < 1) return fpca_fail(ctx, FPCA_E_INVALID_ARG, "gdiag_stride must be >= 1");
  for (int k = 0; k < grid->d; ++k)
    if (!(h[k] > 0.0)) return fpca_fail(ctx, FPCA_E_INVALID_ARG, "h[%d] must be positive", k);
  return launch_sigma2(ctx, grid, cnt, w, v2, h, mu, gdiag, gdiag_prec, gdiag_stride, domain,
                       sigma2_t, status, sigma2);
}

}  // extern "C"
