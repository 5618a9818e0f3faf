// Arithmetic-throughput probes: the measured FP32 and FP64 FMA peaks that the
// roofline fractions of the ALU-bound kernels (the moment sweeps, the FP64
// solves) are quoted against.  Each thread runs 8 independent FMA chains (FP32:
// paired, two FMAs per instruction) long enough that issue and the FMA pipe,
// not latency, bind; the caller times the launch.
#include "fpca_internal.cuh"

namespace {

constexpr int kProbeThreads = 256;

__global__ void __launch_bounds__(kProbeThreads) k_probe_fp32(int iters, float* sink) {
  float2 a[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = make_float2(1e-3f * (threadIdx.x + j), 1e-3f * (blockIdx.x + j));
  const float2 b = make_float2(0.9999999f, 1.0000001f), c = make_float2(1e-7f, -1e-7f);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r)
#pragma unroll
      for (int j = 0; j < 8; ++j) a[j] = __ffma2_rn(a[j], b, c);
  }
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += a[j].x + a[j].y;
  if (s == 1234.5678f) sink[0] = s;  // keeps the chains live
}

__global__ void __launch_bounds__(kProbeThreads) k_probe_fp64(int iters, double* sink) {
  double a[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = 1e-3 * (threadIdx.x + j + blockIdx.x);
  const double b = 0.9999999999, c = 1e-12;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 16; ++r)
#pragma unroll
      for (int j = 0; j < 8; ++j) a[j] = fma(a[j], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += a[j];
  if (s == 1234.5678) sink[0] = s;
}

}  // namespace

extern "C" fpca_status fpca_alu_probe(fpca_ctx* ctx, int fp64, int blocks, int iters,
                                      double* flops) {
  if (!ctx) return FPCA_E_INVALID_ARG;
  if (blocks < 1 || iters < 1 || !flops)
    return fpca_fail(ctx, FPCA_E_INVALID_ARG, "blocks >= 1, iters >= 1 and flops are required");
  void* sink = fpca_workspace(ctx, 64);
  if (!sink) return fpca_fail(ctx, FPCA_E_OOM, "workspace");
  fpca_prof_mark(ctx);
  const double per_thread = (double)iters * 16.0 * 8.0 * (fp64 ? 2.0 : 4.0);
  *flops = per_thread * kProbeThreads * (double)blocks;
  if (fp64)
    k_probe_fp64<<<blocks, kProbeThreads, 0, ctx->stream>>>(iters, static_cast<double*>(sink));
  else
    k_probe_fp32<<<blocks, kProbeThreads, 0, ctx->stream>>>(iters, static_cast<float*>(sink));
  FPCA_LAUNCHED(ctx, fp64 ? "probe_fp64" : "probe_fp32");
  return FPCA_OK;
}
