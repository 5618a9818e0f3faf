// Bandwidth-proposal network: 32 -> 256 -> 256 -> 256 -> 6 with exact GELU,
// FP16 weights (the FP32 master copy is rounded on load) and FP32
// accumulation.  Forward, manual backward of the masked squared error, and
// AdamW, all on the device.
//
// The paper chooses bandwidths by cross-validation over candidates (Section
// 3.3); this network proposes the CV-optimal log bandwidths from a summary of
// the binned data, so that one smoothing pass (plus a CV check) can stand in
// for a grid.
//
// Parameter vector: for each layer, W (fan_in x fan_out, row-major) then b.
#include <cuda_fp16.h>

#include <cstdio>
#include <cstring>
#include <vector>

#include "fpca_internal.cuh"

namespace {

constexpr int NLAYER = 4;
__host__ __device__ constexpr int layer_in(int l) { return l == 0 ? 32 : 256; }
__host__ __device__ constexpr int layer_out(int l) { return l == 3 ? 6 : 256; }
__host__ __device__ constexpr long long layer_off(int l) {
  return l == 0 ? 0 : layer_off(l - 1) + (long long)layer_in(l - 1) * layer_out(l - 1) + layer_out(l - 1);
}
constexpr long long kParamCount = layer_off(NLAYER);

__device__ __forceinline__ float as_fp16(float w) { return __half2float(__float2half_rn(w)); }

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * expf(-0.5f * z * z) * 0.3989422804014327f;
}

// Epilogues of the small GEMM.
enum { EPI_STORE = 0, EPI_BIAS_GELU = 1, EPI_BIAS = 2, EPI_GELU_GRAD = 3 };

// C[m][n] = sum_k A(m,k) B(k,n); A(m,k) = TA ? A[k*lda+m] : A[m*lda+k],
// B(k,n) = TB ? B[n*ldb+k] : B[k*ldb+n]; B rounded to FP16 when RB.
// 32 x 32 output tile per block of 256 threads (4 outputs each).
template <bool TA, bool TB, bool RB>
__global__ void __launch_bounds__(256)
    k_gemm_small(int M, int N, int K, const float* __restrict__ A, int lda,
                 const float* __restrict__ B, int ldb, float* __restrict__ C, int ldc, int epi,
                 const float* __restrict__ bias, const float* __restrict__ aux,
                 float* __restrict__ C2) {
  __shared__ float As[32][33], Bs[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // ty 0..7
  const int m0 = blockIdx.y * 32, n0 = blockIdx.x * 32;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int k0 = 0; k0 < K; k0 += 32) {
    for (int r = ty; r < 32; r += 8) {
      const int m = m0 + r, k = k0 + tx;
      As[r][tx] = (m < M && k < K) ? (TA ? A[(long long)k * lda + m] : A[(long long)m * lda + k]) : 0.f;
      const int kk = k0 + r, n = n0 + tx;
      float b = 0.f;
      if (kk < K && n < N) b = TB ? B[(long long)n * ldb + kk] : B[(long long)kk * ldb + n];
      Bs[r][tx] = RB ? as_fp16(b) : b;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
      const float bv = Bs[k][tx];
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[j] = fmaf(As[ty + 8 * j][k], bv, acc[j]);
    }
    __syncthreads();
  }
  const int n = n0 + tx;
  if (n >= N) return;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int m = m0 + ty + 8 * j;
    if (m >= M) continue;
    float v = acc[j];
    const long long o = (long long)m * ldc + n;
    if (epi == EPI_BIAS_GELU) {
      v += bias[n];
      C[o] = v;           // pre-activation
      C2[o] = gelu(v);    // activation
    } else if (epi == EPI_BIAS) {
      C[o] = v + bias[n];
    } else if (epi == EPI_GELU_GRAD) {
      C[o] = v * gelu_grad(aux[o]);
    } else {
      C[o] = v;
    }
  }
}

// column sums: out[n] = sum_m X[m][n]
__global__ void k_colsum(int M, int N, const float* __restrict__ X, float* __restrict__ out) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int m = 0; m < M; ++m) s += X[(long long)m * N + n];
  out[n] = s;
}

// dO = 2 M (O - Y) / sum M and the masked loss, one block.
__global__ void k_loss_grad(int Bn, const float* __restrict__ O, const float* __restrict__ Y,
                            const uint8_t* __restrict__ Mk, float* __restrict__ dO,
                            float* __restrict__ loss) {
  __shared__ float rs[256], rm[256];
  float s = 0.f, msum = 0.f;
  const int n = Bn * 6;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const float mk = Mk[e] ? 1.f : 0.f;
    const float d = O[e] - Y[e];
    s += mk * d * d;
    msum += mk;
  }
  rs[threadIdx.x] = s;
  rm[threadIdx.x] = msum;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) {
      rs[threadIdx.x] += rs[threadIdx.x + k];
      rm[threadIdx.x] += rm[threadIdx.x + k];
    }
    __syncthreads();
  }
  const float denom = fmaxf(rm[0], 1.f);
  for (int e = threadIdx.x; e < n; e += blockDim.x)
    dO[e] = Mk[e] ? 2.f * (O[e] - Y[e]) / denom : 0.f;
  if (threadIdx.x == 0 && loss) *loss = rs[0] / denom;
}

// AdamW with bias correction; decoupled weight decay on every parameter.
__global__ void k_adamw(long long n, float* __restrict__ th, float* __restrict__ m,
                        float* __restrict__ v, const float* __restrict__ g, float lr, float wd,
                        float bc1, float bc2) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = 0.9f * m[i] + 0.1f * gi;
  const float vi = 0.999f * v[i] + 0.001f * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float mh = mi / bc1, vh = vi / bc2;
  th[i] -= lr * (mh / (sqrtf(vh) + 1e-8f) + wd * th[i]);
}

template <bool TA, bool TB, bool RB>
fpca_status gemm(fpca_ctx* ctx, int M, int N, int K, const float* A, int lda, const float* B,
                 int ldb, float* C, int ldc, int epi, const float* bias, const float* aux,
                 float* C2) {
  dim3 grid((N + 31) / 32, (M + 31) / 32);
  k_gemm_small<TA, TB, RB><<<grid, 256, 0, ctx->stream>>>(M, N, K, A, lda, B, ldb, C, ldc, epi,
                                                          bias, aux, C2);
  FPCA_LAUNCHED(ctx, "mlp_gemm");
  return FPCA_OK;
}

struct MlpWork {
  float* Z[3];  // pre-activations of the hidden layers (B x 256)
  float* H[3];  // activations
  float* O;     // outputs (B x 6)
  float* dA;    // B x 256
  float* dB;    // B x 256
  float* grad;  // param count
};

fpca_status mlp_workspace(fpca_ctx* ctx, int Bn, MlpWork& w) {
  const size_t act = (size_t)Bn * 256;
  const size_t need = 8 * WsCarve::round(sizeof(float) * act) + WsCarve::round(sizeof(float) * Bn * 6) +
                      WsCarve::round(sizeof(float) * kParamCount) + 4096;
  void* ws = fpca_workspace(ctx, need);
  if (!ws) return fpca_fail(ctx, FPCA_E_OOM, "workspace (%zu bytes)", need);
  WsCarve c(ws);
  for (int l = 0; l < 3; ++l) {
    w.Z[l] = c.take<float>(act);
    w.H[l] = c.take<float>(act);
  }
  w.O = c.take<float>((size_t)Bn * 6);
  w.dA = c.take<float>(act);
  w.dB = c.take<float>(act);
  w.grad = c.take<float>(kParamCount);
  return FPCA_OK;
}

fpca_status mlp_forward(fpca_ctx* ctx, const float* th, const float* X, int Bn, MlpWork& w,
                        float* out) {
  const float* h = X;
  for (int l = 0; l < NLAYER; ++l) {
    const int fi = layer_in(l), fo = layer_out(l);
    const float* W = th + layer_off(l);
    const float* b = W + (long long)fi * fo;
    fpca_status s;
    if (l < NLAYER - 1) {
      s = gemm<false, false, true>(ctx, Bn, fo, fi, h, fi, W, fo, w.Z[l], fo, EPI_BIAS_GELU, b,
                                   nullptr, w.H[l]);
      h = w.H[l];
    } else {
      s = gemm<false, false, true>(ctx, Bn, fo, fi, h, fi, W, fo, out, fo, EPI_BIAS, b, nullptr,
                                   nullptr);
    }
    if (s != FPCA_OK) return s;
  }
  return FPCA_OK;
}

// splitmix64 (Steele, Lea and Flood 2014): the finaliser applied to a counter.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// He-normal initial weights N(0, 2 / fan_in) and zero biases.  Parameter e draws
// its normal value by the Box-Muller transform of two uniforms in (0, 1] taken
// from the counter (seed, e): the result depends only on the seed.
__global__ void k_mlp_init(uint64_t seed, float* __restrict__ params) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= kParamCount) return;
  int l = 0;
  while (l + 1 < NLAYER && e >= layer_off(l + 1)) ++l;
  const long long r = e - layer_off(l);
  const int fi = layer_in(l), fo = layer_out(l);
  if (r >= (long long)fi * fo) {
    params[e] = 0.f;  // bias
    return;
  }
  const uint64_t a = splitmix64(seed * 0x2545F4914F6CDD1Dull + 2ull * (uint64_t)e);
  const uint64_t b = splitmix64(seed * 0x2545F4914F6CDD1Dull + 2ull * (uint64_t)e + 1ull);
  const double u1 = ((double)(a >> 11) + 1.0) * 0x1.0p-53;  // (0, 1]
  const double u2 = (double)(b >> 11) * 0x1.0p-53;          // [0, 1)
  const double z = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
  params[e] = (float)(z * sqrt(2.0 / (double)fi));
}

// File layout of fpca_bw_mlp_io: magic, parameter count, the parameters, the
// 32 feature means and the 32 feature scales, all little-endian.
constexpr char kMlpMagic[8] = {'F', 'P', 'C', 'A', 'B', 'W', '0', '1'};

}  // namespace

extern "C" {

int64_t fpca_bw_param_count(void) { return kParamCount; }

fpca_status fpca_bw_mlp_init(fpca_ctx* ctx, uint64_t seed, float* params) {
  if (!ctx) return FPCA_E_INVALID_ARG;
  fpca_prof_mark(ctx);
  if (!params) return fpca_fail(ctx, FPCA_E_INVALID_ARG, "params is NULL");
  k_mlp_init<<<(int)((kParamCount + 255) / 256), 256, 0, ctx->stream>>>(seed, params);
  FPCA_LAUNCHED(ctx, "mlp_init");
  return FPCA_OK;
}

fpca_status fpca_bw_mlp_io(fpca_ctx* ctx, float* params, float* feat_mu, float* feat_sd,
                           const char* path, int save) {
  if (!ctx) return FPCA_E_INVALID_ARG;
  if (!params || !path) return fpca_fail(ctx, FPCA_E_INVALID_ARG, "params and path are required");
  if (fpca_no_capture(ctx, "fpca_bw_mlp_io") != FPCA_OK) return FPCA_E_UNSUPPORTED;
  std::vector<float> buf((size_t)kParamCount + 64, 0.f);
  const size_t nbytes = sizeof(float) * buf.size();
  if (save) {
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess)
      return fpca_check_launch(ctx, "mlp_io: stream");
    cudaError_t e = cudaMemcpy(buf.data(), params, sizeof(float) * kParamCount,
                               cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && feat_mu)
      e = cudaMemcpy(buf.data() + kParamCount, feat_mu, 32 * sizeof(float), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && feat_sd)
      e = cudaMemcpy(buf.data() + kParamCount + 32, feat_sd, 32 * sizeof(float),
                     cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fpca_fail(ctx, FPCA_E_CUDA, "mlp_io: %s", cudaGetErrorString(e));
    FILE* f = std::fopen(path, "wb");
    if (!f) return fpca_fail(ctx, FPCA_E_INVALID_ARG, "mlp_io: cannot write %s", path);
    const int64_t count = kParamCount;
    const bool ok = std::fwrite(kMlpMagic, 1, 8, f) == 8 && std::fwrite(&count, 8, 1, f) == 1 &&
                    std::fwrite(buf.data(), 1, nbytes, f) == nbytes;
    if (std::fclose(f) != 0 || !ok)
      return fpca_fail(ctx, FPCA_E_INVALID_ARG, "mlp_io: short write to %s", path);
    return FPCA_OK;
  }
  FILE* f = std::fopen(path, "rb");
  if (!f) return fpca_fail(ctx, FPCA_E_INVALID_ARG, "mlp_io: cannot read %s", path);
  char magic[8];
  int64_t count = 0;
  const bool head = std::fread(magic, 1, 8, f) == 8 && std::fread(&count, 8, 1, f) == 1;
  const bool body = head && std::memcmp(magic, kMlpMagic, 8) == 0 && count == kParamCount &&
                    std::fread(buf.data(), 1, nbytes, f) == nbytes;
  std::fclose(f);
  if (!body)
    return fpca_fail(ctx, FPCA_E_INVALID_ARG,
                     "mlp_io: %s is not a saved network of %lld parameters", path,
                     (long long)kParamCount);
  cudaError_t e = cudaMemcpyAsync(params, buf.data(), sizeof(float) * kParamCount,
                                  cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess && feat_mu)
    e = cudaMemcpyAsync(feat_mu, buf.data() + kParamCount, 32 * sizeof(float),
                        cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess && feat_sd)
    e = cudaMemcpyAsync(feat_sd, buf.data() + kParamCount + 32, 32 * sizeof(float),
                        cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);  // buf is a host temporary
  if (e != cudaSuccess) return fpca_fail(ctx, FPCA_E_CUDA, "mlp_io: %s", cudaGetErrorString(e));
  return FPCA_OK;
}

fpca_status fpca_bw_predict(fpca_ctx* ctx, const float* params, const float* feat, int B,
                            float* out) {
  if (!ctx) return FPCA_E_INVALID_ARG;
  fpca_prof_mark(ctx);
  if (!params || !feat || !out || B < 1)
    return fpca_fail(ctx, FPCA_E_INVALID_ARG, "params, feat, out and B >= 1 are required");
  MlpWork w;
  fpca_status s = mlp_workspace(ctx, B, w);
  if (s != FPCA_OK) return s;
  return mlp_forward(ctx, params, feat, B, w, out);
}

fpca_status fpca_bw_train_step(fpca_ctx* ctx, float* params, float* adam_m, float* adam_v,
                               int step, const float* feat, const float* target,
                               const uint8_t* tmask, int B, float lr, float wd, float* loss,
                               float* grad_out) {
  if (!ctx) return FPCA_E_INVALID_ARG;
  fpca_prof_mark(ctx);
  if (!params || !feat || !target || !tmask || B < 1)
    return fpca_fail(ctx, FPCA_E_INVALID_ARG, "params, feat, target, tmask and B >= 1 are required");
  if (step >= 1 && (!adam_m || !adam_v))
    return fpca_fail(ctx, FPCA_E_INVALID_ARG, "an update step needs the AdamW moments");
  MlpWork w;
  fpca_status s = mlp_workspace(ctx, B, w);
  if (s != FPCA_OK) return s;
  s = mlp_forward(ctx, params, feat, B, w, w.O);
  if (s != FPCA_OK) return s;
  // dO into dA (B x 6)
  k_loss_grad<<<1, 256, 0, ctx->stream>>>(B, w.O, target, tmask, w.dA, loss);
  FPCA_LAUNCHED(ctx, "mlp_loss");
  float* g = grad_out ? grad_out : w.grad;
  float* dcur = w.dA;   // gradient w.r.t. the current layer's pre-activation
  float* dnext = w.dB;
  for (int l = NLAYER - 1; l >= 0; --l) {
    const int fi = layer_in(l), fo = layer_out(l);
    const float* W = params + layer_off(l);
    float* gW = g + layer_off(l);
    float* gb = gW + (long long)fi * fo;
    const float* hin = l == 0 ? feat : w.H[l - 1];
    // gW = hin' dcur (fi x fo), gb = column sums of dcur
    s = gemm<true, false, false>(ctx, fi, fo, B, hin, fi, dcur, fo, gW, fo, EPI_STORE, nullptr,
                                 nullptr, nullptr);
    if (s != FPCA_OK) return s;
    k_colsum<<<(fo + 127) / 128, 128, 0, ctx->stream>>>(B, fo, dcur, gb);
    FPCA_LAUNCHED(ctx, "mlp_colsum");
    if (l > 0) {
      // d(previous pre-activation) = (dcur W') * gelu'(Z_{l-1})
      s = gemm<false, true, true>(ctx, B, fi, fo, dcur, fo, W, fo, dnext, fi, EPI_GELU_GRAD,
                                  nullptr, w.Z[l - 1], nullptr);
      if (s != FPCA_OK) return s;
      float* t = dcur;
      dcur = dnext;
      dnext = t;
    }
  }
  if (step >= 1) {
    const float bc1 = 1.f - powf(0.9f, (float)step), bc2 = 1.f - powf(0.999f, (float)step);
    k_adamw<<<(int)((kParamCount + 255) / 256), 256, 0, ctx->stream>>>(kParamCount, params, adam_m,
                                                                     adam_v, g, lr, wd, bc1, bc2);
    FPCA_LAUNCHED(ctx, "mlp_adamw");
  }
  return FPCA_OK;
}

}  // extern "C"
