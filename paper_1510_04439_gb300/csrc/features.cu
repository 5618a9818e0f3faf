// The 32-number dataset summary fed to the bandwidth network.
//
// It describes what drives the optimal bandwidths of Eq. (2.3)-(2.4):
// sample size and sampling density (n, N_i, bin occupancy), noise against
// signal, and the roughness of the binned mean and covariance.  Sums are
// reduced in FP64 (atomics into a small accumulator block), and one thread
// turns them into features:
//   0 d; 1 log n; 2 log mean N_i; 3 std/mean N_i; 4 log min N_i; 5 log max N_i;
//   6 log(1 + mean bin count); 7 var/mean^2 of bin counts; 8 their skewness;
//   9 fraction of empty bins; 10 log mean within-bin variance V2/W - (V/W)^2;
//   11 log variance of the binned mean mb = V/W; 12-14 log mean squared 2nd
//   difference of mb along axes 0..2 minus feature 11; 15-16 the same with
//   1st differences along axes 0..1; 17 zero; 18 log roughness of the
//   covariance raw means g = V/W along s_1, 19 along the (s_1, t_1)
//   diagonal (both relative to var g); 20 log(1 + mean pair count);
//   21 fraction of covariance bins with a pair; 22-24 log 1/M_k; 25-31 zero.
#include <cmath>

#include "fpca_internal.cuh"

namespace {

// accumulator layout (doubles)
enum {
  A_N = 0, A_N2, A_NMIN, A_NMAX, A_NSUB,                     // subjects
  A_C1, A_C2, A_C3, A_EMPTY, A_SB, A_MB, A_MB2, A_NE,        // mean bins
  A_R2 = 13,   // 3 sums + 3 counts  (13..18)
  A_R1 = 19,   // 2 sums + 2 counts  (19..22)
  A_G1 = 23, A_G2, A_GN, A_RS, A_RSN, A_RD, A_RDN, A_CC, A_CPOS,  // covariance
  A_COUNT = 32
};

__device__ __forceinline__ void atomic_min_d(double* a, double v) {
  unsigned long long* p = reinterpret_cast<unsigned long long*>(a);
  unsigned long long old = *p;
  while (v < __longlong_as_double(old)) {
    const unsigned long long prev = atomicCAS(p, old, __double_as_longlong(v));
    if (prev == old) break;
    old = prev;
  }
}
__device__ __forceinline__ void atomic_max_d(double* a, double v) {
  unsigned long long* p = reinterpret_cast<unsigned long long*>(a);
  unsigned long long old = *p;
  while (v > __longlong_as_double(old)) {
    const unsigned long long prev = atomicCAS(p, old, __double_as_longlong(v));
    if (prev == old) break;
    old = prev;
  }
}

__global__ void k_feat_init(double* acc) {
  const int i = threadIdx.x;
  if (i < A_COUNT) acc[i] = (i == A_NMIN) ? 1e300 : (i == A_NMAX ? -1e300 : 0.0);
}

// per-subject counts: from mask rows (dense, computed by the caller) or offsets
__global__ void k_feat_subjects(int n, const int32_t* __restrict__ Ni, const int64_t* __restrict__ offs,
                                double* acc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double N = Ni ? (double)Ni[i] : (double)(offs[i + 1] - offs[i]);
  atomicAdd(acc + A_N, N);
  atomicAdd(acc + A_N2, N * N);
  atomicAdd(acc + A_NSUB, 1.0);
  atomic_min_d(acc + A_NMIN, N);
  atomic_max_d(acc + A_NMAX, N);
}

struct GridInfo {
  int d;
  int m[3];
  int stride[3];  // flat step of each axis
};

__device__ __forceinline__ bool bin_mean_at(const double* w, const double* v, int b, double& mb) {
  if (!(w[b] > 0.0)) return false;
  mb = v[b] / w[b];
  return true;
}

__global__ void k_feat_bins(int P, GridInfo gi, const int32_t* __restrict__ cnt,
                            const double* __restrict__ w, const double* __restrict__ v,
                            const double* __restrict__ v2, double* acc) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= P) return;
  const double c = (double)cnt[b];
  atomicAdd(acc + A_C1, c);
  atomicAdd(acc + A_C2, c * c);
  atomicAdd(acc + A_C3, c * c * c);
  if (cnt[b] == 0) atomicAdd(acc + A_EMPTY, 1.0);
  double mb;
  if (!bin_mean_at(w, v, b, mb)) return;
  const double sb = v2 ? v2[b] / w[b] - mb * mb : 0.0;
  atomicAdd(acc + A_SB, fmax(sb, 0.0));
  atomicAdd(acc + A_MB, mb);
  atomicAdd(acc + A_MB2, mb * mb);
  atomicAdd(acc + A_NE, 1.0);
  int coord[3];
  {
    int rem = b;
    for (int k = gi.d - 1; k >= 0; --k) {
      coord[k] = rem % gi.m[k];
      rem /= gi.m[k];
    }
  }
  for (int k = 0; k < gi.d; ++k) {
    double m1, m2;
    if (k < 2 && coord[k] + 1 < gi.m[k] && bin_mean_at(w, v, b + gi.stride[k], m1)) {
      atomicAdd(acc + A_R1 + k, (m1 - mb) * (m1 - mb));
      atomicAdd(acc + A_R1 + 2 + k, 1.0);
    }
    if (coord[k] + 2 < gi.m[k] && bin_mean_at(w, v, b + gi.stride[k], m1) &&
        bin_mean_at(w, v, b + 2 * gi.stride[k], m2)) {
      const double d2 = m2 - 2.0 * m1 + mb;
      atomicAdd(acc + A_R2 + k, d2 * d2);
      atomicAdd(acc + A_R2 + 3 + k, 1.0);
    }
  }
}

// Covariance-bin sums over the pooled fold slices (F slices of PP entries).
template <typename T>
__global__ void k_feat_cov(long long PP, int P, int s0, int F, const int32_t* __restrict__ C,
                           const T* __restrict__ W, const T* __restrict__ V, double* acc) {
  __shared__ double red[9][8];
  double loc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  auto pooled = [&](long long e, double& w, double& v) {
    w = 0.0;
    v = 0.0;
    for (int f = 0; f < F; ++f) {
      w += (double)W[f * PP + e];
      v += (double)V[f * PP + e];
    }
  };
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < PP;
       e += (long long)gridDim.x * blockDim.x) {
    int cc = 0;
    for (int f = 0; f < F; ++f) cc += C[f * PP + e];
    loc[7] += (double)cc;
    if (cc > 0) loc[8] += 1.0;
    double wv, vv;
    pooled(e, wv, vv);
    if (!(wv > 0.0)) continue;
    const double g = vv / wv;
    loc[0] += g;
    loc[1] += g * g;
    loc[2] += 1.0;
    const int p = (int)(e / P), q = (int)(e - (long long)p * P);
    if (p + s0 < P) {
      const long long e1 = e + (long long)s0 * P;
      double w1, v1;
      pooled(e1, w1, v1);
      if (w1 > 0.0) {
        const double dd = v1 / w1 - g;
        loc[3] += dd * dd;
        loc[4] += 1.0;
      }
      if (q + s0 < P) {
        const long long e2 = e1 + s0;
        double w2, v2;
        pooled(e2, w2, v2);
        if (w2 > 0.0) {
          const double dd = v2 / w2 - g;
          loc[5] += dd * dd;
          loc[6] += 1.0;
        }
      }
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int j = 0; j < 9; ++j) {
    double x = loc[j];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) red[j][wid] = x;
  }
  __syncthreads();
  if (threadIdx.x < 9) {
    double x = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) x += red[threadIdx.x][k];
    atomicAdd(acc + A_G1 + threadIdx.x, x);
  }
}

__global__ void k_feat_finish(GridInfo gi, int P, long long PP, const double* __restrict__ acc,
                              float* __restrict__ feat) {
  if (threadIdx.x != 0) return;
  const double eps = 1e-12;
  double f[32];
  for (int i = 0; i < 32; ++i) f[i] = 0.0;
  const double ns = acc[A_NSUB];
  const double mN = acc[A_N] / ns;
  const double vN = fmax(acc[A_N2] / ns - mN * mN, 0.0);
  f[0] = gi.d;
  f[1] = log(ns);
  f[2] = log(fmax(mN, eps));
  f[3] = sqrt(vN) / fmax(mN, eps);
  f[4] = log(fmax(acc[A_NMIN], 1.0));
  f[5] = log(fmax(acc[A_NMAX], 1.0));
  const double mc = acc[A_C1] / P;
  const double ec2 = acc[A_C2] / P, ec3 = acc[A_C3] / P;
  const double vc = fmax(ec2 - mc * mc, 0.0);
  f[6] = log1p(mc);
  f[7] = mc > 0.0 ? vc / (mc * mc) : 0.0;
  const double sd = sqrt(vc);
  f[8] = sd > 0.0 ? (ec3 - 3.0 * mc * ec2 + 2.0 * mc * mc * mc) / (sd * sd * sd) : 0.0;
  f[9] = acc[A_EMPTY] / P;
  const double ne = acc[A_NE];
  f[10] = ne > 0.0 ? log(acc[A_SB] / ne + eps) : 0.0;
  const double mmb = ne > 0.0 ? acc[A_MB] / ne : 0.0;
  const double varmb = ne > 0.0 ? fmax(acc[A_MB2] / ne - mmb * mmb, 0.0) : 0.0;
  f[11] = log(varmb + eps);
  for (int k = 0; k < 3; ++k)
    if (k < gi.d) {
      const double cntk = acc[A_R2 + 3 + k];
      f[12 + k] = log((cntk > 0.0 ? acc[A_R2 + k] / cntk : 0.0) + eps) - f[11];
    }
  for (int k = 0; k < 2; ++k)
    if (k < gi.d) {
      const double cntk = acc[A_R1 + 2 + k];
      f[15 + k] = log((cntk > 0.0 ? acc[A_R1 + k] / cntk : 0.0) + eps) - f[11];
    }
  const double gn = acc[A_GN];
  const double mg = gn > 0.0 ? acc[A_G1] / gn : 0.0;
  const double varg = gn > 0.0 ? fmax(acc[A_G2] / gn - mg * mg, 0.0) : 0.0;
  const double lvg = log(varg + eps);
  if (P > gi.stride[0]) {
    f[18] = log((acc[A_RSN] > 0.0 ? acc[A_RS] / acc[A_RSN] : 0.0) + eps) - lvg;
    f[19] = log((acc[A_RDN] > 0.0 ? acc[A_RD] / acc[A_RDN] : 0.0) + eps) - lvg;
  }
  f[20] = log1p(acc[A_CC] / (double)PP);
  f[21] = acc[A_CPOS] / (double)PP;
  for (int k = 0; k < 3; ++k)
    if (k < gi.d) f[22 + k] = log(1.0 / gi.m[k]);
  for (int i = 0; i < 32; ++i) feat[i] = (float)f[i];
}

}  // namespace

extern "C" fpca_status fpca_bw_features(fpca_ctx* ctx, const fpca_data* data,
                                        const fpca_grid* grid, const int32_t* cnt,
                                        const double* w, const double* v, const double* v2,
                                        const fpca_covbins* bins, float* feat) {
  if (!ctx) return FPCA_E_INVALID_ARG;
  fpca_prof_mark(ctx);
  if (!data || !grid || !cnt || !w || !v || !bins || !bins->cnt || !bins->w || !bins->v || !feat)
    return fpca_fail(ctx, FPCA_E_INVALID_ARG, "data, grid, mean bins, covariance bins and feat are required");
  if (grid->d < 1 || grid->d > 3) return fpca_fail(ctx, FPCA_E_INVALID_ARG, "grid.d must be 1..3");
  if (data->n < 1) return fpca_fail(ctx, FPCA_E_INVALID_ARG, "data.n must be >= 1");
  const int P = grid_P(grid);
  const long long PP = (long long)P * P;
  const int F = bins->nfold > 0 ? bins->nfold : 1;
  GridInfo gi{};
  gi.d = grid->d;
  for (int k = 0; k < 3; ++k) gi.m[k] = k < grid->d ? grid->m[k] : 1;
  for (int k = 0; k < 3; ++k) {
    int st = 1;
    for (int j = k + 1; j < grid->d; ++j) st *= grid->m[j];
    gi.stride[k] = st;
  }
  const size_t need = WsCarve::round(sizeof(double) * A_COUNT) + WsCarve::round(sizeof(int32_t) * data->n) + 1024;
  void* ws = fpca_workspace(ctx, need);
  if (!ws) return fpca_fail(ctx, FPCA_E_OOM, "workspace");
  WsCarve carve(ws);
  double* acc = carve.take<double>(A_COUNT);
  int32_t* Ni = carve.take<int32_t>(data->n);
  k_feat_init<<<1, 64, 0, ctx->stream>>>(acc);
  FPCA_LAUNCHED(ctx, "feat_init");
  if (data->layout == FPCA_DENSE) {
    fpca_status s = launch_subject_counts_dense(ctx, data->n, P, data->mask, Ni);
    if (s != FPCA_OK) return s;
    k_feat_subjects<<<(data->n + 255) / 256, 256, 0, ctx->stream>>>(data->n, Ni, nullptr, acc);
  } else {
    k_feat_subjects<<<(data->n + 255) / 256, 256, 0, ctx->stream>>>(data->n, nullptr, data->offs, acc);
  }
  FPCA_LAUNCHED(ctx, "feat_subjects");
  k_feat_bins<<<(P + 255) / 256, 256, 0, ctx->stream>>>(P, gi, cnt, w, v, v2, acc);
  FPCA_LAUNCHED(ctx, "feat_bins");
  const int nb = (int)std::min<long long>((PP + 255) / 256, 4096);
  if (bins->prec == FPCA_F64)
    k_feat_cov<double><<<nb, 256, 0, ctx->stream>>>(PP, P, gi.stride[0], F, bins->cnt,
                                                    static_cast<const double*>(bins->w),
                                                    static_cast<const double*>(bins->v), acc);
  else
    k_feat_cov<float><<<nb, 256, 0, ctx->stream>>>(PP, P, gi.stride[0], F, bins->cnt,
                                                   static_cast<const float*>(bins->w),
                                                   static_cast<const float*>(bins->v), acc);
  FPCA_LAUNCHED(ctx, "feat_cov");
  k_feat_finish<<<1, 32, 0, ctx->stream>>>(gi, P, PP, acc, feat);
  FPCA_LAUNCHED(ctx, "feat_finish");
  return FPCA_OK;
}
