// Principal component scores and reconstruction (Section 2.1).
//
// PACE, Eq. (2.7): A_i = Lambda Phi_i' (Phi_i Lambda Phi_i' + sigma^2 I)^{-1} Y_i^C.
// By the push-through identity Lambda Phi' (Phi Lambda Phi' + sigma^2 I)^{-1} =
// (sigma^2 Lambda^{-1} + Phi'Phi)^{-1} Phi', each subject needs only the L x L
// system (sigma^2 Lambda^{-1} + Phi_i'Phi_i) A_i = Phi_i' Y_i^C instead of an
// N_i x N_i one: one warp accumulates Phi_i'Phi_i and Phi_i'Y_i^C over the
// subject's observations (in chunks of 32 staged in shared memory), one lane
// solves by Cholesky in FP64.  Functions known on the grid are read at the bin
// of each observation (Section 3.2 binning).
//
// Scores by integration (dense data): A_il = dV sum over observed nodes of
// (Y_i - mu) phi_l; reconstruction X_i = mu + sum_l A_il phi_l at the nodes.
#include <cmath>

#include "fpca_internal.cuh"

namespace {

constexpr int SC_LMAX = 16;
constexpr int SC_WARPS = 4;  // warps per block

struct ScGrid {
  int d, m[3], P;
};

__device__ __forceinline__ int sc_bin(const ScGrid& g, const double* t) {
  int b = 0;
  for (int k = 0; k < g.d; ++k) {
    const double x = floor(__dmul_rn(t[k], (double)g.m[k]));
    b = b * g.m[k] + (int)fmin(fmax(x, 0.0), (double)(g.m[k] - 1));
  }
  return b;
}

// layout 0: dense y (n x P, FP32/FP64 per yprec) with mask (or NULL);
// layout 1: scattered offs / t / y (FP64).
__global__ void __launch_bounds__(32 * SC_WARPS, 4)
    k_scores_pace(ScGrid g, int n, int layout, const void* __restrict__ y, int yprec,
                  const uint8_t* __restrict__ mask, const int64_t* __restrict__ offs,
                  const double* __restrict__ t, const double* __restrict__ mu,
                  const double* __restrict__ lam, const double* __restrict__ phi, int L,
                  const double* __restrict__ sigma2p, double* __restrict__ scores,
                  int* __restrict__ err) {
  __shared__ double rows[SC_WARPS][32][SC_LMAX + 1];  // phi rows, then the residual
  __shared__ double sysA[SC_WARPS][SC_LMAX][SC_LMAX + 1];
  __shared__ double sysb[SC_WARPS][SC_LMAX];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int NE = L * (L + 1) / 2;
  for (int i = blockIdx.x * SC_WARPS + warp; i < n; i += gridDim.x * SC_WARPS) {
    // Upper-triangle entries e = lane + 32 q (row-major) of Phi_i' Phi_i held by this lane.
    int er[5], ec[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      int r = 0, rem = lane + 32 * q;
      while (r < L && rem >= L - r) {
        rem -= L - r;
        ++r;
      }
      er[q] = r;  // r == L: no entry
      ec[q] = r + rem;
    }
    double accG[5] = {0, 0, 0, 0, 0};
    double accb = 0.0;  // entry lane (< L) of Phi_i' Y_i^C
    long long j0, j1;
    if (layout == 1) {
      j0 = offs[i];
      j1 = offs[i + 1];
    } else {
      j0 = 0;
      j1 = g.P;
    }
    for (long long c0 = j0; c0 < j1; c0 += 32) {
      const long long j = c0 + lane;
      int b = -1;
      double yc = 0.0;
      if (j < j1) {
        if (layout == 1) {
          b = sc_bin(g, t + j * g.d);
          yc = static_cast<const double*>(y)[j] - mu[b];
        } else if (!mask || mask[(long long)i * g.P + j]) {
          b = (int)j;
          const long long e = (long long)i * g.P + j;
          const double yv = yprec == FPCA_F64 ? static_cast<const double*>(y)[e]
                                              : (double)static_cast<const float*>(y)[e];
          yc = yv - mu[b];
        }
      }
      for (int l = 0; l < L; ++l) rows[warp][lane][l] = b >= 0 ? phi[(long long)l * g.P + b] : 0.0;
      rows[warp][lane][SC_LMAX] = yc;
      __syncwarp();
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        if (er[q] < L) {
          double sacc = accG[q];
          for (int k = 0; k < 32; ++k) sacc = fma(rows[warp][k][er[q]], rows[warp][k][ec[q]], sacc);
          accG[q] = sacc;
        }
      }
      if (lane < L) {
        double sacc = accb;
        for (int k = 0; k < 32; ++k) sacc = fma(rows[warp][k][lane], rows[warp][k][SC_LMAX], sacc);
        accb = sacc;
      }
      __syncwarp();
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) {
      if (er[q] < L) {
        sysA[warp][er[q]][ec[q]] = accG[q];
        sysA[warp][ec[q]][er[q]] = accG[q];
      }
    }
    if (lane < L) sysb[warp][lane] = accb;
    __syncwarp();
    if (lane == 0) {
      // (sigma^2 Lambda^{-1} + G) a = b by Cholesky in FP64, solved in place in bb.
      double (*A)[SC_LMAX + 1] = sysA[warp];
      double* bb = sysb[warp];
      const double sigma2 = *sigma2p;
      bool ok = sigma2 >= 0.0;
      for (int l = 0; l < L; ++l) {
        if (!(lam[l] > 0.0)) ok = false;
        A[l][l] += sigma2 / lam[l];
      }
      for (int jj = 0; jj < L && ok; ++jj) {
        double dj = A[jj][jj];
        for (int k = 0; k < jj; ++k) dj -= A[jj][k] * A[jj][k];
        if (!(dj > 0.0)) {
          ok = false;
          break;
        }
        const double ljj = sqrt(dj), il = 1.0 / ljj;
        A[jj][jj] = ljj;
        for (int r = jj + 1; r < L; ++r) {
          double v = A[r][jj];
          for (int k = 0; k < jj; ++k) v -= A[r][k] * A[jj][k];
          A[r][jj] = v * il;
        }
      }
      if (ok) {
        for (int r = 0; r < L; ++r) {
          double v = bb[r];
          for (int k = 0; k < r; ++k) v -= A[r][k] * bb[k];
          bb[r] = v / A[r][r];
        }
        for (int r = L - 1; r >= 0; --r) {
          double v = bb[r];
          for (int k = r + 1; k < L; ++k) v -= A[k][r] * bb[k];
          bb[r] = v / A[r][r];
        }
      } else {
        atomicExch(err, DERR_NUMERIC);
        for (int r = 0; r < L; ++r) bb[r] = __longlong_as_double(0x7ff8000000000000ll);
      }
    }
    __syncwarp();
    if (lane < L) scores[(long long)i * L + lane] = sysb[warp][lane];
    __syncwarp();
  }
}

// A_il = dV sum_p mask (Y_ip - mu_p) phi_l(p): one warp per subject.
__global__ void __launch_bounds__(256)
    k_scores_integral(int n, int P, const void* __restrict__ y, int yprec,
                      const uint8_t* __restrict__ mask, const double* __restrict__ mu,
                      const double* __restrict__ phi, int L, double dv,
                      double* __restrict__ scores) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n) return;
  const long long row = (long long)warp * P;
  double acc[SC_LMAX];
#pragma unroll
  for (int l = 0; l < SC_LMAX; ++l) acc[l] = 0.0;
  for (int p = lane; p < P; p += 32) {
    if (mask && !mask[row + p]) continue;
    const double yv = yprec == FPCA_F64 ? static_cast<const double*>(y)[row + p]
                                        : (double)static_cast<const float*>(y)[row + p];
    const double r = yv - mu[p];
#pragma unroll
    for (int l = 0; l < SC_LMAX; ++l)
      if (l < L) acc[l] = fma(r, phi[(long long)l * P + p], acc[l]);
  }
#pragma unroll
  for (int l = 0; l < SC_LMAX; ++l) {
    if (l >= L) break;
    double v = acc[l];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) scores[(long long)warp * L + l] = v * dv;
  }
}

// X_i(p) = mu_p + sum_l A_il phi_l(p), FP32 out.
__global__ void k_reconstruct(int n, int P, const double* __restrict__ mu,
                              const double* __restrict__ phi, int L,
                              const double* __restrict__ scores, float* __restrict__ xhat) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)n * P) return;
  const int i = (int)(e / P), p = (int)(e - (long long)i * P);
  double v = mu[p];
  for (int l = 0; l < L; ++l) v = fma(scores[(long long)i * L + l], phi[(long long)l * P + p], v);
  xhat[e] = (float)v;
}

ScGrid sc_grid(const fpca_grid* g) {
  ScGrid s{};
  s.d = g->d;
  s.P = 1;
  for (int k = 0; k < 3; ++k) {
    s.m[k] = k < g->d ? g->m[k] : 1;
    if (k < g->d) s.P *= g->m[k];
  }
  return s;
}

bool sc_valid(fpca_ctx* ctx, const fpca_grid* g, int L) {
  if (!g || g->d < 1 || g->d > 3) {
    fpca_fail(ctx, FPCA_E_INVALID_ARG, "grid.d must be 1..3");
    return false;
  }
  for (int k = 0; k < g->d; ++k)
    if (g->m[k] < 1) {
      fpca_fail(ctx, FPCA_E_INVALID_ARG, "grid.m[%d] must be positive", k);
      return false;
    }
  if (L < 1 || L > SC_LMAX) {
    fpca_fail(ctx, FPCA_E_INVALID_ARG, "L must be 1..%d", SC_LMAX);
    return false;
  }
  return true;
}

}  // namespace

extern "C" {

fpca_status fpca_scores_pace(fpca_ctx* ctx, const fpca_data* data, const fpca_grid* grid,
                             const double* mu, const double* evals, const double* evecs, int L,
                             const double* sigma2, double* scores) {
  if (!ctx) return FPCA_E_INVALID_ARG;
  fpca_prof_mark(ctx);
  if (!sc_valid(ctx, grid, L)) return FPCA_E_INVALID_ARG;
  if (!data || !mu || !evals || !evecs || !sigma2 || !scores)
    return fpca_fail(ctx, FPCA_E_INVALID_ARG,
                     "data, mu, evals, evecs, sigma2 and scores are required");
  if (data->n < 1 || !data->y) return fpca_fail(ctx, FPCA_E_INVALID_ARG, "data.n >= 1 and y");
  if (data->layout == FPCA_SPARSE && (!data->offs || !data->t))
    return fpca_fail(ctx, FPCA_E_INVALID_ARG, "scattered data need offs and t");
  const ScGrid g = sc_grid(grid);
  const int blocks = (data->n + SC_WARPS - 1) / SC_WARPS;
  k_scores_pace<<<blocks, 32 * SC_WARPS, 0, ctx->stream>>>(
      g, data->n, data->layout == FPCA_SPARSE ? 1 : 0, data->y, data->y_prec, data->mask,
      data->offs, data->t, mu, evals, evecs, L, sigma2, scores, ctx->d_err);
  FPCA_LAUNCHED(ctx, "scores_pace");
  return FPCA_OK;
}

fpca_status fpca_scores_integral(fpca_ctx* ctx, const fpca_data* data, const fpca_grid* grid,
                                 const double* mu, const double* evecs, int L, double* scores) {
  if (!ctx) return FPCA_E_INVALID_ARG;
  fpca_prof_mark(ctx);
  if (!sc_valid(ctx, grid, L)) return FPCA_E_INVALID_ARG;
  if (!data || !mu || !evecs || !scores)
    return fpca_fail(ctx, FPCA_E_INVALID_ARG, "data, mu, evecs and scores are required");
  if (data->layout != FPCA_DENSE || !data->y || data->n < 1)
    return fpca_fail(ctx, FPCA_E_INVALID_ARG, "scores by integration need gridded (dense) data");
  const ScGrid g = sc_grid(grid);
  const long long threads = (long long)data->n * 32;
  k_scores_integral<<<(int)((threads + 255) / 256), 256, 0, ctx->stream>>>(
      data->n, g.P, data->y, data->y_prec, data->mask, mu, evecs, L, 1.0 / (double)g.P, scores);
  FPCA_LAUNCHED(ctx, "scores_integral");
  return FPCA_OK;
}

fpca_status fpca_reconstruct(fpca_ctx* ctx, const fpca_grid* grid, const double* mu,
                             const double* evecs, int L, const double* scores, int n,
                             float* xhat) {
  if (!ctx) return FPCA_E_INVALID_ARG;
  fpca_prof_mark(ctx);
  if (!sc_valid(ctx, grid, L)) return FPCA_E_INVALID_ARG;
  if (!mu || !evecs || !scores || !xhat || n < 1)
    return fpca_fail(ctx, FPCA_E_INVALID_ARG, "mu, evecs, scores, xhat and n >= 1 are required");
  const ScGrid g = sc_grid(grid);
  const long long tot = (long long)n * g.P;
  k_reconstruct<<<(int)((tot + 255) / 256), 256, 0, ctx->stream>>>(n, g.P, mu, evecs, L, scores,
                                                                   xhat);
  FPCA_LAUNCHED(ctx, "reconstruct");
  return FPCA_OK;
}

}  // extern "C"
