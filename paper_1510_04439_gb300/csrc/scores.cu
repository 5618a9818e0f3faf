// Principal component scores, reconstruction and its error (Section 2.1, Section 4).
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
// (Y_i - mu) phi_l; reconstruction X_i = mu + sum_l A_il phi_l at the nodes; the
// MISE of a reconstruction (Section 4) is the mean over subjects of the Riemann
// sum of (Xhat_i - X_i)^2.
//
// Arithmetic: the long sums run in FP32 with error-free transformations (the
// compensated dot product of Ogita, Rump and Oishi, "Accurate sum and dot
// product", 2005, on float-float inputs from ff.cuh): about FP64 accuracy at
// FP32 cost, since FP64 throughput on this GPU is 1/64 of FP32.  mu and phi are
// split into float-float once per call; the small L x L solves stay FP64.
#include <algorithm>
#include <cmath>

#include "fpca_internal.cuh"
#include "ff.cuh"

namespace {

constexpr int SC_LMAX = 16;

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

// Compensated accumulator: s + c is the running sum; each product a b of two
// float-float numbers enters through a two-product and a two-sum, and all the
// rounding errors are collected in c.
struct Acc {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add_prod(ff::F2 a, ff::F2 b) {
    const ff::F2 p = ff::two_prod(a.hi, b.hi);
    const ff::F2 t = ff::two_sum(s, p.hi);
    s = t.hi;
    c += t.lo + (p.lo + fmaf(a.hi, b.lo, a.lo * b.hi));
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

__device__ __forceinline__ ff::F2 split(double x) {
  const float hi = (float)x;
  return {hi, (float)(x - (double)hi)};
}

// y[e] - m in float-float, y FP32 or FP64, m = mu as float-float
__device__ __forceinline__ ff::F2 centred(const void* y, int yprec, long long e, ff::F2 m) {
  if (yprec == FPCA_F64)
    return split(static_cast<const double*>(y)[e] - ((double)m.hi + (double)m.lo));
  const ff::F2 t = ff::two_sum(static_cast<const float*>(y)[e], -m.hi);
  return ff::fast_two_sum(t.hi, t.lo - m.lo);
}

// out[e] = float-float split of in[e]
__global__ void k_split_ff(long long n, const double* __restrict__ in, float2* __restrict__ out) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
       e += (long long)gridDim.x * blockDim.x) {
    const ff::F2 v = split(in[e]);
    out[e] = make_float2(v.hi, v.lo);
  }
}

// layout 0: dense y (n x P, FP32/FP64 per yprec) with mask (or NULL);
// layout 1: scattered offs / t / y (FP64).  mu2 (P) and phi2 (L x P) float-float.
// WPS warps share a subject (its observations in chunks of 32, dealt round-robin);
// their partial sums are added in FP64 through shared memory before one thread
// solves.  Gridded data use WPS = 8 (thousands of nodes per subject), scattered
// data WPS = 1 with 4 subjects per block.
template <int WPS>
constexpr int pace_threads() { return WPS == 1 ? 128 : 256; }

template <int WPS>
__global__ void __launch_bounds__(pace_threads<WPS>())
    k_scores_pace(ScGrid g, int n, int layout, const void* __restrict__ y, int yprec,
                  const uint8_t* __restrict__ mask, const int64_t* __restrict__ offs,
                  const double* __restrict__ t, const float2* __restrict__ mu2,
                  const double* __restrict__ lam, const float2* __restrict__ phi2, int L,
                  const double* __restrict__ sigma2p, double* __restrict__ scores,
                  int* __restrict__ err) {
  constexpr int PACE_THREADS = pace_threads<WPS>();
  constexpr int NW = PACE_THREADS / 32;  // warps per block
  constexpr int SPB = NW / WPS;          // subjects per block
  constexpr int NEMAX = SC_LMAX * (SC_LMAX + 1) / 2 + SC_LMAX;
  __shared__ float2 rows[NW][32][SC_LMAX + 1];  // phi rows, then the residual
  __shared__ double part[NW][NEMAX];             // each warp's sums: G entries, then b
  __shared__ double sysA[SPB][SC_LMAX][SC_LMAX + 1];
  __shared__ double sysb[SPB][SC_LMAX];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int slot = warp / WPS, wsub = warp % WPS;
  const int NE = L * (L + 1) / 2;
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
  for (int i0 = blockIdx.x * SPB; i0 < n; i0 += gridDim.x * SPB) {
    const int i = i0 + slot;
    const bool active = i < n;
    Acc accG[5];
    Acc accb;  // entry lane (< L) of Phi_i' Y_i^C
    long long j0 = 0, j1 = 0;
    if (active) {
      if (layout == 1) {
        j0 = offs[i];
        j1 = offs[i + 1];
      } else {
        j1 = g.P;
      }
    }
    for (long long c0 = j0 + 32 * wsub; c0 < j1; c0 += 32 * WPS) {
      const long long j = c0 + lane;
      int b = -1;
      ff::F2 yc = ff::make(0.f);
      if (j < j1) {
        if (layout == 1) {
          b = sc_bin(g, t + j * g.d);
          const float2 m = mu2[b];
          yc = split(static_cast<const double*>(y)[j] - ((double)m.x + (double)m.y));
        } else if (!mask || mask[(long long)i * g.P + j]) {
          b = (int)j;
          const float2 m = mu2[b];
          yc = centred(y, yprec, (long long)i * g.P + j, ff::F2{m.x, m.y});
        }
      }
      for (int l = 0; l < L; ++l)
        rows[warp][lane][l] = b >= 0 ? phi2[(long long)l * g.P + b] : make_float2(0.f, 0.f);
      rows[warp][lane][SC_LMAX] = make_float2(yc.hi, yc.lo);
      __syncwarp();
#pragma unroll
      for (int q = 0; q < 5; ++q) {
        if (er[q] < L) {
          for (int k = 0; k < 32; ++k) {
            const float2 a = rows[warp][k][er[q]], c = rows[warp][k][ec[q]];
            accG[q].add_prod(ff::F2{a.x, a.y}, ff::F2{c.x, c.y});
          }
        }
      }
      if (lane < L) {
        for (int k = 0; k < 32; ++k) {
          const float2 a = rows[warp][k][lane], c = rows[warp][k][SC_LMAX];
          accb.add_prod(ff::F2{a.x, a.y}, ff::F2{c.x, c.y});
        }
      }
      __syncwarp();
    }
#pragma unroll
    for (int q = 0; q < 5; ++q)
      if (er[q] < L) part[warp][lane + 32 * q] = accG[q].value();
    if (lane < L) part[warp][NE + lane] = accb.value();
    __syncthreads();
    // the subject's sums, warps added in a fixed order
    for (int e = threadIdx.x; e < SPB * (NE + L); e += PACE_THREADS) {
      const int sl = e / (NE + L), k = e - sl * (NE + L);
      double v = 0.0;
      for (int w = 0; w < WPS; ++w) v += part[sl * WPS + w][k];
      if (k < NE) {
        int r = 0, rem = k;
        while (rem >= L - r) {
          rem -= L - r;
          ++r;
        }
        sysA[sl][r][r + rem] = v;
        sysA[sl][r + rem][r] = v;
      } else {
        sysb[sl][k - NE] = v;
      }
    }
    __syncthreads();
    if (wsub == 0 && lane == 0 && active) {
      // (sigma^2 Lambda^{-1} + G) a = b by Cholesky in FP64, solved in place in bb.
      double (*A)[SC_LMAX + 1] = sysA[slot];
      double* bb = sysb[slot];
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
    __syncthreads();
    if (wsub == 0 && lane < L && active) scores[(long long)i * L + lane] = sysb[slot][lane];
    __syncthreads();
  }
}

// A_il = dV sum_p mask (Y_ip - mu_p) phi_l(p): one block of 8 warps per subject,
// compensated per-thread sums joined in FP64 (shuffles, then the warps in order).
template <int LM>
__global__ void __launch_bounds__(256)
    k_scores_integral(int n, int P, const void* __restrict__ y, int yprec,
                      const uint8_t* __restrict__ mask, const float2* __restrict__ mu2,
                      const float2* __restrict__ phi2, int L, double dv,
                      double* __restrict__ scores) {
  __shared__ double wsum[8][LM];
  const int i = blockIdx.x, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long row = (long long)i * P;
  Acc acc[LM];
  for (int p = threadIdx.x; p < P; p += 256) {
    if (mask && !mask[row + p]) continue;
    const float2 m = mu2[p];
    const ff::F2 r = centred(y, yprec, row + p, ff::F2{m.x, m.y});
#pragma unroll
    for (int l = 0; l < LM; ++l) {
      if (l < L) {
        const float2 f = phi2[(long long)l * P + p];
        acc[l].add_prod(r, ff::F2{f.x, f.y});
      }
    }
  }
#pragma unroll
  for (int l = 0; l < LM; ++l) {
    double v = acc[l].value();
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) wsum[warp][l] = v;
  }
  __syncthreads();
  if (threadIdx.x < L) {
    double v = 0.0;
    for (int w = 0; w < 8; ++w) v += wsum[w][threadIdx.x];
    scores[(long long)i * L + threadIdx.x] = v * dv;
  }
}

// X_i(p) = mu_p + sum_l A_il phi_l(p), compensated, rounded once to FP32.  A
// thread keeps node p's mu and phi in registers and walks RC_SUB subjects whose
// scores were split into shared memory once per block.
constexpr int RC_SUB = 16;
template <int LM>
__global__ void __launch_bounds__(256)
    k_reconstruct(int n, int P, const float2* __restrict__ mu2, const float2* __restrict__ phi2,
                  int L, const double* __restrict__ scores, float* __restrict__ xhat) {
  __shared__ float2 a2[RC_SUB][LM];
  const int i0 = blockIdx.y * RC_SUB;
  for (int e = threadIdx.x; e < RC_SUB * LM; e += blockDim.x) {
    const int ii = e / LM, l = e - ii * LM;
    ff::F2 v = ff::make(0.f);
    if (i0 + ii < n && l < L) v = split(scores[(long long)(i0 + ii) * L + l]);
    a2[ii][l] = make_float2(v.hi, v.lo);
  }
  __syncthreads();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const float2 m = mu2[p];
  float2 f[LM];
#pragma unroll
  for (int l = 0; l < LM; ++l) f[l] = l < L ? phi2[(long long)l * P + p] : make_float2(0.f, 0.f);
  for (int ii = 0; ii < RC_SUB && i0 + ii < n; ++ii) {
    Acc acc;
    acc.s = m.x;
    acc.c = m.y;
#pragma unroll
    for (int l = 0; l < LM; ++l)
      if (l < L) acc.add_prod(ff::F2{a2[ii][l].x, a2[ii][l].y}, ff::F2{f[l].x, f[l].y});
    xhat[(long long)(i0 + ii) * P + p] = acc.s + acc.c;
  }
}

// Per-block partial sums of (xhat - x)^2 (compensated per thread, pairwise tree
// per block).
constexpr int MS_THREADS = 256;
__global__ void __launch_bounds__(MS_THREADS)
    k_mise_partial(long long ne, const float* __restrict__ xhat, const void* __restrict__ x,
                   int xprec, double* __restrict__ part) {
  __shared__ double red[MS_THREADS];
  Acc acc;
  for (long long e = blockIdx.x * (long long)MS_THREADS + threadIdx.x; e < ne;
       e += (long long)gridDim.x * MS_THREADS) {
    ff::F2 d;
    if (xprec == FPCA_F64)
      d = split((double)xhat[e] - static_cast<const double*>(x)[e]);
    else
      d = ff::two_sum(xhat[e], -static_cast<const float*>(x)[e]);
    acc.add_prod(d, d);
  }
  red[threadIdx.x] = acc.value();
  __syncthreads();
  for (int h = MS_THREADS / 2; h >= 1; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// out = scale * (sum of the nb partials), fixed pairwise tree in one block.
__global__ void __launch_bounds__(MS_THREADS)
    k_mise_final(int nb, const double* __restrict__ part, double scale, double* __restrict__ out) {
  __shared__ double red[MS_THREADS];
  double v = 0.0;
  for (int b = threadIdx.x; b < nb; b += MS_THREADS) v += part[b];
  red[threadIdx.x] = v;
  __syncthreads();
  for (int h = MS_THREADS / 2; h >= 1; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0] * scale;
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

bool sc_valid_grid(fpca_ctx* ctx, const fpca_grid* g) {
  if (!g || g->d < 1 || g->d > 3) {
    fpca_fail(ctx, FPCA_E_INVALID_ARG, "grid.d must be 1..3");
    return false;
  }
  for (int k = 0; k < g->d; ++k)
    if (g->m[k] < 1) {
      fpca_fail(ctx, FPCA_E_INVALID_ARG, "grid.m[%d] must be positive", k);
      return false;
    }
  return true;
}

bool sc_valid(fpca_ctx* ctx, const fpca_grid* g, int L) {
  if (!sc_valid_grid(ctx, g)) return false;
  if (L < 1 || L > SC_LMAX) {
    fpca_fail(ctx, FPCA_E_INVALID_ARG, "L must be 1..%d", SC_LMAX);
    return false;
  }
  return true;
}

// mu (P) and the first L eigenfunctions (L x P) as float-float in the workspace.
fpca_status sc_split(fpca_ctx* ctx, int P, int L, const double* mu, const double* evecs,
                     float2** mu2, float2** phi2) {
  const size_t nmu = (size_t)P, nphi = (size_t)L * P;
  float2* ws = static_cast<float2*>(fpca_workspace(ctx, sizeof(float2) * (nmu + nphi)));
  if (!ws) return fpca_fail(ctx, FPCA_E_OOM, "workspace");
  *mu2 = ws;
  *phi2 = ws + nmu;
  k_split_ff<<<(int)std::min<size_t>((nmu + 255) / 256, 4096), 256, 0, ctx->stream>>>(
      (long long)nmu, mu, *mu2);
  FPCA_LAUNCHED(ctx, "split_ff");
  k_split_ff<<<(int)std::min<size_t>((nphi + 255) / 256, 4096), 256, 0, ctx->stream>>>(
      (long long)nphi, evecs, *phi2);
  FPCA_LAUNCHED(ctx, "split_ff");
  return FPCA_OK;
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
  float2 *mu2 = nullptr, *phi2 = nullptr;
  fpca_status s = sc_split(ctx, g.P, L, mu, evecs, &mu2, &phi2);
  if (s != FPCA_OK) return s;
  if (data->layout == FPCA_SPARSE) {
    const int blocks = (data->n + 3) / 4;
    k_scores_pace<1><<<blocks, pace_threads<1>(), 0, ctx->stream>>>(
        g, data->n, 1, data->y, data->y_prec, data->mask, data->offs, data->t, mu2, evals, phi2,
        L, sigma2, scores, ctx->d_err);
  } else {
    k_scores_pace<8><<<data->n, pace_threads<8>(), 0, ctx->stream>>>(
        g, data->n, 0, data->y, data->y_prec, data->mask, data->offs, data->t, mu2, evals, phi2,
        L, sigma2, scores, ctx->d_err);
  }
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
  float2 *mu2 = nullptr, *phi2 = nullptr;
  fpca_status s = sc_split(ctx, g.P, L, mu, evecs, &mu2, &phi2);
  if (s != FPCA_OK) return s;
  const double dv = 1.0 / (double)g.P;
  if (L <= 8)
    k_scores_integral<8><<<data->n, 256, 0, ctx->stream>>>(data->n, g.P, data->y, data->y_prec,
                                                           data->mask, mu2, phi2, L, dv, scores);
  else
    k_scores_integral<16><<<data->n, 256, 0, ctx->stream>>>(data->n, g.P, data->y, data->y_prec,
                                                            data->mask, mu2, phi2, L, dv, scores);
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
  const int nsub = (n + RC_SUB - 1) / RC_SUB;
  if (nsub > 65535) return fpca_fail(ctx, FPCA_E_UNSUPPORTED, "more than 2^20 subjects per call");
  const ScGrid g = sc_grid(grid);
  float2 *mu2 = nullptr, *phi2 = nullptr;
  fpca_status s = sc_split(ctx, g.P, L, mu, evecs, &mu2, &phi2);
  if (s != FPCA_OK) return s;
  const dim3 grid2((g.P + 255) / 256, nsub);
  if (L <= 8)
    k_reconstruct<8><<<grid2, 256, 0, ctx->stream>>>(n, g.P, mu2, phi2, L, scores, xhat);
  else
    k_reconstruct<16><<<grid2, 256, 0, ctx->stream>>>(n, g.P, mu2, phi2, L, scores, xhat);
  FPCA_LAUNCHED(ctx, "reconstruct");
  return FPCA_OK;
}

fpca_status fpca_mise(fpca_ctx* ctx, const fpca_grid* grid, const float* xhat, const void* x,
                      int x_prec, int n, double* mise) {
  if (!ctx) return FPCA_E_INVALID_ARG;
  fpca_prof_mark(ctx);
  if (!sc_valid_grid(ctx, grid)) return FPCA_E_INVALID_ARG;
  if (!xhat || !x || !mise || n < 1)
    return fpca_fail(ctx, FPCA_E_INVALID_ARG, "xhat, x, mise and n >= 1 are required");
  if (x_prec != FPCA_F64 && x_prec != FPCA_F32)
    return fpca_fail(ctx, FPCA_E_INVALID_ARG, "x_prec must be FPCA_F64 or FPCA_F32");
  const ScGrid g = sc_grid(grid);
  const long long ne = (long long)n * g.P;
  const int nb = (int)std::min<long long>((ne + MS_THREADS - 1) / MS_THREADS,
                                          (long long)std::max(1, ctx->num_sms) * 8);
  double* part = static_cast<double*>(fpca_workspace(ctx, sizeof(double) * nb));
  if (!part) return fpca_fail(ctx, FPCA_E_OOM, "workspace");
  k_mise_partial<<<nb, MS_THREADS, 0, ctx->stream>>>(ne, xhat, x, x_prec, part);
  FPCA_LAUNCHED(ctx, "mise");
  k_mise_final<<<1, MS_THREADS, 0, ctx->stream>>>(nb, part, 1.0 / ((double)g.P * (double)n),
                                                  mise);
  FPCA_LAUNCHED(ctx, "mise");
  return FPCA_OK;
}

}  // extern "C"
