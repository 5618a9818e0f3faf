// Eigen step: matrixisation (Section 3.1, Eq. 3.1) and the random projection
// of Section 3.4 (range finder with power iterations and Rayleigh-Ritz).
//
//  Sigma    = (G + G')/2, NaN -> 0, rows/columns outside the domain -> 0
//  Y        = Sigma Omega;  repeat q times { Q = orth(Y); Y = Sigma Q }
//  Q        = orth(Y) by CholeskyQR2 (compensated FP32 Gram, float-float Cholesky)
//  B        = Q' Sigma Q (FP64), eigenpairs of B by cyclic Jacobi (FP64)
//  Psi      = Q U;  lambda = theta dV;  phi = psi / sqrt(dV);  dV = 1/P
// The dense path (full = 1) runs the same Jacobi solver on Sigma itself.
#include <cmath>

#include "fpca_internal.cuh"
#include "ff.cuh"

namespace {

template <typename TG>
__device__ __forceinline__ double gval(const TG* G, long long idx) {
  const double x = (double)G[idx];
  return isnan(x) ? 0.0 : x;
}

// Sigma = sym(G) with NaN and out-of-domain entries zeroed; trace accumulated.
// The arithmetic is done in the type of Sigma (FP32 for the projected path).
template <typename TG, typename TS>
__global__ void k_matrixize(int P, const TG* __restrict__ G, const int32_t* __restrict__ dom,
                            TS* __restrict__ S, double* __restrict__ trace) {
  __shared__ TS tile[32][33];
  __shared__ double dsum;  // this block's part of the trace (diagonal blocks only)
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  if (threadIdx.x == 0 && threadIdx.y == 0) dsum = 0.0;
  // transposed tile: rows q in [bx, bx+32), columns p in [by, by+32)
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int q = bx + r, p = by + threadIdx.x;
    TS v = TS(0);
    if (q < P && p < P) {
      v = (TS)G[(long long)q * P + p];
      if (isnan(v)) v = TS(0);
    }
    tile[r][threadIdx.x] = v;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int p = by + r, q = bx + threadIdx.x;
    if (p < P && q < P) {
      TS g = (TS)G[(long long)p * P + q];
      if (isnan(g)) g = TS(0);
      TS sv = TS(0.5) * (g + tile[threadIdx.x][r]);
      if (dom && (dom[p] <= 0 || dom[q] <= 0)) sv = TS(0);
      S[(long long)p * P + q] = sv;
      if (p == q) atomicAdd(&dsum, (double)sv);
    }
  }
  // one global atomic per diagonal block instead of one per diagonal entry
  __syncthreads();
  if (bx == by && threadIdx.x == 0 && threadIdx.y == 0) atomicAdd(trace, dsum);
}

// Y (P x l) = S (P x P) X (P x l): a warp per RPW rows, lanes stride over the
// columns of S, X staged in shared memory in chunks of QCH rows.
// The column range is split over gridDim.y blocks (split-K); partial sums
// are added to Y (zeroed beforehand) with atomics.
template <typename TS, typename TX, int LM, int RPW>
__global__ void __launch_bounds__(256)
    k_proj(int P, int l, const TS* __restrict__ S, const TX* __restrict__ X,
           TX* __restrict__ Y) {
  constexpr int QCH = LM > 32 ? 128 : 256;
  constexpr int LP = LM + 1;
  __shared__ TX xs[QCH * LP];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row0 = (blockIdx.x * 8 + warp) * RPW;
  TX acc[RPW][LM];
#pragma unroll
  for (int r = 0; r < RPW; ++r)
#pragma unroll
    for (int c = 0; c < LM; ++c) acc[r][c] = TX(0);
  const int span = (P + gridDim.y - 1) / gridDim.y;
  const int qbeg = blockIdx.y * span, qend = min(P, qbeg + span);
  for (int q0 = qbeg; q0 < qend; q0 += QCH) {
    __syncthreads();
    for (int e = threadIdx.x; e < QCH * LM; e += 256) {
      const int qq = e / LM, c = e - qq * LM;
      xs[qq * LP + c] = (q0 + qq < qend && c < l) ? X[(long long)(q0 + qq) * l + c] : TX(0);
    }
    __syncthreads();
    // all of this chunk's Sigma loads are issued before the FMAs
    constexpr int NQ = QCH / 32;
    TX sv[NQ][RPW];
#pragma unroll
    for (int u = 0; u < NQ; ++u) {
      const int q = q0 + lane + 32 * u;
#pragma unroll
      for (int r = 0; r < RPW; ++r)
        sv[u][r] = (q < qend && row0 + r < P) ? (TX)S[(long long)(row0 + r) * P + q] : TX(0);
    }
#pragma unroll
    for (int u = 0; u < NQ; ++u) {
      const int t = lane + 32 * u;
#pragma unroll
      for (int c = 0; c < LM; ++c) {
        const TX xv = xs[t * LP + c];
#pragma unroll
        for (int r = 0; r < RPW; ++r) acc[r][c] = fma(sv[u][r], xv, acc[r][c]);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < RPW; ++r)
#pragma unroll
    for (int c = 0; c < LM; ++c) {
      TX v = acc[r][c];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      acc[r][c] = v;
    }
  if (lane == 0) {
#pragma unroll
    for (int r = 0; r < RPW; ++r)
      if (row0 + r < P) {
#pragma unroll
        for (int c = 0; c < LM; ++c)
          if (c < l) atomicAdd(Y + (long long)(row0 + r) * l + c, acc[r][c]);
      }
  }
}

// Partial Gram products A'B (l x l) over blocks of GR_ROWS rows (A, B: P x l),
// written per block and summed in block order by k_gram_sum (no atomics, so the
// result does not depend on scheduling).
//
// FP32 inputs use error-free transformations so that the sums keep about FP64
// accuracy at FP32 speed (GB300 runs FP64 at 1/64 of the FP32 rate): each
// product a*b is split exactly as p + e with e = fma(a, b, -p) (Dekker's
// two-product through an FMA), p is accumulated by Knuth's two-sum and the
// rounding errors are summed separately (the compensated dot product of Ogita,
// Rump and Oishi, "Accurate sum and dot product", 2005).  FP64 inputs use
// plain FP64 sums.
constexpr int GR_ROWS = 64;  // short per-entry chains, a wide grid
constexpr int GR_SUB = 32;

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float z = s - a;
  e = (a - (s - z)) + (b - z);
}

template <typename TX>
__global__ void __launch_bounds__(256)
    k_cross_gram(int P, int l, const TX* __restrict__ A, const TX* __restrict__ B,
                 double* __restrict__ part) {
  __shared__ TX As[GR_SUB * 64], Bs[GR_SUB * 64];
  const int r0 = blockIdx.x * GR_ROWS, r1 = min(P, r0 + GR_ROWS);
  const int ne = l * l;
  // up to 16 entries per thread (l <= 64, 256 threads)
  float hs[16], hc[16];
  double dsum[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    hs[k] = 0.f;
    hc[k] = 0.f;
    dsum[k] = 0.0;
  }
  for (int rb = r0; rb < r1; rb += GR_SUB) {
    const int nr = min(GR_SUB, r1 - rb);
    __syncthreads();
    for (int e = threadIdx.x; e < nr * l; e += blockDim.x) {
      As[e] = A[(long long)rb * l + e];
      Bs[e] = B[(long long)rb * l + e];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int e = threadIdx.x + k * 256;
      if (e >= ne) break;
      const int i = e / l, j = e - (e / l) * l;
      if constexpr (sizeof(TX) == 4) {
        float s = hs[k], c = hc[k];
        for (int r = 0; r < nr; ++r) {
          const float a = As[r * l + i], b = Bs[r * l + j];
          const float pp = a * b;
          const float pe = fmaf(a, b, -pp);
          float t, te;
          two_sum(s, pp, t, te);
          s = t;
          c += te + pe;
        }
        hs[k] = s;
        hc[k] = c;
      } else {
        double d = dsum[k];
        for (int r = 0; r < nr; ++r) d += (double)As[r * l + i] * (double)Bs[r * l + j];
        dsum[k] = d;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int e = threadIdx.x + k * 256;
    if (e >= ne) break;
    part[(long long)blockIdx.x * ne + e] =
        sizeof(TX) == 4 ? (double)hs[k] + (double)hc[k] : dsum[k];
  }
}

// G = sum over blocks of the partial products (FP64), one warp per entry: each
// lane adds its blocks in two interleaved chains, then a fixed shuffle tree
// combines the lanes, so the result does not depend on scheduling and the
// dependent FP64 adds (long-latency on this GPU) stay few.
__global__ void k_gram_sum(int nb, int ne, const double* __restrict__ part, double* __restrict__ G) {
  const int e = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (e >= ne) return;
  double s0 = 0.0, s1 = 0.0;
  for (int b = lane; b < nb; b += 64) {
    s0 += part[(long long)b * ne + e];
    if (b + 32 < nb) s1 += part[(long long)(b + 32) * ne + e];
  }
  double s = s0 + s1;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) G[e] = s;
}

template <typename TX>
fpca_status launch_cross_gram(fpca_ctx* ctx, int P, int l, const TX* A, const TX* B, double* part,
                              double* G, const char* name) {
  const int nb = (P + GR_ROWS - 1) / GR_ROWS;
  k_cross_gram<TX><<<nb, 256, 0, ctx->stream>>>(P, l, A, B, part);
  FPCA_LAUNCHED(ctx, name);
  k_gram_sum<<<(l * l + 7) / 8, 256, 0, ctx->stream>>>(nb, l * l, part, G);
  FPCA_LAUNCHED(ctx, "gram_sum");
  return FPCA_OK;
}

// 1/sqrt(a) in float-float for a > 0 in FP32 range: the FP32 estimate y0 and one
// Newton-Raphson step on f(y) = y^-2 - a, y1 = y0 + y0 (1 - a y0^2) / 2, with the
// residual 1 - a y0^2 formed in float-float (error about 1e-14 relative).
__device__ __forceinline__ ff::F2 rsqrt_ff(ff::F2 a) {
  const float y0 = rsqrtf(a.hi);
  const ff::F2 ay2 = ff::mul(a, ff::two_prod(y0, y0));
  const ff::F2 e = ff::add(ff::make(1.0f), ff::neg(ay2));
  return ff::fast_two_sum(y0, 0.5f * y0 * e.hi);
}

__device__ __forceinline__ ff::F2 ff_of(double x) {
  const float hi = (float)x;
  return {hi, (float)(x - (double)hi)};
}

// Upper Cholesky G = R'R and R^-1 in float-float (l <= 64), one block of
// CH_THREADS threads, everything in shared memory.  Float-float rather than
// FP64: FP64 operations have long latency on this GPU and both factorisations
// are serial chains of l steps (the Gram matrix factored here is itself
// accurate to about 1e-14, from the compensated Gram kernel).  Each step's
// updates are spread over all threads, so a step costs a few dependent
// float-float operations and two barriers.
//   Cholesky, right-looking: step j forms 1/sqrt(G_jj) and row j of R, then
//   G_ik -= R_ji R_jk over the trailing upper triangle i <= k.
//   Inverse, by rows from the bottom: x_ic = (delta_ic - a_ic) / R_ii for every
//   column c >= i, then a_kc += R_ki x_ic for k < i (a starts at 0).
// Output: R^-1 (l x l row-major, upper triangular) as hi parts Ih and lo parts
// Il.  Rank-deficient directions (pivot <= 1e-13 of the largest diagonal) get a
// zero row and column.
constexpr int CH_THREADS = 256;
inline size_t chol_ff_smem(int l) { return sizeof(float) * (4 * (size_t)l * (l + 1) + 2 * l + 1); }

__global__ void __launch_bounds__(CH_THREADS) k_chol_ff(int l, const double* __restrict__ G,
                                                        float* __restrict__ Ih,
                                                        float* __restrict__ Il) {
  extern __shared__ float chs[];
  const int ld = l + 1;
  float* Gh = chs;              // [l][ld] trailing matrix, then R by rows
  float* Gl = Gh + l * ld;
  float* Ah = Gl + l * ld;      // [l][ld] sums of the inverse's back substitution
  float* Al = Ah + l * ld;
  float* yh = Al + l * ld;      // [l] 1 / R_jj
  float* yl = yh + l;
  float* dmax_s = yl + l;
  const int t = threadIdx.x;
  for (int e = t; e < l * l; e += CH_THREADS) {
    const int i = e / l, k = e - i * l;
    const ff::F2 g = ff_of(G[e]);
    Gh[i * ld + k] = g.hi;
    Gl[i * ld + k] = g.lo;
    Ah[i * ld + k] = 0.f;
    Al[i * ld + k] = 0.f;
  }
  __syncthreads();
  if (t < 32) {
    float dm = 0.f;
    for (int i = t; i < l; i += 32) dm = fmaxf(dm, Gh[i * ld + i]);
    for (int o = 16; o > 0; o >>= 1) dm = fmaxf(dm, __shfl_xor_sync(0xffffffffu, dm, o));
    if (t == 0) *dmax_s = dm;
  }
  __syncthreads();
  const float dmax = *dmax_s;
#pragma unroll 1
  for (int j = 0; j < l; ++j) {
    // row j of R (entries k >= j), every thread computing the same 1/sqrt(pivot)
    const ff::F2 piv = {Gh[j * ld + j], Gl[j * ld + j]};
    ff::F2 y = ff::make(0.f);
    if (piv.hi > 1e-13f * dmax) y = rsqrt_ff(piv);
    __syncthreads();  // every thread has read the pivot
    for (int k = j + t; k < l; k += CH_THREADS) {
      const ff::F2 r = ff::mul(k == j ? piv : ff::F2{Gh[j * ld + k], Gl[j * ld + k]}, y);
      Gh[j * ld + k] = r.hi;
      Gl[j * ld + k] = r.lo;
    }
    if (t == 0) {
      yh[j] = y.hi;
      yl[j] = y.lo;
    }
    __syncthreads();
    // trailing upper triangle j < i <= k < l
    const int m = l - j - 1;
    for (int e = t; e < m * m; e += CH_THREADS) {
      const int i = j + 1 + e / m, k = j + 1 + e % m;
      if (k < i) continue;
      const ff::F2 g = ff::sub_mul(ff::F2{Gh[i * ld + k], Gl[i * ld + k]},
                                   ff::F2{Gh[j * ld + i], Gl[j * ld + i]},
                                   ff::F2{Gh[j * ld + k], Gl[j * ld + k]});
      Gh[i * ld + k] = g.hi;
      Gl[i * ld + k] = g.lo;
    }
    __syncthreads();
  }
  // R^-1 by rows from the bottom; row i of R^-1 goes straight to Ih/Il
#pragma unroll 1
  for (int i = l - 1; i >= 0; --i) {
    const ff::F2 d = {yh[i], yl[i]};
    for (int c = t; c < l; c += CH_THREADS) {
      ff::F2 x = ff::make(0.f);
      if (c >= i)
        x = ff::mul(ff::add(ff::make(c == i ? 1.f : 0.f), ff::neg(ff::F2{Ah[i * ld + c], Al[i * ld + c]})),
                    d);
      Ih[i * l + c] = x.hi;
      Il[i * l + c] = x.lo;
      Ah[i * ld + c] = x.hi;  // row i of the sums is dead: keep x there for the update
      Al[i * ld + c] = x.lo;
    }
    __syncthreads();
    for (int e = t; e < i * l; e += CH_THREADS) {
      const int k = e / l, c = e % l;
      if (c < i) continue;
      const ff::F2 a = ff::add(ff::F2{Ah[k * ld + c], Al[k * ld + c]},
                               ff::mul(ff::F2{Gh[k * ld + i], Gl[k * ld + i]},
                                       ff::F2{Ah[i * ld + c], Al[i * ld + c]}));
      Ah[k * ld + c] = a.hi;
      Al[k * ld + c] = a.lo;
    }
    __syncthreads();
  }
}

// Q = Y R^-1 with R^-1 from k_chol_ff, one thread per entry (row r, column j):
// q_rj = sum_{k <= j} y_rk R^-1[k][j], products and sum in float-float (R^-1 of
// an ill-conditioned basis has large entries whose contributions cancel), so
// the work spreads over P l threads and each chain is at most l terms long.
template <typename TX>
__global__ void __launch_bounds__(256) k_apply_ff(int P, int l, const TX* __restrict__ Y,
                                                  const float* __restrict__ Ih,
                                                  const float* __restrict__ Il,
                                                  TX* __restrict__ Q) {
  __shared__ float sh[64 * 64], sl[64 * 64];
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
    sh[e] = Ih[e];
    sl[e] = Il[e];
  }
  __syncthreads();
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)P * l) return;
  const long long r = e / l;
  const int j = (int)(e - r * l);
  const TX* yr = Y + r * l;
  ff::F2 acc = ff::make(0.f);
  for (int k = 0; k <= j; ++k) {
    ff::F2 yk;
    if constexpr (sizeof(TX) == 4)
      yk = ff::make((float)yr[k]);
    else
      yk = ff_of((double)yr[k]);
    acc = ff::add(acc, ff::mul(yk, ff::F2{sh[k * l + j], sl[k * l + j]}));
  }
  Q[e] = (TX)ff::to_double(acc);
}

// Cyclic parallel Jacobi (one block) on the symmetric n x n matrix A (global,
// FP64, destroyed), V <- eigenvectors (columns).  Pairs follow the circle
// method: n/2 disjoint rotations per step, n-1 steps per sweep.
__global__ void __launch_bounds__(1024)
    k_jacobi(int n, double* __restrict__ A, double* __restrict__ V, double* __restrict__ cs,
             int* __restrict__ pairs, int max_sweeps) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int ne = (n + 1) & ~1;  // even count (index n is a dummy when n is odd)
  const int np = ne / 2;
  for (int e = tid; e < n * n; e += nt) V[e] = (e / n == e % n) ? 1.0 : 0.0;
  __shared__ double red[32];
  __shared__ int done;
  __syncthreads();
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    // convergence: off-diagonal vs diagonal mass
    double off = 0.0, dia = 0.0;
    for (int e = tid; e < n * n; e += nt) {
      const int i = e / n, j = e - (e / n) * n;
      const double a = A[e];
      if (i == j) dia += a * a;
      else off += a * a;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      dia += __shfl_xor_sync(0xffffffffu, dia, o);
    }
    if ((tid & 31) == 0) red[tid >> 5] = off;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int w = 0; w < (nt + 31) / 32; ++w) s += red[w];
      red[0] = s;
    }
    __syncthreads();
    const double off_tot = red[0];
    __syncthreads();
    if ((tid & 31) == 0) red[tid >> 5] = dia;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int w = 0; w < (nt + 31) / 32; ++w) s += red[w];
      done = (off_tot <= 1e-26 * s) || off_tot == 0.0;
    }
    __syncthreads();
    if (done) break;
    for (int step = 0; step < ne - 1; ++step) {
      // pairs of this step and their rotations
      for (int i = tid; i < np; i += nt) {
        int p, q;
        if (i == 0) {
          p = ne - 1;
          q = step;
        } else {
          p = (step + i) % (ne - 1);
          q = (step - i + (ne - 1)) % (ne - 1);
        }
        if (p > q) {
          const int t = p;
          p = q;
          q = t;
        }
        double c = 1.0, s = 0.0;
        if (q < n) {
          const double apq = A[(long long)p * n + q];
          const double app = A[(long long)p * n + p], aqq = A[(long long)q * n + q];
          if (fabs(apq) > 1e-300 && fabs(apq) > 1e-18 * sqrt(fabs(app * aqq))) {
            const double tau = (aqq - app) / (2.0 * apq);
            const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            s = t * c;
          }
        }
        pairs[2 * i] = p;
        pairs[2 * i + 1] = q;
        cs[2 * i] = c;
        cs[2 * i + 1] = s;
      }
      __syncthreads();
      // A <- A J (columns p, q of every row)
      for (int e = tid; e < np * n; e += nt) {
        const int i = e / n, k = e - (e / n) * n;
        const int p = pairs[2 * i], q = pairs[2 * i + 1];
        if (q >= n) continue;
        const double c = cs[2 * i], s = cs[2 * i + 1];
        const double akp = A[(long long)k * n + p], akq = A[(long long)k * n + q];
        A[(long long)k * n + p] = c * akp - s * akq;
        A[(long long)k * n + q] = s * akp + c * akq;
        const double vkp = V[(long long)k * n + p], vkq = V[(long long)k * n + q];
        V[(long long)k * n + p] = c * vkp - s * vkq;
        V[(long long)k * n + q] = s * vkp + c * vkq;
      }
      __syncthreads();
      // A <- J' A (rows p, q of every column)
      for (int e = tid; e < np * n; e += nt) {
        const int i = e / n, k = e - (e / n) * n;
        const int p = pairs[2 * i], q = pairs[2 * i + 1];
        if (q >= n) continue;
        const double c = cs[2 * i], s = cs[2 * i + 1];
        const double apk = A[(long long)p * n + k], aqk = A[(long long)q * n + k];
        A[(long long)p * n + k] = c * apk - s * aqk;
        A[(long long)q * n + k] = s * apk + c * aqk;
      }
      __syncthreads();
    }
  }
}

// Cyclic parallel Jacobi sweeps (the pair schedule of k_jacobi) on A and V
// in shared memory, in the arithmetic of T, until off(A)^2 <= tol * diag(A)^2
// or max_sweeps; every thread of the block takes part.
template <typename T>
__device__ void jacobi_sweeps(int n, int ld, T* A, T* V, int max_sweeps, double tol, T* cs,
                              int* pr, double* red, int* done) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int ne = (n + 1) & ~1;
  const int np = ne / 2;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    // the stopping test in the working type T: an FP32 Jacobi needs no FP64
    // sums here (serial FP64 adds are slow on this GPU)
    T off = T(0), dia = T(0);
    for (int e = tid; e < n * n; e += nt) {
      const int r = e / n, c = e - r * n;
      const T a = A[r * ld + c];
      if (r == c) dia += a * a;
      else off += a * a;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      dia += __shfl_xor_sync(0xffffffffu, dia, o);
    }
    if ((tid & 31) == 0) {
      red[2 * (tid >> 5)] = (double)off;
      red[2 * (tid >> 5) + 1] = (double)dia;
    }
    __syncthreads();
    if (tid == 0) {
      T ot = T(0), dt = T(0);
      for (int w = 0; w < nt / 32; ++w) {
        ot += (T)red[2 * w];
        dt += (T)red[2 * w + 1];
      }
      *done = ((double)ot <= tol * (double)dt) || ot == T(0);
    }
    __syncthreads();
    if (*done) break;
    for (int step = 0; step < ne - 1; ++step) {
      if (tid < np) {
        const int i = tid;
        int p, q;
        if (i == 0) {
          p = ne - 1;
          q = step;
        } else {
          p = (step + i) % (ne - 1);
          q = (step - i + (ne - 1)) % (ne - 1);
        }
        if (p > q) {
          const int tt = p;
          p = q;
          q = tt;
        }
        T c = T(1), sn = T(0);
        if (q < n) {
          const T apq = A[p * ld + q], app = A[p * ld + p], aqq = A[q * ld + q];
          if (fabs(apq) > T(1e-30) && fabs(apq) > T(1e-18) * sqrt(fabs(app) * fabs(aqq))) {
            const T tau = (aqq - app) / (T(2) * apq);
            const T tt = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + sqrt(T(1) + tau * tau));
            c = T(1) / sqrt(T(1) + tt * tt);
            sn = tt * c;
          }
        }
        pr[2 * i] = p;
        pr[2 * i + 1] = q;
        cs[2 * i] = c;
        cs[2 * i + 1] = sn;
      }
      __syncthreads();
      for (int e = tid; e < np * n; e += nt) {
        const int i = e / n, k = e - (e / n) * n;
        const int p = pr[2 * i], q = pr[2 * i + 1];
        if (q >= n) continue;
        const T c = cs[2 * i], sn = cs[2 * i + 1];
        const T akp = A[k * ld + p], akq = A[k * ld + q];
        A[k * ld + p] = c * akp - sn * akq;
        A[k * ld + q] = sn * akp + c * akq;
        const T vkp = V[k * ld + p], vkq = V[k * ld + q];
        V[k * ld + p] = c * vkp - sn * vkq;
        V[k * ld + q] = sn * vkp + c * vkq;
      }
      __syncthreads();
      for (int e = tid; e < np * n; e += nt) {
        const int i = e / n, k = e - (e / n) * n;
        const int p = pr[2 * i], q = pr[2 * i + 1];
        if (q >= n) continue;
        const T c = cs[2 * i], sn = cs[2 * i + 1];
        const T apk = A[p * ld + k], aqk = A[q * ld + k];
        A[p * ld + k] = c * apk - sn * aqk;
        A[q * ld + k] = sn * apk + c * aqk;
      }
      __syncthreads();
    }
  }
}

// Symmetric eigendecomposition of the n x n (n <= 64) Rayleigh-Ritz matrix with an
// FP64 result at a fraction of the FP64 work (FP64 is slow on this GPU):
//  1. cyclic Jacobi in FP32 on (A + A')/2 (off-diagonal to 3e-5 of the diagonal, at
//     most 10 sweeps: FP32 rounding stalls it near 1e-7), one block;
//  2. two steps of the iterative refinement of Ogita and Aishima ("Iterative
//     refinement for symmetric eigenvalue decomposition", 2018) in FP64 on the FP32
//     eigenvectors X:  R = I - X'X,  S = X'AX,  lambda_i = s_ii / (1 - r_ii),
//     E_ij = (s_ij + lambda_j r_ij) / (lambda_j - lambda_i) for separated pairs and
//     r_ij / 2 inside clusters (gap <= delta = 2(|S - diag S| + |A| |R|), Frobenius
//     norms), X <- X + X E.  Each step squares the error, so two steps reach FP64.
//     Both steps run in one block (k_rr_refine) for n <= 32, as separate launches
//     spread over n blocks beyond.
// Outputs: A <- diag(lambda), V <- eigenvectors (columns, FP64).
__global__ void __launch_bounds__(1024)
    k_rr_jacobi32(int n, double* __restrict__ Ag, double* __restrict__ Asym,
                  double* __restrict__ X) {
  __shared__ float A32[64 * 65], V32[64 * 65];
  __shared__ float cs32[64];
  __shared__ int pr[64];
  __shared__ double red[64];
  __shared__ int done;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < n * n; e += nt) {
    const int i = e / n, j = e - (e / n) * n;
    const double a = 0.5 * (Ag[e] + Ag[j * n + i]);
    Asym[e] = a;
    A32[i * (n + 1) + j] = (float)a;
    V32[i * (n + 1) + j] = (i == j) ? 1.f : 0.f;
  }
  __syncthreads();
  jacobi_sweeps<float>(n, n + 1, A32, V32, 10, 1e-9, cs32, pr, red, &done);
  for (int e = tid; e < n * n; e += nt) X[e] = (double)V32[(e / n) * (n + 1) + e % n];
}

// The refinement for l > 32 (one SM's FP64 throughput is too low for the fused
// k_rr_refine at that size): the n x n x n products spread over n blocks.
// Row i (block) of C = op(L) M (+ D): op(L) = L' when tl, else L; one thread per column.
__global__ void k_rr_rowmm(int n, const double* __restrict__ L, int tl, const double* __restrict__ M,
                           double* __restrict__ C, double diag, double sign) {
  const int i = blockIdx.x, j = threadIdx.x;
  if (j >= n) return;
  double s = 0.0;
  for (int k = 0; k < n; ++k) s += (tl ? L[k * n + i] : L[i * n + k]) * M[k * n + j];
  C[i * n + j] = ((i == j) ? diag : 0.0) + sign * s;
}

// lambda, the cluster threshold and E (one block).
__global__ void __launch_bounds__(1024)
    k_rr_correction(int n, const double* __restrict__ A, const double* __restrict__ R,
                    const double* __restrict__ S, double* __restrict__ E, double* __restrict__ lam) {
  __shared__ double red[32][3];
  __shared__ double lm[64];
  __shared__ double delta;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < n; i += nt) lm[i] = S[i * n + i] / (1.0 - R[i * n + i]);
  double so = 0.0, an = 0.0, rn = 0.0;
  for (int e = tid; e < n * n; e += nt) {
    const int i = e / n, j = e - (e / n) * n;
    if (i != j) so += S[e] * S[e];
    an += A[e] * A[e];
    rn += R[e] * R[e];
  }
  for (int o = 16; o > 0; o >>= 1) {
    so += __shfl_xor_sync(0xffffffffu, so, o);
    an += __shfl_xor_sync(0xffffffffu, an, o);
    rn += __shfl_xor_sync(0xffffffffu, rn, o);
  }
  if ((tid & 31) == 0) {
    red[tid >> 5][0] = so;
    red[tid >> 5][1] = an;
    red[tid >> 5][2] = rn;
  }
  __syncthreads();
  if (tid == 0) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (int w = 0; w < nt / 32; ++w) {
      a += red[w][0];
      b += red[w][1];
      c += red[w][2];
    }
    delta = 2.0 * (sqrt(a) + sqrt(b) * sqrt(c));
  }
  __syncthreads();
  for (int e = tid; e < n * n; e += nt) {
    const int i = e / n, j = e - (e / n) * n;
    const double gap = lm[j] - lm[i];
    E[e] = (i == j || fabs(gap) <= delta) ? 0.5 * R[e] : (S[e] + lm[j] * R[e]) / gap;
  }
  for (int i = tid; i < n; i += nt) lam[i] = lm[i];
}

// X <- X + X E (row i per block; the row is read before it is written).
__global__ void k_rr_update(int n, double* __restrict__ X, const double* __restrict__ E) {
  __shared__ double row[64];
  const int i = blockIdx.x, j = threadIdx.x;
  if (j < n) row[j] = X[i * n + j];
  __syncthreads();
  if (j >= n) return;
  double s = row[j];
  for (int k = 0; k < n; ++k) s += row[k] * E[k * n + j];
  X[i * n + j] = s;
}

__global__ void k_rr_out(int n, const double* __restrict__ lam, const double* __restrict__ X,
                         double* __restrict__ Ag, double* __restrict__ Vg) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += gridDim.x * blockDim.x) {
    const int i = e / n, j = e - (e / n) * n;
    Ag[e] = (i == j) ? lam[i] : 0.0;
    Vg[e] = X[e];
  }
}

// Rank of each eigenvalue (descending; ties by index) -> order[rank] = index.
__global__ void k_eig_order(int n, const double* __restrict__ A, int* __restrict__ order) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double ti = A[(long long)i * n + i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const double tj = A[(long long)j * n + j];
      rank += (tj > ti) || (tj == ti && j < i);
    }
    order[rank] = i;
  }
}

// psi_j = Q u_{order[j]} (Q: P x l of type TX, U: l x l FP64), j < k.
template <typename TX>
__global__ void k_ritz_vectors(int P, int l, int k, const TX* __restrict__ Q,
                               const double* __restrict__ U, const int* __restrict__ order,
                               double* __restrict__ psi) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= P) return;
  for (int j = 0; j < k; ++j) {
    const int col = order[j];
    double s = 0.0;
    for (int i = 0; i < l; ++i) s += (double)Q[(long long)r * l + i] * U[(long long)i * l + col];
    psi[(long long)j * P + r] = s;
  }
}

// Dense path: psi_j = V[:, order[j]].
__global__ void k_dense_vectors(int P, int k, const double* __restrict__ V,
                                const int* __restrict__ order, double* __restrict__ psi) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)P * k) return;
  const int j = (int)(e / P), r = (int)(e - (long long)j * P);
  psi[e] = V[(long long)r * P + order[j]];
}

// Sign (largest-magnitude entry positive, first occurrence on ties), rescale
// phi = psi / sqrt(dV), lambda = theta dV, FVE.  One block per eigenvector.
__global__ void k_finish(int P, int n, int k, double dv, const double* __restrict__ Aeig,
                         const int* __restrict__ order, const double* __restrict__ trace,
                         double* __restrict__ evals, double* __restrict__ evecs,
                         double* __restrict__ fve) {
  const int j = blockIdx.x;
  double* v = evecs + (long long)j * P;
  __shared__ double bv[1024];
  __shared__ int bi[1024];
  double best = -1.0;
  int bidx = 0x7fffffff;
  for (int r = threadIdx.x; r < P; r += blockDim.x) {
    const double a = fabs(v[r]);
    if (a > best || (a == best && r < bidx)) {
      best = a;
      bidx = r;
    }
  }
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = bidx;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      const double ob = bv[threadIdx.x + s];
      const int oi = bi[threadIdx.x + s];
      if (ob > bv[threadIdx.x] || (ob == bv[threadIdx.x] && oi < bi[threadIdx.x])) {
        bv[threadIdx.x] = ob;
        bi[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  const double sign = v[bi[0]] < 0.0 ? -1.0 : 1.0;
  const double scale = sign / sqrt(dv);
  __syncthreads();
  for (int r = threadIdx.x; r < P; r += blockDim.x) v[r] *= scale;
  if (threadIdx.x == 0) {
    const double th = Aeig[(long long)order[j] * n + order[j]];
    evals[j] = th * dv;
    if (fve) {
      double cum = 0.0;
      for (int i = 0; i <= j; ++i) cum += Aeig[(long long)order[i] * n + order[i]] * dv;
      fve[j] = cum / (trace[0] * dv);
    }
  }
}

// Both Ogita-Aishima refinement steps of k_rr_jacobi32's eigenvectors in one block
// (l <= 32), with the l x l matrices in shared memory: per step
// R = I - X'X, U = A X, S = X'U, lambda_i = s_ii / (1 - r_ii),
// delta = 2 (|S - diag S| + |A| |R|), E_ij = (s_ij + lambda_j r_ij) / (lambda_j - lambda_i)
// or r_ij / 2 inside clusters, X <- X + X E; then A <- diag(lambda), V <- X.
// Each product entry is split into two half-length dot products (neighbouring
// threads), so the serial FP64 chains (long-latency on this GPU) stay about l/2
// long.
constexpr int RF_THREADS = 1024;
__device__ __forceinline__ void rf_product(int n, const double* L, bool tl, const double* M,
                                           double* C, double diag, double sign) {
  // C = diag I + sign op(L) M, op(L) = L' when tl; entry o by threads 2o and
  // 2o + 1 (neighbouring lanes), each summing half of k, joined by a shuffle
  const int h = (n + 1) / 2;
  const int ne2 = 2 * n * n;
  for (int base = 0; base < ne2; base += RF_THREADS) {
    const int e = base + threadIdx.x;
    const int o = e >> 1, part = e & 1;
    double acc = 0.0;
    if (e < ne2) {
      const int i = o / n, j = o - i * n;
      const int k0 = part * h, k1 = min(n, k0 + h);
      for (int k = k0; k < k1; ++k) acc = fma(tl ? L[k * n + i] : L[i * n + k], M[k * n + j], acc);
    }
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    if (e < ne2 && part == 0) {
      const int i = o / n, j = o - i * n;
      C[o] = ((i == j) ? diag : 0.0) + sign * acc;
    }
  }
  __syncthreads();
}

__device__ __forceinline__ double rf_block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    double x = red[lane];  // RF_THREADS / 32 == 32 partials
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) red[32] = x;
  }
  __syncthreads();
  const double r = red[32];
  __syncthreads();
  return r;
}

inline size_t rr_refine_smem(int n) { return sizeof(double) * (5 * (size_t)n * n + n + 33); }

__global__ void __launch_bounds__(RF_THREADS)
    k_rr_refine(int n, const double* __restrict__ Asym, const double* __restrict__ X0,
                double* __restrict__ Ag, double* __restrict__ Vg) {
  extern __shared__ double rfs[];
  double* A = rfs;
  double* X = A + n * n;
  double* R = X + n * n;
  double* U = R + n * n;
  double* S = U + n * n;
  double* lam = S + n * n;
  double* red = lam + n;  // [33]
  const int t = threadIdx.x, nn = n * n;
  for (int e = t; e < nn; e += RF_THREADS) {
    A[e] = Asym[e];
    X[e] = X0[e];
  }
  __syncthreads();
  double an = 0.0;
  for (int e = t; e < nn; e += RF_THREADS) an += A[e] * A[e];
  an = rf_block_sum(an, red);
  for (int step = 0; step < 2; ++step) {
    rf_product(n, X, true, X, R, 1.0, -1.0);  // R = I - X'X
    rf_product(n, A, false, X, U, 0.0, 1.0);  // U = A X
    rf_product(n, X, true, U, S, 0.0, 1.0);   // S = X'AX
    for (int i = t; i < n; i += RF_THREADS) lam[i] = S[i * n + i] / (1.0 - R[i * n + i]);
    double so = 0.0, rn = 0.0;
    for (int e = t; e < nn; e += RF_THREADS) {
      if (e / n != e % n) so += S[e] * S[e];
      rn += R[e] * R[e];
    }
    so = rf_block_sum(so, red);  // (the barriers inside also publish lam)
    rn = rf_block_sum(rn, red);
    const double delta = 2.0 * (sqrt(so) + sqrt(an) * sqrt(rn));
    for (int e = t; e < nn; e += RF_THREADS) {  // E into U (dead once S is formed)
      const int i = e / n, j = e - i * n;
      const double gap = lam[j] - lam[i];
      U[e] = (i == j || fabs(gap) <= delta) ? 0.5 * R[e] : (S[e] + lam[j] * R[e]) / gap;
    }
    __syncthreads();
    rf_product(n, X, false, U, S, 0.0, 1.0);  // S = X E
    for (int e = t; e < nn; e += RF_THREADS) X[e] += S[e];
    __syncthreads();
  }
  for (int e = t; e < nn; e += RF_THREADS) {
    const int i = e / n, j = e - i * n;
    Ag[e] = (i == j) ? lam[i] : 0.0;
    Vg[e] = X[e];
  }
}

// Rayleigh-Ritz eigensolver (FP32 Jacobi + two FP64 refinement steps); scratch
// holds 5 l^2 + l doubles.
fpca_status launch_jacobi_rr(fpca_ctx* ctx, int l, double* A, double* V, double* scratch) {
  const size_t nn = (size_t)l * l;
  double* As = scratch;   // symmetrised input
  double* X = As + nn;    // FP32 Jacobi eigenvectors, refined in place
  double* R = X + nn;
  double* U = R + nn;
  double* S = U + nn;
  double* lam = S + nn;
  double* E = U;  // U is dead once S is formed
  // one thread per element of a step's rotations (np pairs x l): wider blocks only
  // make the three barriers of every step dearer
  const int jt = min(1024, max(64, ((((l + 1) & ~1) / 2 * l + 31) / 32) * 32));
  k_rr_jacobi32<<<1, jt, 0, ctx->stream>>>(l, A, As, X);
  FPCA_LAUNCHED(ctx, "jacobi");
  if (l <= 32) {
    k_rr_refine<<<1, RF_THREADS, rr_refine_smem(l), ctx->stream>>>(l, As, X, A, V);
    FPCA_LAUNCHED(ctx, "jacobi");
    return FPCA_OK;
  }
  for (int step = 0; step < 2; ++step) {
    k_rr_rowmm<<<l, 64, 0, ctx->stream>>>(l, X, 1, X, R, 1.0, -1.0);   // R = I - X'X
    FPCA_LAUNCHED(ctx, "jacobi");
    k_rr_rowmm<<<l, 64, 0, ctx->stream>>>(l, As, 0, X, U, 0.0, 1.0);   // U = A X
    FPCA_LAUNCHED(ctx, "jacobi");
    k_rr_rowmm<<<l, 64, 0, ctx->stream>>>(l, X, 1, U, S, 0.0, 1.0);    // S = X' A X
    FPCA_LAUNCHED(ctx, "jacobi");
    k_rr_correction<<<1, 1024, 0, ctx->stream>>>(l, As, R, S, E, lam);
    FPCA_LAUNCHED(ctx, "jacobi");
    k_rr_update<<<l, 64, 0, ctx->stream>>>(l, X, E);
    FPCA_LAUNCHED(ctx, "jacobi");
  }
  k_rr_out<<<(int)((nn + 255) / 256), 256, 0, ctx->stream>>>(l, lam, X, A, V);
  FPCA_LAUNCHED(ctx, "jacobi");
  return FPCA_OK;
}

template <typename TS>
fpca_status launch_proj(fpca_ctx* ctx, int P, int l, const TS* S, const TS* X, TS* Y) {
  const int nb8 = (P + 7) / 8;
  const int ksplit = P >= 2048 ? 8 : 1;
  const int ksplit2 = P >= 2048 ? 2 : 1;   // (measured best for 4 rows per warp)
  cudaMemsetAsync(Y, 0, sizeof(TS) * (size_t)P * l, ctx->stream);
  if (l <= 8) {
    k_proj<TS, TS, 8, 4><<<dim3((nb8 + 3) / 4, ksplit), 256, 0, ctx->stream>>>(P, l, S, X, Y);
  } else if (l <= 20) {
    k_proj<TS, TS, 20, 4><<<dim3((nb8 + 3) / 4, ksplit2), 256, 0, ctx->stream>>>(P, l, S, X, Y);
  } else if (l <= 24) {
    k_proj<TS, TS, 24, 4><<<dim3((nb8 + 3) / 4, ksplit2), 256, 0, ctx->stream>>>(P, l, S, X, Y);
  } else if (l <= 64) {
    k_proj<TS, TS, 64, 1><<<dim3(nb8, ksplit), 256, 0, ctx->stream>>>(P, l, S, X, Y);
  } else {
    return fpca_fail(ctx, FPCA_E_UNSUPPORTED, "projection built for l <= 64");
  }
  FPCA_LAUNCHED(ctx, "proj");
  return FPCA_OK;
}

// Orthonormal basis Q of range(Y) by Cholesky QR: passes = 2 (CholeskyQR2) for the
// basis of the Rayleigh-Ritz step; one pass between power iterations, where only
// a well-conditioned basis of the range is needed.
template <typename TS>
fpca_status orth_cqr2(fpca_ctx* ctx, int P, int l, TS* Y, TS* Q, double* G, double* Rinv,
                      double* work, double* part, int passes = 2) {
  (void)work;
  for (int pass = 0; pass < passes; ++pass) {
    TS* src = pass == 0 ? Y : Q;
    fpca_status gs = launch_cross_gram<TS>(ctx, P, l, src, src, part, G, "gram");
    if (gs != FPCA_OK) return gs;
    // Rinv holds R^-1 as hi and lo parts (l <= 64)
    float* Ih = reinterpret_cast<float*>(Rinv);
    float* Il = Ih + l * l;
    cudaFuncSetAttribute(k_chol_ff, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)chol_ff_smem(l));
    k_chol_ff<<<1, CH_THREADS, chol_ff_smem(l), ctx->stream>>>(l, G, Ih, Il);
    FPCA_LAUNCHED(ctx, "chol_inv");
    const long long ne = (long long)P * l;
    k_apply_ff<TS><<<(int)((ne + 255) / 256), 256, 0, ctx->stream>>>(P, l, src, Ih, Il, Q);
    FPCA_LAUNCHED(ctx, "apply_rinv");
  }
  return FPCA_OK;
}

template <typename TG, typename TS>
fpca_status rproj_typed(fpca_ctx* ctx, const fpca_grid* g, const TG* gamma, const int32_t* domain,
                        const float* omega, int l, int k, int power_iters, int full,
                        double* evals, double* evecs, double* fve) {
  const int P = grid_P(g);
  const long long PP = (long long)P * P;
  const double dv = 1.0 / (double)P;
  const int n = full ? P : l;
  const size_t need = WsCarve::round(sizeof(TS) * PP) + WsCarve::round(sizeof(double) * 4) +
                      4 * WsCarve::round(sizeof(TS) * (size_t)P * l) +
                      3 * WsCarve::round(sizeof(double) * (size_t)l * l) +
                      2 * WsCarve::round(sizeof(double) * (size_t)n * n) +
                      WsCarve::round(sizeof(double) * 2 * n) + WsCarve::round(sizeof(int) * 3 * n) +
                      WsCarve::round(sizeof(double) * (size_t)((P + GR_ROWS - 1) / GR_ROWS) * l * l) +
                      WsCarve::round(sizeof(double) * (5 * (size_t)l * l + l)) + 4096;
  void* ws = fpca_workspace(ctx, need);
  if (!ws) return fpca_fail(ctx, FPCA_E_OOM, "workspace (%zu bytes)", need);
  WsCarve carve(ws);
  TS* S = carve.take<TS>(PP);
  double* trace = carve.take<double>(4);
  TS* Y = carve.take<TS>((size_t)P * l);
  TS* Q = carve.take<TS>((size_t)P * l);
  TS* Z = carve.take<TS>((size_t)P * l);
  TS* Om = carve.take<TS>((size_t)P * l);
  double* G = carve.take<double>((size_t)l * l);
  double* Rinv = carve.take<double>((size_t)l * l);
  double* work = carve.take<double>((size_t)l * l);
  double* A = carve.take<double>((size_t)n * n);
  double* V = carve.take<double>((size_t)n * n);
  double* cs = carve.take<double>(2 * n);
  int* pairs = carve.take<int>(2 * n);
  int* order = carve.take<int>(n);
  double* part = carve.take<double>((size_t)((P + GR_ROWS - 1) / GR_ROWS) * l * l);
  double* rrs = carve.take<double>(5 * (size_t)l * l + l);

  cudaMemsetAsync(trace, 0, sizeof(double), ctx->stream);
  k_matrixize<TG, TS><<<dim3((P + 31) / 32, (P + 31) / 32), dim3(32, 8), 0, ctx->stream>>>(
      P, gamma, domain, S, trace);
  FPCA_LAUNCHED(ctx, "matrixize");
  if (full) {
    // dense eigenpairs of Sigma (FP64 copy)
    if constexpr (sizeof(TS) == 8) {
      cudaMemcpyAsync(A, S, sizeof(double) * PP, cudaMemcpyDeviceToDevice, ctx->stream);
    } else {
      return fpca_fail(ctx, FPCA_E_UNSUPPORTED, "dense eigensolver needs FP64 gamma");
    }
    k_jacobi<<<1, 1024, 0, ctx->stream>>>(P, A, V, cs, pairs, 40);
    FPCA_LAUNCHED(ctx, "jacobi");
    k_eig_order<<<1, 1024, 0, ctx->stream>>>(P, A, order);
    FPCA_LAUNCHED(ctx, "eig_order");
    k_dense_vectors<<<(int)(((long long)P * k + 255) / 256), 256, 0, ctx->stream>>>(P, k, V, order,
                                                                                    evecs);
    FPCA_LAUNCHED(ctx, "dense_vectors");
    k_finish<<<k, 1024, 0, ctx->stream>>>(P, P, k, dv, A, order, trace, evals, evecs, fve);
    FPCA_LAUNCHED(ctx, "eig_finish");
    return FPCA_OK;
  }
  // Omega in the working type
  if constexpr (sizeof(TS) == 4) {
    cudaMemcpyAsync(Om, omega, sizeof(float) * (size_t)P * l, cudaMemcpyDeviceToDevice, ctx->stream);
  } else {
    return fpca_fail(ctx, FPCA_E_UNSUPPORTED, "random projection runs on FP32 Sigma");
  }
  fpca_status s = launch_proj<TS>(ctx, P, l, S, Om, Y);
  if (s != FPCA_OK) return s;
  for (int it = 0; it < power_iters; ++it) {
    s = orth_cqr2<TS>(ctx, P, l, Y, Q, G, Rinv, work, part, 1);
    if (s != FPCA_OK) return s;
    s = launch_proj<TS>(ctx, P, l, S, Q, Y);
    if (s != FPCA_OK) return s;
  }
  s = orth_cqr2<TS>(ctx, P, l, Y, Q, G, Rinv, work, part);
  if (s != FPCA_OK) return s;
  s = launch_proj<TS>(ctx, P, l, S, Q, Z);
  if (s != FPCA_OK) return s;
  s = launch_cross_gram<TS>(ctx, P, l, Q, Z, part, A, "ritz_gram");
  if (s != FPCA_OK) return s;
  {
    fpca_status js = launch_jacobi_rr(ctx, l, A, V, rrs);
    if (js != FPCA_OK) return js;
  }
  k_eig_order<<<1, 1024, 0, ctx->stream>>>(l, A, order);
  FPCA_LAUNCHED(ctx, "eig_order");
  k_ritz_vectors<TS><<<(P + 127) / 128, 128, 0, ctx->stream>>>(P, l, k, Q, V, order, evecs);
  FPCA_LAUNCHED(ctx, "ritz_vectors");
  k_finish<<<k, 1024, 0, ctx->stream>>>(P, l, k, dv, A, order, trace, evals, evecs, fve);
  FPCA_LAUNCHED(ctx, "eig_finish");
  return FPCA_OK;
}

}  // namespace

fpca_status rproj_eig_run(fpca_ctx* ctx, const fpca_grid* g, const void* gamma, int gamma_prec,
                          const int32_t* domain, const float* omega, int l, int k,
                          int power_iters, int full, double* evals, double* evecs,
                          double* fve) {
  if (full) {
    if (gamma_prec == FPCA_F64)
      return rproj_typed<double, double>(ctx, g, static_cast<const double*>(gamma), domain, omega,
                                         l, k, power_iters, 1, evals, evecs, fve);
    return fpca_fail(ctx, FPCA_E_UNSUPPORTED, "dense eigensolver needs FP64 gamma");
  }
  if (gamma_prec == FPCA_F64)
    return rproj_typed<double, float>(ctx, g, static_cast<const double*>(gamma), domain, omega, l,
                                      k, power_iters, 0, evals, evecs, fve);
  return rproj_typed<float, float>(ctx, g, static_cast<const float*>(gamma), domain, omega, l, k,
                                   power_iters, 0, evals, evecs, fve);
}

// ---------------------------------------------------------------------------
// Random projection of Section 3.4 on an operator: the covariance matrix is
// never formed, only its products Y = Sigma X (P x l, FP32, row-major) through
// op.apply.  The steps are those of the dense path above: range finder with
// CholeskyQR2 and power iterations, Rayleigh-Ritz in FP64, rescaling and FVE
// (trace of Sigma supplied by the caller in ws.trace[0], unscaled).
// ---------------------------------------------------------------------------
size_t rproj_ws_bytes(int P, int l) {
  return 3 * WsCarve::round(sizeof(float) * (size_t)P * l) +
         5 * WsCarve::round(sizeof(double) * (size_t)l * l) + WsCarve::round(sizeof(double) * 4) +
         WsCarve::round(sizeof(int) * 3 * (size_t)l) +
         WsCarve::round(sizeof(double) * (size_t)((P + GR_ROWS - 1) / GR_ROWS) * l * l) +
         WsCarve::round(sizeof(double) * (5 * (size_t)l * l + l)) + 2048;
}

void rproj_ws_carve(WsCarve& c, int P, int l, RprojWs& w) {
  w.Y = c.take<float>((size_t)P * l);
  w.Q = c.take<float>((size_t)P * l);
  w.Z = c.take<float>((size_t)P * l);
  w.G = c.take<double>((size_t)l * l);
  w.Rinv = c.take<double>((size_t)l * l);
  w.work = c.take<double>((size_t)l * l);
  w.A = c.take<double>((size_t)l * l);
  w.V = c.take<double>((size_t)l * l);
  w.trace = c.take<double>(4);
  w.order = c.take<int>(3 * (size_t)l);
  w.part = c.take<double>((size_t)((P + GR_ROWS - 1) / GR_ROWS) * l * l);
  w.rr = c.take<double>(5 * (size_t)l * l + l);
}

fpca_status rproj_operator(fpca_ctx* ctx, int P, int l, int k, int power_iters, double dv,
                           const float* omega, RprojOp op, const RprojWs& w, double* evals,
                           double* evecs, double* fve) {
  fpca_status s = op.apply(op.self, omega, w.Y);
  if (s != FPCA_OK) return s;
  for (int it = 0; it < power_iters; ++it) {
    s = orth_cqr2<float>(ctx, P, l, w.Y, w.Q, w.G, w.Rinv, w.work, w.part, 1);
    if (s != FPCA_OK) return s;
    s = op.apply(op.self, w.Q, w.Y);
    if (s != FPCA_OK) return s;
  }
  s = orth_cqr2<float>(ctx, P, l, w.Y, w.Q, w.G, w.Rinv, w.work, w.part);
  if (s != FPCA_OK) return s;
  s = op.apply(op.self, w.Q, w.Z);
  if (s != FPCA_OK) return s;
  s = launch_cross_gram<float>(ctx, P, l, w.Q, w.Z, w.part, w.A, "ritz_gram");
  if (s != FPCA_OK) return s;
  s = launch_jacobi_rr(ctx, l, w.A, w.V, w.rr);
  if (s != FPCA_OK) return s;
  k_eig_order<<<1, 1024, 0, ctx->stream>>>(l, w.A, w.order);
  FPCA_LAUNCHED(ctx, "eig_order");
  k_ritz_vectors<float><<<(P + 127) / 128, 128, 0, ctx->stream>>>(P, l, k, w.Q, w.V, w.order,
                                                                   evecs);
  FPCA_LAUNCHED(ctx, "ritz_vectors");
  k_finish<<<k, 1024, 0, ctx->stream>>>(P, l, k, dv, w.A, w.order, w.trace, evals, evecs, fve);
  FPCA_LAUNCHED(ctx, "eig_finish");
  return FPCA_OK;
}
