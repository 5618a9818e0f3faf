// Eigen step: matrixisation (Section 3.1, Eq. 3.1) and the random projection
// of Section 3.4 (range finder with power iterations and Rayleigh-Ritz).
//
//  Sigma    = (G + G')/2, NaN -> 0, rows/columns outside the domain -> 0
//  Y        = Sigma Omega;  repeat q times { Q = orth(Y); Y = Sigma Q }
//  Q        = orth(Y) by CholeskyQR2 (FP64 Gram and Cholesky)
//  B        = Q' Sigma Q (FP64), eigenpairs of B by cyclic Jacobi (FP64)
//  Psi      = Q U;  lambda = theta dV;  phi = psi / sqrt(dV);  dV = 1/P
// The dense path (full = 1) runs the same Jacobi solver on Sigma itself.
#include <cmath>

#include "fpca_internal.cuh"

namespace {

template <typename TG>
__device__ __forceinline__ double gval(const TG* G, long long idx) {
  const double x = (double)G[idx];
  return isnan(x) ? 0.0 : x;
}

// Sigma = sym(G) with NaN and out-of-domain entries zeroed; trace accumulated.
template <typename TG, typename TS>
__global__ void k_matrixize(int P, const TG* __restrict__ G, const int32_t* __restrict__ dom,
                            TS* __restrict__ S, double* __restrict__ trace) {
  __shared__ double tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  // transposed tile: rows q in [bx, bx+32), columns p in [by, by+32)
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int q = bx + r, p = by + threadIdx.x;
    tile[r][threadIdx.x] = (q < P && p < P) ? gval(G, (long long)q * P + p) : 0.0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int p = by + r, q = bx + threadIdx.x;
    if (p < P && q < P) {
      double s = 0.5 * (gval(G, (long long)p * P + q) + tile[threadIdx.x][r]);
      if (dom && (dom[p] <= 0 || dom[q] <= 0)) s = 0.0;
      S[(long long)p * P + q] = (TS)s;
      if (p == q) atomicAdd(trace, s);
    }
  }
}

// Y (P x l) = S (P x P) X (P x l): a warp per RPW rows, lanes stride over the
// columns of S, X staged in shared memory in chunks of QCH rows.
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
  for (int q0 = 0; q0 < P; q0 += QCH) {
    __syncthreads();
    for (int e = threadIdx.x; e < QCH * LM; e += 256) {
      const int qq = e / LM, c = e - qq * LM;
      xs[qq * LP + c] = (q0 + qq < P && c < l) ? X[(long long)(q0 + qq) * l + c] : TX(0);
    }
    __syncthreads();
#pragma unroll 2
    for (int t = lane; t < QCH; t += 32) {
      const int q = q0 + t;
      if (q >= P) break;
      TX sv[RPW];
#pragma unroll
      for (int r = 0; r < RPW; ++r)
        sv[r] = (row0 + r < P) ? (TX)S[(long long)(row0 + r) * P + q] : TX(0);
#pragma unroll
      for (int c = 0; c < LM; ++c) {
        const TX xv = xs[t * LP + c];
#pragma unroll
        for (int r = 0; r < RPW; ++r) acc[r][c] = fma(sv[r], xv, acc[r][c]);
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
          if (c < l) Y[(long long)(row0 + r) * l + c] = acc[r][c];
      }
  }
}

// G (l x l, FP64) += A' B over a chunk of rows (A, B: P x l).
template <typename TX>
__global__ void k_cross_gram(int P, int l, const TX* __restrict__ A, const TX* __restrict__ B,
                             double* __restrict__ G) {
  const int rows_per_block = 64;
  const int r0 = blockIdx.x * rows_per_block;
  const int r1 = min(P, r0 + rows_per_block);
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) {
    const int i = e / l, j = e - (e / l) * l;
    double s = 0.0;
    for (int r = r0; r < r1; ++r) s += (double)A[(long long)r * l + i] * (double)B[(long long)r * l + j];
    atomicAdd(G + e, s);
  }
}

// Upper Cholesky G = R'R (one thread; l <= 128) and Rinv; rank-deficient
// directions (pivot <= 1e-13 of the largest diagonal) get a zero column.
__global__ void k_chol_inv(int l, const double* __restrict__ G, double* __restrict__ Rinv,
                           double* __restrict__ work) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double* R = work;  // l x l
  double dmax = 0.0;
  for (int i = 0; i < l; ++i) dmax = fmax(dmax, G[i * l + i]);
  for (int i = 0; i < l * l; ++i) R[i] = 0.0;
  for (int j = 0; j < l; ++j) {
    double s = G[j * l + j];
    for (int k = 0; k < j; ++k) s -= R[k * l + j] * R[k * l + j];
    if (!(s > 1e-13 * dmax)) {
      R[j * l + j] = 0.0;  // dropped direction
      continue;
    }
    const double rjj = sqrt(s);
    R[j * l + j] = rjj;
    for (int i = j + 1; i < l; ++i) {
      double t = G[j * l + i];
      for (int k = 0; k < j; ++k) t -= R[k * l + j] * R[k * l + i];
      R[j * l + i] = t / rjj;
    }
  }
  // Rinv: upper triangular inverse, zero rows/columns for dropped directions
  for (int i = 0; i < l * l; ++i) Rinv[i] = 0.0;
  for (int j = 0; j < l; ++j) {
    if (R[j * l + j] == 0.0) continue;
    Rinv[j * l + j] = 1.0 / R[j * l + j];
    for (int i = j - 1; i >= 0; --i) {
      if (R[i * l + i] == 0.0) continue;
      double s = 0.0;
      for (int k = i + 1; k <= j; ++k) s += R[i * l + k] * Rinv[k * l + j];
      Rinv[i * l + j] = -s / R[i * l + i];
    }
  }
}

// Q = Y Rinv (row-wise).
template <typename TX>
__global__ void k_apply_rinv(int P, int l, const TX* __restrict__ Y, const double* __restrict__ Rinv,
                             TX* __restrict__ Q) {
  extern __shared__ double rs[];
  for (int e = threadIdx.x; e < l * l; e += blockDim.x) rs[e] = Rinv[e];
  __syncthreads();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= P) return;
  double yr[128];
  for (int i = 0; i < l; ++i) yr[i] = (double)Y[(long long)r * l + i];
  for (int j = 0; j < l; ++j) {
    double s = 0.0;
    for (int i = 0; i <= j; ++i) s += yr[i] * rs[i * l + j];
    Q[(long long)r * l + j] = (TX)s;
  }
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
      done = (off_tot <= 1e-30 * s) || off_tot == 0.0;
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

template <typename TS>
fpca_status launch_proj(fpca_ctx* ctx, int P, int l, const TS* S, const TS* X, TS* Y) {
  const int nb8 = (P + 7) / 8;
  if (l <= 8) {
    k_proj<TS, TS, 8, 4><<<(nb8 + 3) / 4, 256, 0, ctx->stream>>>(P, l, S, X, Y);
  } else if (l <= 24) {
    k_proj<TS, TS, 24, 2><<<(nb8 + 1) / 2, 256, 0, ctx->stream>>>(P, l, S, X, Y);
  } else if (l <= 64) {
    k_proj<TS, TS, 64, 1><<<nb8, 256, 0, ctx->stream>>>(P, l, S, X, Y);
  } else {
    return fpca_fail(ctx, FPCA_E_UNSUPPORTED, "projection built for l <= 64");
  }
  FPCA_LAUNCHED(ctx, "proj");
  return FPCA_OK;
}

template <typename TS>
fpca_status orth_cqr2(fpca_ctx* ctx, int P, int l, TS* Y, TS* Q, double* G, double* Rinv,
                      double* work) {
  for (int pass = 0; pass < 2; ++pass) {
    TS* src = pass == 0 ? Y : Q;
    cudaMemsetAsync(G, 0, sizeof(double) * l * l, ctx->stream);
    k_cross_gram<TS><<<(P + 63) / 64, 256, 0, ctx->stream>>>(P, l, src, src, G);
    FPCA_LAUNCHED(ctx, "gram");
    k_chol_inv<<<1, 32, 0, ctx->stream>>>(l, G, Rinv, work);
    FPCA_LAUNCHED(ctx, "chol_inv");
    k_apply_rinv<TS><<<(P + 127) / 128, 128, sizeof(double) * l * l, ctx->stream>>>(P, l, src, Rinv, Q);
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
                      4096;
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
    s = orth_cqr2<TS>(ctx, P, l, Y, Q, G, Rinv, work);
    if (s != FPCA_OK) return s;
    s = launch_proj<TS>(ctx, P, l, S, Q, Y);
    if (s != FPCA_OK) return s;
  }
  s = orth_cqr2<TS>(ctx, P, l, Y, Q, G, Rinv, work);
  if (s != FPCA_OK) return s;
  s = launch_proj<TS>(ctx, P, l, S, Q, Z);
  if (s != FPCA_OK) return s;
  cudaMemsetAsync(A, 0, sizeof(double) * l * l, ctx->stream);
  k_cross_gram<TS><<<(P + 63) / 64, 256, 0, ctx->stream>>>(P, l, Q, Z, A);
  FPCA_LAUNCHED(ctx, "ritz_gram");
  k_jacobi<<<1, 1024, 0, ctx->stream>>>(l, A, V, cs, pairs, 60);
  FPCA_LAUNCHED(ctx, "jacobi");
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
