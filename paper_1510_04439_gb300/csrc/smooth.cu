// Local linear smoothing of binned data: the mean, Eq. (2.3), and the
// covariance surface, Eq. (2.4), with the product Epanechnikov kernel.
//
// At an output bin centre x the fit solves A beta = r with
//   A = sum_b K(u_b) W_b z_b z_b',  r = sum_b K(u_b) V_b z_b,
//   z_b = [1, u_b],  u_b = (c_b - x)/h (per axis),
// and returns beta_0 (the 1/h factors of K_h cancel in beta_0).  For the
// covariance, b runs over bin pairs (p, q), z = [1, u_s, u_t] has 2d + 1
// entries and the kernel is K(u_s) K(u_t).
//
// Covariance moments.  The product kernel makes every entry of A and r a
// separable sum over the 2d axes: S_alpha = sum K W prod u^alpha (|alpha| <= 2)
// and T_alpha = sum K V prod u^alpha (|alpha| <= 1).  The P x P bin arrays
// (row = s node, column = t node) are swept in three stages:
//   1. vertical pass along s_d (rows within one s_1 block), coalesced over t,
//   2. vertical pass along s_1,
//   3. per output row x_s: the t-side 2-D sweep (t_1 across rows of the
//      t-plane, then t_2 along them) in shared memory, the per-point
//      (2d+1) x (2d+1) solve in registers, and the write of Gamma_hat.
// A box-filter pass of the indicator [count > 0] runs alongside and gives
// the number of non-empty bin pairs in each window.
#include <algorithm>
#include <cmath>

#include "fpca_internal.cuh"

namespace {

constexpr int TMAX = 63;          // largest tap offset supported (m <= 64)
constexpr int TW = 2 * TMAX + 1;  // table width
constexpr int TROWS = 4;          // K, K u, K u^2, box (1 inside the support)

// Thresholds of the per-point status rules.
constexpr double PIVOT_RTOL_F64 = 1e-9;  // FP64 moments: fallback at or below
constexpr double PIVOT_RTOL_F32 = 1e-5;  // FP32 moments: fallback at or below
constexpr double ESCALATE_F32 = 1e-2;    // FP32 solve redone in FP64 below this

struct TapParams {
  int d;
  int m[3];
  double h[3];
};

// tab[k][row][t + TMAX]: weights of axis k at bin offset t, u = t / (h_k M_k).
__global__ void k_taps(TapParams tp, double* __restrict__ tab) {
  const int k = blockIdx.x;
  for (int t = threadIdx.x; t < TW; t += blockDim.x) {
    const double off = (double)(t - TMAX);
    const double hm = __dmul_rn(tp.h[k], (double)tp.m[k]);
    const double u = __ddiv_rn(off, hm);
    const bool in = fabs(u) < 1.0 && fabs(off) < (double)tp.m[k];
    const double K = in ? __dmul_rn(0.75, __dsub_rn(1.0, __dmul_rn(u, u))) : 0.0;
    double* base = tab + (size_t)k * TROWS * TW;
    base[0 * TW + t] = K;
    base[1 * TW + t] = __dmul_rn(K, u);
    base[2 * TW + t] = __dmul_rn(K, __dmul_rn(u, u));
    base[3 * TW + t] = in ? 1.0 : 0.0;
  }
}

// Largest offset j < M with j / (h M) < 1 (same double arithmetic as the tables).
int host_taps(double h, int M) {
  const double hm = h * (double)M;
  for (int j = M - 1; j >= 1; --j)
    if ((double)j / hm < 1.0) return j;
  return 0;
}

// ---------------------------------------------------------------------------
// natural-order symmetric elimination: beta_0 and the smallest pivot ratio
// (Schur-complement diagonal / original diagonal), i.e. the Cholesky pivots
// ---------------------------------------------------------------------------
template <int D, typename T>
__device__ __forceinline__ T elim_solve(T (&A)[D][D], T (&r)[D], double& minratio) {
  T diag[D];
#pragma unroll
  for (int i = 0; i < D; ++i) diag[i] = A[i][i];
  minratio = 1e300;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const T piv = A[k][k];
    const double ratio = diag[k] > T(0) ? (double)piv / (double)diag[k] : -1.0;
    minratio = fmin(minratio, ratio);
    if (!(piv > T(0))) {
      minratio = -1.0;
      return T(0);
    }
    const T inv = T(1) / piv;
#pragma unroll
    for (int i = k + 1; i < D; ++i) {
      const T l = A[k][i] * inv;
#pragma unroll
      for (int j = i; j < D; ++j) A[i][j] -= l * A[k][j];
      r[i] -= l * r[k];
    }
  }
  T x[D];
#pragma unroll
  for (int k = D - 1; k >= 0; --k) {
    T s = r[k];
#pragma unroll
    for (int j = k + 1; j < D; ++j) s -= A[k][j] * x[j];
    x[k] = s / A[k][k];
  }
  return x[0];
}

// Status and value of one local fit from its normal equations (in T) and the
// number of non-empty bins in the window.
template <int D, typename T>
__device__ __forceinline__ double fit_point(T (&A)[D][D], T (&r)[D], double nonempty,
                                            uint8_t& st) {
  if (!(A[0][0] > T(0))) {
    st = FPCA_PT_EMPTY;
    return __longlong_as_double(0x7ff8000000000000ll);
  }
  const double lc = (double)r[0] / (double)A[0][0];
  if (nonempty < (double)D) {
    st = FPCA_PT_FALLBACK;
    return lc;
  }
  if constexpr (sizeof(T) == 8) {
    double ratio;
    const double b = elim_solve<D, T>(A, r, ratio);
    if (ratio <= PIVOT_RTOL_F64) {
      st = FPCA_PT_FALLBACK;
      return lc;
    }
    st = FPCA_PT_OK;
    return b;
  } else {
    double Ad[D][D], rd[D];
#pragma unroll
    for (int i = 0; i < D; ++i) {
      rd[i] = (double)r[i];
#pragma unroll
      for (int j = 0; j < D; ++j) Ad[i][j] = (double)A[i][j];
    }
    double ratio;
    const T b = elim_solve<D, T>(A, r, ratio);
    if (ratio >= ESCALATE_F32) {
      st = FPCA_PT_OK;
      return (double)b;
    }
    const double bd = elim_solve<D, double>(Ad, rd, ratio);
    if (ratio <= PIVOT_RTOL_F32) {
      st = FPCA_PT_FALLBACK;
      return lc;
    }
    st = FPCA_PT_OK;
    return bd;
  }
}

// ---------------------------------------------------------------------------
// mean smoother, Eq. (2.3): one thread per output node, FP64 window sums
// ---------------------------------------------------------------------------
template <int DIM>
__global__ void k_smooth_mean(int P, TapParams tp, const double* __restrict__ tab,
                              const int32_t* __restrict__ cnt, const double* __restrict__ w,
                              const double* __restrict__ v, double* __restrict__ mu,
                              uint8_t* __restrict__ status, int T0, int T1, int T2) {
  constexpr int D = DIM + 1;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  int j[3] = {0, 0, 0};
  {
    int rem = p;
    for (int k = DIM - 1; k >= 0; --k) {
      j[k] = rem % tp.m[k];
      rem /= tp.m[k];
    }
  }
  const int taps[3] = {T0, T1, T2};
  double A[D][D], r[D];
#pragma unroll
  for (int a = 0; a < D; ++a) {
    r[a] = 0.0;
#pragma unroll
    for (int b = 0; b < D; ++b) A[a][b] = 0.0;
  }
  double nonempty = 0.0;
  int lo[3], hi[3];
  for (int k = 0; k < 3; ++k) {
    lo[k] = 0;
    hi[k] = 0;
  }
  for (int k = 0; k < DIM; ++k) {
    lo[k] = max(-taps[k], -j[k]);
    hi[k] = min(taps[k], tp.m[k] - 1 - j[k]);
  }
  for (int o0 = lo[0]; o0 <= hi[0]; ++o0)
    for (int o1 = lo[1]; o1 <= hi[1]; ++o1)
      for (int o2 = lo[2]; o2 <= hi[2]; ++o2) {
        const int off[3] = {o0, o1, o2};
        int b = 0;
        double K = 1.0;
        double u[3];
#pragma unroll
        for (int k = 0; k < DIM; ++k) {
          b = b * tp.m[k] + (j[k] + off[k]);
          const double* tk = tab + (size_t)k * TROWS * TW;
          K *= tk[off[k] + TMAX];
          u[k] = __ddiv_rn((double)off[k], __dmul_rn(tp.h[k], (double)tp.m[k]));
        }
        if (K == 0.0) continue;
        const double kw = K * w[b], kv = K * v[b];
        nonempty += cnt[b] > 0 ? 1.0 : 0.0;
        double z[D];
        z[0] = 1.0;
#pragma unroll
        for (int k = 0; k < DIM; ++k) z[k + 1] = u[k];
#pragma unroll
        for (int a = 0; a < D; ++a) {
          r[a] += kv * z[a];
#pragma unroll
          for (int c = a; c < D; ++c) A[a][c] += kw * z[a] * z[c];
        }
      }
#pragma unroll
  for (int a = 0; a < D; ++a)
#pragma unroll
    for (int c = 0; c < a; ++c) A[a][c] = A[c][a];
  uint8_t st;
  mu[p] = fit_point<D, double>(A, r, nonempty, st);
  if (status) status[p] = st;
}

// ---------------------------------------------------------------------------
// covariance: moment bookkeeping
// ---------------------------------------------------------------------------
// Arrays after the s-side passes (d = 2): W with s-exponents (s1,s2) =
// (0,0) (1,0) (2,0) (0,1) (1,1) (0,2); V with (0,0) (1,0) (0,1); the
// indicator.  Moment slots: S over exponents (s1,s2,t1,t2) with |e| <= 2 in
// the order 1, s1, s2, t1, t2, s1s1, s1s2, s1t1, s1t2, s2s2, s2t1, s2t2,
// t1t1, t1t2, t2t2 (0..14); T with |e| <= 1: 1, s1, s2, t1, t2 (15..19);
// the non-empty count (20).
__host__ __device__ constexpr int narr(int d) { return d == 2 ? 10 : 6; }
__host__ __device__ constexpr int nslot(int d) { return d == 2 ? 21 : 10; }
// largest t-degree of array a
__host__ __device__ constexpr int maxdeg(int d, int a) {
  return d == 2 ? (a == 0 ? 2 : (a == 1 || a == 3 || a == 6) ? 1 : 0)
                : (a == 0 ? 2 : (a == 1 || a == 3) ? 1 : 0);
}
__host__ __device__ constexpr bool is_indicator(int d, int a) { return a == narr(d) - 1; }
// slot of t-exponents (a1 across t-plane rows, a2 along them) of array a
__host__ __device__ constexpr int slot_of(int d, int a, int a1, int a2) {
  if (d == 2) {
    switch (a * 9 + a1 * 3 + a2) {
      case 0 * 9 + 0: return 0;
      case 0 * 9 + 1: return 4;
      case 0 * 9 + 2: return 14;
      case 0 * 9 + 3: return 3;
      case 0 * 9 + 4: return 13;
      case 0 * 9 + 6: return 12;
      case 1 * 9 + 0: return 1;
      case 1 * 9 + 1: return 8;
      case 1 * 9 + 3: return 7;
      case 2 * 9 + 0: return 5;
      case 3 * 9 + 0: return 2;
      case 3 * 9 + 1: return 11;
      case 3 * 9 + 3: return 10;
      case 4 * 9 + 0: return 6;
      case 5 * 9 + 0: return 9;
      case 6 * 9 + 0: return 15;
      case 6 * 9 + 1: return 19;
      case 6 * 9 + 3: return 18;
      case 7 * 9 + 0: return 16;
      case 8 * 9 + 0: return 17;
      case 9 * 9 + 0: return 20;
      default: return -1;
    }
  }
  // d = 1: arrays W s^0, W s^1, W s^2, V s^0, V s^1, indicator; a1 is always 0
  switch (a * 3 + a2) {
    case 0 * 3 + 0: return 0;
    case 0 * 3 + 1: return 2;
    case 0 * 3 + 2: return 5;
    case 1 * 3 + 0: return 1;
    case 1 * 3 + 1: return 4;
    case 2 * 3 + 0: return 3;
    case 3 * 3 + 0: return 6;
    case 3 * 3 + 1: return 8;
    case 4 * 3 + 0: return 7;
    case 5 * 3 + 0: return 9;
    default: return -1;
  }
}
// slot of normal-matrix entry (i, j), i <= j (unknown order [1, s.., t..])
__host__ __device__ constexpr int aslot(int d, int i, int j) {
  return d == 2 ? (i == 0 ? j : i == 1 ? 4 + j : i == 2 ? 7 + j : i == 3 ? 9 + j : 14)
                : (i == 0 ? j : i == 1 ? 2 + j : 5);
}
__host__ __device__ constexpr int rslot(int d, int i) { return d == 2 ? 15 + i : 6 + i; }

template <typename T, bool COMP>
__device__ __forceinline__ void kadd(T& s, T& c, T w, T x) {
  if constexpr (COMP) {
    const T y = fma(w, x, -c);
    const T t = s + y;
    c = (t - s) - y;
    s = t;
  } else {
    s = fma(w, x, s);
  }
}

// ---------------------------------------------------------------------------
// vertical pass: 1-D sums along the row index of P x P arrays
// ---------------------------------------------------------------------------
// One input array per job; the value read is in[e] - sub[e] (sub may be
// NULL), or for counts the indicator [in[e] - sub[e] > 0].  Subtracting a
// fold's bins from the pooled bins gives the training bins of that fold.
struct VJob {
  const void* in;
  const void* sub;
  int in_int;       // 1: int32 counts read as the indicator
  int npow;         // outputs
  int row[3];       // table rows used (0 K, 1 K u, 2 K u^2, 3 box)
  void* out[3];
};
struct VJobs {
  VJob j[6];
};

constexpr int VCOLS = 128;

// Line L holds rows base + a*stride, a = 0..Ma-1, base = (L/stride)*Ma*stride + L%stride.
template <typename T, bool COMP>
__global__ void __launch_bounds__(VCOLS)
    k_vpass(VJobs jobs, int P, int Ma, int stride, int taps, const double* __restrict__ tab) {
  extern __shared__ unsigned char vsm[];
  T* wt = reinterpret_cast<T*>(vsm);   // [TROWS][TW]
  T* tile = wt + TROWS * TW;           // [Ma][VCOLS]
  const VJob& jb = jobs.j[blockIdx.z];
  for (int i = threadIdx.x; i < TROWS * TW; i += VCOLS) wt[i] = (T)tab[i];
  const int col = blockIdx.x * VCOLS + threadIdx.x;
  const int L = blockIdx.y;
  const long long base = (long long)(L / stride) * Ma * stride + (L % stride);
  for (int a = 0; a < Ma; ++a) {
    const long long row = base + (long long)a * stride;
    T val = T(0);
    if (col < P) {
      const long long e = row * P + col;
      if (jb.in_int) {
        int c = static_cast<const int32_t*>(jb.in)[e];
        if (jb.sub) c -= static_cast<const int32_t*>(jb.sub)[e];
        val = c > 0 ? T(1) : T(0);
      } else {
        val = static_cast<const T*>(jb.in)[e];
        if (jb.sub) val -= static_cast<const T*>(jb.sub)[e];
      }
    }
    tile[a * VCOLS + threadIdx.x] = val;
  }
  __syncthreads();
  if (col >= P) return;
  for (int x = 0; x < Ma; ++x) {
    const int lo = max(-taps, -x), hi = min(taps, Ma - 1 - x);
    T s0 = 0, s1 = 0, s2 = 0, c0 = 0, c1 = 0, c2 = 0;
    const T* w0 = wt + jb.row[0] * TW + TMAX;
    const T* w1 = wt + jb.row[jb.npow > 1 ? 1 : 0] * TW + TMAX;
    const T* w2 = wt + jb.row[jb.npow > 2 ? 2 : 0] * TW + TMAX;
    if (jb.npow == 3) {
      for (int k = lo; k <= hi; ++k) {
        const T vv = tile[(x + k) * VCOLS + threadIdx.x];
        kadd<T, COMP>(s0, c0, w0[k], vv);
        kadd<T, COMP>(s1, c1, w1[k], vv);
        kadd<T, COMP>(s2, c2, w2[k], vv);
      }
    } else if (jb.npow == 2) {
      for (int k = lo; k <= hi; ++k) {
        const T vv = tile[(x + k) * VCOLS + threadIdx.x];
        kadd<T, COMP>(s0, c0, w0[k], vv);
        kadd<T, COMP>(s1, c1, w1[k], vv);
      }
    } else {
      for (int k = lo; k <= hi; ++k) {
        const T vv = tile[(x + k) * VCOLS + threadIdx.x];
        kadd<T, COMP>(s0, c0, w0[k], vv);
      }
    }
    const long long o = (base + (long long)x * stride) * P + col;
    static_cast<T*>(jb.out[0])[o] = s0;
    if (jb.npow > 1) static_cast<T*>(jb.out[1])[o] = s1;
    if (jb.npow > 2) static_cast<T*>(jb.out[2])[o] = s2;
  }
}

// ---------------------------------------------------------------------------
// horizontal t-side sweep + per-point solve + epilogues
// ---------------------------------------------------------------------------
// Optional outputs besides Gamma_hat and status:
//  y += G Omega   (row x_s of y gets sum_t G(x_s, t) Omega(t, :); EMPTY = 0)
//  cv terms of one fold f: err = sum (Q_f - 2 G V_f + G^2 W_f) and w_in =
//  sum W_f over non-EMPTY points, w_out = sum W_f over EMPTY points.
template <typename T>
struct Epilogue {
  const float* omega;  // P x l or NULL
  int l;
  float* y;            // P x l (accumulated with atomics)
  const T* wf;         // held-out fold's bins (P x P) or NULL
  const T* vf;
  const T* qf;
  double* cvacc;       // [3]: err, w_in, w_out
};

constexpr int MAXL = 64;

template <int NT>
__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < NT / 32; ++w) s += red[w];
  __syncthreads();
  return s;
}

// Block: output row x_s (blockIdx.y), t-plane rows [a0, a0 + th) (blockIdx.x).
// The t-plane of row x_s is R rows x C columns (d = 2: t1 x t2; d = 1: 1 x t1).
template <int d, typename T, bool COMP, int NT, int PPT>
__global__ void __launch_bounds__(NT)
    k_hpass_solve(const T* __restrict__ varr, int P, int R, int C, int TH, int Tr, int Tc,
                  const double* __restrict__ tabr, const double* __restrict__ tabc,
                  const double* __restrict__ mu_raw, T* __restrict__ gamma,
                  uint8_t* __restrict__ status, Epilogue<T> ep) {
  constexpr int NA = narr(d), NS = nslot(d), D = 2 * d + 1;
  extern __shared__ unsigned char hsm[];
  __shared__ double red[NT / 32];
  T* wr = reinterpret_cast<T*>(hsm);       // [TROWS][TW]
  T* wc = wr + TROWS * TW;                 // [TROWS][TW]
  const int xs = blockIdx.y;
  const int a0 = blockIdx.x * TH;
  const int th = min(TH, R - a0);
  const int r0 = max(0, a0 - Tr), r1 = min(R, a0 + th + Tr);
  const int nr = r1 - r0;
  T* in = wc + TROWS * TW;                 // [NA][nr][C]
  T* mid = in + (size_t)NA * nr * C;       // [3][th][C]
  for (int i = threadIdx.x; i < TROWS * TW; i += NT) {
    wr[i] = (T)tabr[i];
    wc[i] = (T)tabc[i];
  }
  const long long PP = (long long)P * P;
  for (int a = 0; a < NA; ++a) {
    const T* src = varr + a * PP + (long long)xs * P + (long long)r0 * C;
    T* dst = in + (size_t)a * nr * C;
    for (int e = threadIdx.x; e < nr * C; e += NT) dst[e] = src[e];
  }
  __syncthreads();

  const int npts = th * C;
  T acc[PPT][NS];
#pragma unroll
  for (int j = 0; j < PPT; ++j)
#pragma unroll
    for (int s = 0; s < NS; ++s) acc[j][s] = T(0);

#pragma unroll
  for (int a = 0; a < NA; ++a) {
    const int md = maxdeg(d, a);
    const bool box = is_indicator(d, a);
    const T* ina = in + (size_t)a * nr * C;
    if constexpr (d == 2) {
      // pass across t-plane rows (t1): mid[a1][i][c]
      for (int e = threadIdx.x; e < npts; e += NT) {
        const int i = e / C, c = e - (e / C) * C;
        const int xr = a0 + i;
        const int lo = max(-Tr, -xr), hi = min(Tr, R - 1 - xr);
        const T* col = ina + (size_t)(xr - r0) * C + c;
#pragma unroll
        for (int a1 = 0; a1 < 3; ++a1) {
          if (a1 > md) break;
          const T* w = wr + (box ? 3 : a1) * TW + TMAX;
          T s = 0, cmp = 0;
          for (int k = lo; k <= hi; ++k) kadd<T, COMP>(s, cmp, w[k], col[k * C]);
          mid[(size_t)a1 * npts + e] = s;
        }
      }
      __syncthreads();
    }
    // pass along t-plane rows (t2 for d = 2, t1 for d = 1) for own points
#pragma unroll
    for (int j = 0; j < PPT; ++j) {
      const int e = threadIdx.x + j * NT;
      if (e < npts) {
        const int i = e / C, c = e - (e / C) * C;
        const int lo = max(-Tc, -c), hi = min(Tc, C - 1 - c);
#pragma unroll
        for (int a1 = 0; a1 < 3; ++a1) {
#pragma unroll
          for (int a2 = 0; a2 < 3; ++a2) {
            const int slot = slot_of(d, a, a1, a2);
            if (slot < 0) continue;
            const T* rowp = (d == 2) ? mid + (size_t)a1 * npts + (size_t)i * C
                                     : ina + (size_t)(a0 + i - r0) * C;
            const T* w = wc + (box ? 3 : a2) * TW + TMAX;
            T s = 0, cmp = 0;
            for (int k = lo; k <= hi; ++k) kadd<T, COMP>(s, cmp, w[k], rowp[c + k]);
            acc[j][slot] = s;
          }
        }
      }
    }
    if constexpr (d == 2) __syncthreads();
  }

  // per-point solve, write, epilogue terms
  double gval[PPT];
  int xts[PPT];
  double cv_err = 0.0, cv_in = 0.0, cv_out = 0.0;
#pragma unroll
  for (int j = 0; j < PPT; ++j) {
    const int e = threadIdx.x + j * NT;
    gval[j] = 0.0;
    xts[j] = -1;
    if (e >= npts) continue;
    const int xt = a0 * C + e;  // flat t index: (a0 + i) * C + c
    T A[D][D], rv[D];
#pragma unroll
    for (int i2 = 0; i2 < D; ++i2) {
      rv[i2] = acc[j][rslot(d, i2)];
#pragma unroll
      for (int j2 = i2; j2 < D; ++j2) {
        A[i2][j2] = acc[j][aslot(d, i2, j2)];
        A[j2][i2] = A[i2][j2];
      }
    }
    uint8_t st;
    double g = fit_point<D, T>(A, rv, (double)acc[j][NS - 1] + 0.25, st);
    if (mu_raw && st != FPCA_PT_EMPTY) g -= mu_raw[xs] * mu_raw[xt];
    const long long o = (long long)xs * P + xt;
    if (gamma) gamma[o] = (T)g;
    if (status) status[o] = st;
    xts[j] = xt;
    gval[j] = st == FPCA_PT_EMPTY ? 0.0 : g;
    if (ep.cvacc) {
      const double wf = (double)ep.wf[o];
      if (st == FPCA_PT_EMPTY) {
        cv_out += wf;
      } else {
        cv_err += (double)ep.qf[o] - 2.0 * g * (double)ep.vf[o] + g * g * wf;
        cv_in += wf;
      }
    }
  }
  if (ep.cvacc) {
    const double s0 = block_sum<NT>(cv_err, red);
    const double s1 = block_sum<NT>(cv_in, red);
    const double s2 = block_sum<NT>(cv_out, red);
    if (threadIdx.x == 0) {
      atomicAdd(ep.cvacc + 0, s0);
      atomicAdd(ep.cvacc + 1, s1);
      atomicAdd(ep.cvacc + 2, s2);
    }
  }
  if (ep.y) {
    for (int c = 0; c < ep.l; ++c) {
      double s = 0.0;
#pragma unroll
      for (int j = 0; j < PPT; ++j)
        if (xts[j] >= 0) s += gval[j] * (double)ep.omega[(long long)xts[j] * ep.l + c];
      s = block_sum<NT>(s, red);
      if (threadIdx.x == 0) atomicAdd(ep.y + (long long)xs * ep.l + c, (float)s);
    }
  }
}

// sum of fold slices: out[e] = sum_f in[f][e]
template <typename T>
__global__ void k_pool_folds(int F, long long PP, const T* __restrict__ in, T* __restrict__ out) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= PP) return;
  T s = 0;
  for (int f = 0; f < F; ++f) s += in[f * PP + e];
  out[e] = s;
}
__global__ void k_pool_counts(int F, long long PP, const int32_t* __restrict__ in,
                              int32_t* __restrict__ out) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= PP) return;
  int s = 0;
  for (int f = 0; f < F; ++f) s += in[f * PP + e];
  out[e] = s;
}

// cv[h] = err / w_in over folds; +inf when EMPTY points hold > 1% of the
// held-out weight or nothing was scored.
__global__ void k_cv_finish(int nh, int F, const double* __restrict__ acc, double* __restrict__ cv) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= nh) return;
  double err = 0.0, win = 0.0, wout = 0.0;
  for (int f = 0; f < F; ++f) {
    err += acc[(h * F + f) * 3 + 0];
    win += acc[(h * F + f) * 3 + 1];
    wout += acc[(h * F + f) * 3 + 2];
  }
  cv[h] = (wout > 0.01 * (win + wout) || !(win > 0.0)) ? __longlong_as_double(0x7ff0000000000000ll)
                                                       : err / win;
}

// One smoothing pass of the P x P bins (optionally train = pooled - sub_*).
template <typename T, bool COMP>
fpca_status cov_smooth_one(fpca_ctx* ctx, const fpca_grid* g, const int32_t* cnt, const T* w,
                           const T* v, const int32_t* sub_cnt, const T* sub_w, const T* sub_v,
                           const double* h, const double* tab, T* mids, T* varr,
                           const double* mu_raw, T* gamma, uint8_t* status, Epilogue<T> ep) {
  const int d = g->d;
  const int P = grid_P(g);
  const long long PP = (long long)P * P;
  const int Tax[2] = {host_taps(h[0], g->m[0]), d > 1 ? host_taps(h[1], g->m[1]) : 0};
  static bool vattr = false;
  if (!vattr) {
    cudaFuncSetAttribute(k_vpass<T, COMP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(sizeof(T) * (TROWS * TW + (size_t)64 * VCOLS)));
    vattr = true;
  }
  const dim3 vblk(VCOLS);
  auto tabk = [&](int k) { return tab + (size_t)k * TROWS * TW; };
  if (d == 2) {
    const int M1 = g->m[0], M2 = g->m[1];
    // pass along s2 (axis 1): rows L*M2 + a
    VJobs j1{};
    j1.j[0] = VJob{w, sub_w, 0, 3, {0, 1, 2}, {mids + 0 * PP, mids + 1 * PP, mids + 2 * PP}};
    j1.j[1] = VJob{v, sub_v, 0, 2, {0, 1, 0}, {mids + 3 * PP, mids + 4 * PP, nullptr}};
    j1.j[2] = VJob{cnt, sub_cnt, 1, 1, {3, 0, 0}, {mids + 5 * PP, nullptr, nullptr}};
    k_vpass<T, COMP><<<dim3((P + VCOLS - 1) / VCOLS, M1, 3), vblk,
                       sizeof(T) * (TROWS * TW + (size_t)M2 * VCOLS), ctx->stream>>>(
        j1, P, M2, 1, Tax[1], tabk(1));
    FPCA_LAUNCHED(ctx, "cov_vpass_s2");
    // pass along s1 (axis 0): rows L + a*M2
    VJobs j2{};
    j2.j[0] = VJob{mids + 0 * PP, nullptr, 0, 3, {0, 1, 2},
                   {varr + 0 * PP, varr + 1 * PP, varr + 2 * PP}};
    j2.j[1] = VJob{mids + 1 * PP, nullptr, 0, 2, {0, 1, 0}, {varr + 3 * PP, varr + 4 * PP, nullptr}};
    j2.j[2] = VJob{mids + 2 * PP, nullptr, 0, 1, {0, 0, 0}, {varr + 5 * PP, nullptr, nullptr}};
    j2.j[3] = VJob{mids + 3 * PP, nullptr, 0, 2, {0, 1, 0}, {varr + 6 * PP, varr + 7 * PP, nullptr}};
    j2.j[4] = VJob{mids + 4 * PP, nullptr, 0, 1, {0, 0, 0}, {varr + 8 * PP, nullptr, nullptr}};
    j2.j[5] = VJob{mids + 5 * PP, nullptr, 0, 1, {3, 0, 0}, {varr + 9 * PP, nullptr, nullptr}};
    k_vpass<T, COMP><<<dim3((P + VCOLS - 1) / VCOLS, M2, 6), vblk,
                       sizeof(T) * (TROWS * TW + (size_t)M1 * VCOLS), ctx->stream>>>(
        j2, P, M1, M2, Tax[0], tabk(0));
    FPCA_LAUNCHED(ctx, "cov_vpass_s1");
    // t-side + solve
    constexpr int NT = 512, PPT = 2;
    const int R = M1, C = M2;
    const int TH = std::min(R, (NT * PPT) / C);
    const int nrmax = std::min(R, TH + 2 * Tax[0]);
    const size_t hsmem =
        sizeof(T) * (2 * TROWS * TW + (size_t)narr(2) * nrmax * C + (size_t)3 * TH * C);
    if (hsmem > ctx->smem_optin)
      return fpca_fail(ctx, FPCA_E_UNSUPPORTED, "t-side tile needs %zu bytes of shared memory",
                       hsmem);
    cudaFuncSetAttribute(k_hpass_solve<2, T, COMP, NT, PPT>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsmem);
    k_hpass_solve<2, T, COMP, NT, PPT><<<dim3((R + TH - 1) / TH, P), NT, hsmem, ctx->stream>>>(
        varr, P, R, C, TH, Tax[0], Tax[1], tabk(0), tabk(1), mu_raw, gamma, status, ep);
    FPCA_LAUNCHED(ctx, "cov_hpass_solve");
    return FPCA_OK;
  }
  // d = 1: one vertical pass along s1, then the t pass + solve
  const int M1 = g->m[0];
  VJobs j1{};
  j1.j[0] = VJob{w, sub_w, 0, 3, {0, 1, 2}, {varr + 0 * PP, varr + 1 * PP, varr + 2 * PP}};
  j1.j[1] = VJob{v, sub_v, 0, 2, {0, 1, 0}, {varr + 3 * PP, varr + 4 * PP, nullptr}};
  j1.j[2] = VJob{cnt, sub_cnt, 1, 1, {3, 0, 0}, {varr + 5 * PP, nullptr, nullptr}};
  k_vpass<T, COMP><<<dim3((P + VCOLS - 1) / VCOLS, 1, 3), vblk,
                     sizeof(T) * (TROWS * TW + (size_t)M1 * VCOLS), ctx->stream>>>(
      j1, P, M1, 1, Tax[0], tabk(0));
  FPCA_LAUNCHED(ctx, "cov_vpass_s1");
  constexpr int NT = 128, PPT = 1;
  if (M1 > NT * PPT) return fpca_fail(ctx, FPCA_E_UNSUPPORTED, "d = 1 needs m <= 128");
  const size_t hsmem = sizeof(T) * (2 * TROWS * TW + (size_t)narr(1) * M1 + (size_t)3 * M1);
  cudaFuncSetAttribute(k_hpass_solve<1, T, COMP, NT, PPT>,
                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsmem);
  k_hpass_solve<1, T, COMP, NT, PPT><<<dim3(1, P), NT, hsmem, ctx->stream>>>(
      varr, P, 1, M1, 1, 0, Tax[0], tabk(0), tabk(0), mu_raw, gamma, status, ep);
  FPCA_LAUNCHED(ctx, "cov_hpass_solve");
  return FPCA_OK;
}

template <typename T, bool COMP>
fpca_status smooth_cov_typed(fpca_ctx* ctx, const fpca_grid* g, const fpca_covbins* bins,
                             const double* h, int nh, const double* mu_raw, const float* omega,
                             int l, T* gamma, uint8_t* status, float* y, double* cv) {
  const int d = g->d;
  const int P = grid_P(g);
  const long long PP = (long long)P * P;
  const int F = bins->nfold > 0 ? bins->nfold : 1;
  const int nmid = d == 2 ? 6 : 0;
  const size_t need = WsCarve::round(sizeof(double) * 3 * TROWS * TW) +
                      WsCarve::round(sizeof(T) * PP * (size_t)(nmid + narr(d))) +
                      (F > 1 ? WsCarve::round(sizeof(T) * PP) * 2 + WsCarve::round(4 * PP) : 0) +
                      WsCarve::round(sizeof(double) * 3 * (size_t)nh * F) + 4096;
  void* ws = fpca_workspace(ctx, need);
  if (!ws) return fpca_fail(ctx, FPCA_E_OOM, "workspace (%zu bytes)", need);
  WsCarve carve(ws);
  double* tab = carve.take<double>(3 * TROWS * TW);
  T* mids = carve.take<T>((size_t)PP * nmid);
  T* varr = carve.take<T>((size_t)PP * narr(d));
  double* cvacc = carve.take<double>((size_t)3 * nh * F);
  const T* w = static_cast<const T*>(bins->w);
  const T* v = static_cast<const T*>(bins->v);
  const int32_t* cnt = bins->cnt;
  if (F > 1) {
    T* wp = carve.take<T>(PP);
    T* vp = carve.take<T>(PP);
    int32_t* cp = carve.take<int32_t>(PP);
    const int nb = (int)((PP + 255) / 256);
    k_pool_folds<T><<<nb, 256, 0, ctx->stream>>>(F, PP, w, wp);
    FPCA_LAUNCHED(ctx, "pool_folds");
    k_pool_folds<T><<<nb, 256, 0, ctx->stream>>>(F, PP, v, vp);
    FPCA_LAUNCHED(ctx, "pool_folds");
    k_pool_counts<<<nb, 256, 0, ctx->stream>>>(F, PP, cnt, cp);
    FPCA_LAUNCHED(ctx, "pool_counts");
    w = wp;
    v = vp;
    cnt = cp;
  }
  if (y) cudaMemsetAsync(y, 0, sizeof(float) * (size_t)nh * P * l, ctx->stream);
  if (cv) cudaMemsetAsync(cvacc, 0, sizeof(double) * 3 * (size_t)nh * F, ctx->stream);
  for (int ih = 0; ih < nh; ++ih) {
    const double* hh = h + (size_t)ih * d;
    TapParams tp{};
    tp.d = d;
    for (int k = 0; k < 3; ++k) {
      tp.m[k] = k < d ? g->m[k] : 1;
      tp.h[k] = k < d ? hh[k] : 1.0;
    }
    k_taps<<<d, 128, 0, ctx->stream>>>(tp, tab);
    FPCA_LAUNCHED(ctx, "taps");
    // the fit on all bins: Gamma_hat, status, projection
    if (gamma || status || y) {
      Epilogue<T> ep{};
      if (y) {
        ep.omega = omega;
        ep.l = l;
        ep.y = y + (size_t)ih * P * l;
      }
      fpca_status s = cov_smooth_one<T, COMP>(
          ctx, g, cnt, w, v, nullptr, nullptr, nullptr, hh, tab, mids, varr, mu_raw,
          gamma ? gamma + (size_t)ih * PP : nullptr, status ? status + (size_t)ih * PP : nullptr,
          ep);
      if (s != FPCA_OK) return s;
    }
    // K-fold CV: fit on the other folds, score the held-out fold
    if (cv) {
      const T* fw = static_cast<const T*>(bins->w);
      const T* fv = static_cast<const T*>(bins->v);
      const T* fq = static_cast<const T*>(bins->q);
      for (int f = 0; f < F; ++f) {
        Epilogue<T> ep{};
        ep.wf = fw + (size_t)f * PP;
        ep.vf = fv + (size_t)f * PP;
        ep.qf = fq + (size_t)f * PP;
        ep.cvacc = cvacc + 3 * ((size_t)ih * F + f);
        fpca_status s = cov_smooth_one<T, COMP>(
            ctx, g, cnt, w, v, bins->cnt + (size_t)f * PP, fw + (size_t)f * PP,
            fv + (size_t)f * PP, hh, tab, mids, varr, mu_raw, nullptr, nullptr, ep);
        if (s != FPCA_OK) return s;
      }
    }
  }
  if (cv) {
    k_cv_finish<<<(nh + 63) / 64, 64, 0, ctx->stream>>>(nh, F, cvacc, cv);
    FPCA_LAUNCHED(ctx, "cv_finish");
  }
  return FPCA_OK;
}

}  // namespace

fpca_status launch_smooth_mean(fpca_ctx* ctx, const fpca_grid* g, const int32_t* cnt,
                               const double* w, const double* v, const double* h, double* mu,
                               uint8_t* status) {
  const int P = grid_P(g);
  for (int k = 0; k < g->d; ++k)
    if (g->m[k] > TMAX + 1)
      return fpca_fail(ctx, FPCA_E_UNSUPPORTED, "mean smoothing is built for m <= %d", TMAX + 1);
  TapParams tp{};
  tp.d = g->d;
  for (int k = 0; k < 3; ++k) {
    tp.m[k] = k < g->d ? g->m[k] : 1;
    tp.h[k] = k < g->d ? h[k] : 1.0;
  }
  double* tab = static_cast<double*>(fpca_workspace(ctx, sizeof(double) * 3 * TROWS * TW));
  if (!tab) return fpca_fail(ctx, FPCA_E_OOM, "workspace");
  k_taps<<<g->d, 128, 0, ctx->stream>>>(tp, tab);
  FPCA_LAUNCHED(ctx, "taps");
  const int T0 = host_taps(tp.h[0], tp.m[0]);
  const int T1 = g->d > 1 ? host_taps(tp.h[1], tp.m[1]) : 0;
  const int T2 = g->d > 2 ? host_taps(tp.h[2], tp.m[2]) : 0;
  const int nb = (P + 127) / 128;
  if (g->d == 1)
    k_smooth_mean<1><<<nb, 128, 0, ctx->stream>>>(P, tp, tab, cnt, w, v, mu, status, T0, T1, T2);
  else if (g->d == 2)
    k_smooth_mean<2><<<nb, 128, 0, ctx->stream>>>(P, tp, tab, cnt, w, v, mu, status, T0, T1, T2);
  else
    k_smooth_mean<3><<<nb, 128, 0, ctx->stream>>>(P, tp, tab, cnt, w, v, mu, status, T0, T1, T2);
  FPCA_LAUNCHED(ctx, "smooth_mean");
  return FPCA_OK;
}

fpca_status smooth_cov_run(fpca_ctx* ctx, const fpca_grid* g, const fpca_covbins* bins,
                           const double* h, int nh, int prec, const double* mu_raw,
                           const float* omega, int l, void* gamma, uint8_t* status, float* y,
                           double* cv) {
  if (l > MAXL) return fpca_fail(ctx, FPCA_E_UNSUPPORTED, "projection built for l <= %d", MAXL);
  for (int ih = 0; ih < nh; ++ih)
    for (int k = 0; k < g->d; ++k)
      if (host_taps(h[(size_t)ih * g->d + k], g->m[k]) > TMAX)
        return fpca_fail(ctx, FPCA_E_UNSUPPORTED, "bandwidth too wide");
  if (prec == FPCA_F64)
    return smooth_cov_typed<double, false>(ctx, g, bins, h, nh, mu_raw, omega, l,
                                           static_cast<double*>(gamma), status, y, cv);
  if (prec == FPCA_F32C)
    return smooth_cov_typed<float, true>(ctx, g, bins, h, nh, mu_raw, omega, l,
                                         static_cast<float*>(gamma), status, y, cv);
  return smooth_cov_typed<float, false>(ctx, g, bins, h, nh, mu_raw, omega, l,
                                        static_cast<float*>(gamma), status, y, cv);
}
