// The t-side moment sweeps of the FP32 covariance smoother (d = 2) and what they
// share with the other smoothing kernels: the tap tables, the per-point local
// solve with its status rules, the bookkeeping of the moment slots and the
// epilogues (CV terms, fused projection, escalation queue).  Included by
// smooth.cu and by the translation units that instantiate the packed sweep
// (tsweep_*.cu).
#pragma once

#include <cstdint>

#include "fpca_internal.cuh"
#include "ptx.cuh"

namespace fpca_sweep {

constexpr int TMAX = 63;          // largest tap offset supported (m <= 64)
constexpr int TW = 2 * TMAX + 1;  // table width
constexpr int TROWS = 4;          // K, K u, K u^2, box (1 inside the support)

// Thresholds of the per-point status rules.
constexpr double PIVOT_RTOL_F64 = 1e-9;  // FP64 moments: fallback at or below
constexpr double PIVOT_RTOL_F32 = 1e-5;  // FP32 moments: fallback at or below
constexpr double ESCALATE_F32 = 1e-2;    // FP32 solve redone in float-float below this


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
    T Ac[D][D], rc[D];
#pragma unroll
    for (int i = 0; i < D; ++i) {
      rc[i] = r[i];
#pragma unroll
      for (int j = 0; j < D; ++j) Ac[i][j] = A[i][j];
    }
    double ratio;
    const T b = elim_solve<D, T>(A, r, ratio);
    if (ratio >= ESCALATE_F32) {
      st = FPCA_PT_OK;
      return (double)b;
    }
    double Ad[D][D], rd[D];
#pragma unroll
    for (int i = 0; i < D; ++i) {
      rd[i] = (double)rc[i];
#pragma unroll
      for (int j = 0; j < D; ++j) Ad[i][j] = (double)Ac[i][j];
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

// FP32 fit without FP64 arithmetic on the common path: pivot tests by
// multiplication (pivot < thr * diagonal) and FP32 divisions; the FP64
// elimination runs only for the rare escalated systems.
// Status code returned when the system must be re-solved at higher precision.
constexpr uint8_t PT_ESCALATE = 255;

template <int D, bool INLINE_FP64 = true>
__device__ __forceinline__ float fit_point_f32(float (&A)[D][D], float (&r)[D], float nonempty,
                                               uint8_t& st) {
  if (!(A[0][0] > 0.f)) {
    st = FPCA_PT_EMPTY;
    return __int_as_float(0x7fc00000);
  }
  if (nonempty < (float)D) {
    st = FPCA_PT_FALLBACK;
    return r[0] / A[0][0];
  }
  float Ac[D][D], rc[D], diag[D];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    rc[i] = r[i];
    diag[i] = A[i][i];
#pragma unroll
    for (int j = 0; j < D; ++j) Ac[i][j] = A[i][j];
  }
  bool escalate = false;
  float invp[D];  // 1 / pivot, reused by the back substitution
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const float piv = A[k][k];
    if (!(piv >= (float)ESCALATE_F32 * diag[k])) escalate = true;
    // the fast reciprocal (about 1 ulp): a system kept in FP32 has every pivot at
    // least 1e-2 of its diagonal, so the solution moves by a few ulps at most; the
    // systems below that are solved again in float-float
    const float inv = piv > 0.f ? __fdividef(1.f, piv) : 0.f;
    invp[k] = inv;
#pragma unroll
    for (int i = k + 1; i < D; ++i) {
      const float l = A[k][i] * inv;
#pragma unroll
      for (int j = i; j < D; ++j) A[i][j] = fmaf(-l, A[k][j], A[i][j]);
      r[i] = fmaf(-l, r[k], r[i]);
    }
  }
  if (!escalate) {
    float x[D];
#pragma unroll
    for (int k = D - 1; k >= 0; --k) {
      float sacc = r[k];
#pragma unroll
      for (int j = k + 1; j < D; ++j) sacc = fmaf(-A[k][j], x[j], sacc);
      x[k] = sacc * invp[k];
    }
    st = FPCA_PT_OK;
    return x[0];
  }
  if constexpr (!INLINE_FP64) {
    st = PT_ESCALATE;
    return 0.f;
  }
  double Ad[D][D], rd[D];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    rd[i] = (double)rc[i];
#pragma unroll
    for (int j = 0; j < D; ++j) Ad[i][j] = (double)Ac[i][j];
  }
  double ratio;
  const double bd = elim_solve<D, double>(Ad, rd, ratio);
  if (ratio <= PIVOT_RTOL_F32) {
    st = FPCA_PT_FALLBACK;
    return rc[0] / Ac[0][0];
  }
  st = FPCA_PT_OK;
  return (float)bd;
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
  // Escalated fits (FP32 pivots below the escalation threshold) are queued
  // here and solved in float-float (about 48 bits) by a separate kernel:
  // entry e holds the 21 moment slots of the point in esc_slots[e*21 ..] and
  // its (xs, xt).
  float* esc_slots;
  int2* esc_idx;
  int* esc_idx_item;   // batched CV grid: the item of each queued point, or NULL
  int esc_item_id;
  unsigned* esc_count;
  int esc_cap;
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


constexpr int HT = 8;     // t-plane rows per block
constexpr int SEG = 8;    // columns per phase-2 item
constexpr int NT2 = 256;  // threads per block
constexpr int NMID = 15;  // mid arrays (d = 2)
constexpr int NSL = 21;   // moment slots (d = 2)

// mid array m -> (s-side array a, t1 power a1; 3 = box weights);
// slot s -> (mid array, t2 power; 3 = box weights).  Items of one warp share
// m (phase 1) or s (phase 2), so the constant-cache reads broadcast.
static __constant__ int8_t c_mid_array[NMID] = {0, 0, 0, 1, 1, 2, 3, 3, 4, 5, 6, 6, 7, 8, 9};
static __constant__ int8_t c_mid_pow[NMID] = {0, 1, 2, 0, 1, 0, 0, 1, 0, 0, 0, 1, 0, 0, 3};
static __constant__ int8_t c_slot_mid[NSL] = {0, 3, 6, 1, 0, 5, 8, 4, 3, 9, 7,
                                       6, 2, 1, 0, 10, 12, 13, 11, 10, 14};
static __constant__ int8_t c_slot_pow[NSL] = {0, 0, 0, 0, 1, 0, 0, 0, 1, 0, 0,
                                       1, 0, 1, 2, 0, 0, 0, 0, 1, 3};


// CV terms a persistent CTA gathers over its tiles (held-out error, scored weight,
// weight of EMPTY points) in shared memory: each warp adds its tile's sums with one
// atomic per term, and the CTA adds the totals to ep.cvacc once (cv_flush).  No
// register is held across tiles and no block barrier is spent per tile.
struct CvShared {
  double v[3];
};

__device__ __forceinline__ void cv_warp_add(CvShared* cvs, float e, float i, float o) {
#pragma unroll
  for (int k = 16; k > 0; k >>= 1) {
    e += __shfl_xor_sync(0xffffffffu, e, k);
    i += __shfl_xor_sync(0xffffffffu, i, k);
    o += __shfl_xor_sync(0xffffffffu, o, k);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&cvs->v[0], (double)e);
    atomicAdd(&cvs->v[1], (double)i);
    atomicAdd(&cvs->v[2], (double)o);
  }
}

// The CTA's CV totals into acc (every thread calls it; the caller's barrier
// precedes it) and the shared sums cleared for the next item.
__device__ __forceinline__ void cv_flush(CvShared* cvs, double* acc) {
  __syncthreads();
  if (threadIdx.x == 0) {
    if (acc) {
      atomicAdd(acc + 0, cvs->v[0]);
      atomicAdd(acc + 1, cvs->v[1]);
      atomicAdd(acc + 2, cvs->v[2]);
    }
    cvs->v[0] = cvs->v[1] = cvs->v[2] = 0.0;
  }
  __syncthreads();
}

// Phase 3 of the t-side sweep (shared by the sweep kernels): per-point 5 x 5 solve
// from the 21 moment slots in shared memory ([NSL][HT][SC]), write of Gamma_hat and
// status, CV terms and the fused y = Gamma_hat Omega epilogue.  `mid` is shared
// scratch of at least HT * C + NTH floats (the y epilogue reuses it).  With `cvs`
// the CV terms go to the CTA's shared sums (the kernel flushes them); without, the
// block adds this tile's terms to ep.cvacc.
template <int C, int NTH>
__device__ __forceinline__ void tside_phase3(const float* __restrict__ slots, int SC, int half,
                                             int P, int xs, int a0, int th,
                                             const double* __restrict__ mu_raw,
                                             float* __restrict__ gamma,
                                             uint8_t* __restrict__ status, const Epilogue<float>& ep,
                                             double* red, float* mid, CvShared* cvs = nullptr) {
  // phase 3: per-point solve, write, epilogue terms (FP32; escalated systems
  // are queued for the float-float kernel; FP64 for the block sums of the CV terms)
  float cv_err = 0.f, cv_in = 0.f, cv_out = 0.f;
  constexpr int PPT3 = (HT * C + NTH - 1) / NTH;
  float gval[PPT3];
  int xts[PPT3];
#pragma unroll
  for (int j = 0; j < PPT3; ++j) {
    const int e = threadIdx.x + j * NTH;
    gval[j] = 0.f;
    xts[j] = -1;
    if (e >= th * C) continue;
    const int i = e / C, c = e % C;
    if (half && (a0 + i) * C + c < xs) continue;  // taken from the mirror (t, s)
    const float* sl = slots + (size_t)i * SC + c;
    float A[5][5], rv[5];
#pragma unroll
    for (int i2 = 0; i2 < 5; ++i2) {
      rv[i2] = sl[(size_t)rslot(2, i2) * HT * SC];
#pragma unroll
      for (int j2 = i2; j2 < 5; ++j2) {
        A[i2][j2] = sl[(size_t)aslot(2, i2, j2) * HT * SC];
        A[j2][i2] = A[i2][j2];
      }
    }
    const float cnt = sl[(size_t)(NSL - 1) * HT * SC];
    uint8_t st;
    float gv = fit_point_f32<5, false>(A, rv, cnt + 0.25f, st);
    const int xt = (a0 + i) * C + c;
    if (st == PT_ESCALATE) {
      const unsigned slot = ep.esc_count ? atomicAdd(ep.esc_count, 1u) : 0xffffffffu;
      if (slot < (unsigned)ep.esc_cap) {
        float* dst = ep.esc_slots + (size_t)slot * NSL;
        for (int q = 0; q < NSL; ++q) dst[q] = sl[(size_t)q * HT * SC];
        ep.esc_idx[slot] = make_int2(xs, xt);
        if (ep.esc_idx_item) ep.esc_idx_item[slot] = ep.esc_item_id;
        continue;  // the escalation kernel writes this point and its epilogue terms
      }
      // queue full: solve here
      float A2[5][5], r2[5];
#pragma unroll
      for (int i2 = 0; i2 < 5; ++i2) {
        r2[i2] = sl[(size_t)rslot(2, i2) * HT * SC];
#pragma unroll
        for (int j2 = i2; j2 < 5; ++j2) {
          A2[i2][j2] = sl[(size_t)aslot(2, i2, j2) * HT * SC];
          A2[j2][i2] = A2[i2][j2];
        }
      }
      gv = fit_point_f32<5, true>(A2, r2, cnt + 0.25f, st);
    }
    if (mu_raw && st != FPCA_PT_EMPTY) gv -= (float)(mu_raw[xs] * mu_raw[xt]);
    const long long o = (long long)xs * P + xt;
    if (gamma) gamma[o] = gv;
    if (status) status[o] = st;
    xts[j] = xt;
    gval[j] = st == FPCA_PT_EMPTY ? 0.f : gv;
    if (ep.cvacc) {
      // in half mode (s, t) also stands for (t, s): the CV bins are symmetric
      const float mul = (half && xt != xs) ? 2.f : 1.f;
      const float wf = ep.wf[o];
      if (st == FPCA_PT_EMPTY) {
        cv_out += mul * wf;
      } else {
        cv_err += mul * (ep.qf[o] - 2.f * gv * ep.vf[o] + gv * gv * wf);
        cv_in += mul * wf;
      }
    }
  }
  if (ep.cvacc && cvs) {
    cv_warp_add(cvs, cv_err, cv_in, cv_out);
  } else if (ep.cvacc) {
    const double s0 = block_sum<NTH>((double)cv_err, red);
    const double s1 = block_sum<NTH>((double)cv_in, red);
    const double s2 = block_sum<NTH>((double)cv_out, red);
    if (threadIdx.x == 0) {
      atomicAdd(ep.cvacc + 0, s0);
      atomicAdd(ep.cvacc + 1, s1);
      atomicAdd(ep.cvacc + 2, s2);
    }
  }
  if (ep.y) {
    // y[s, :] += sum over this block's t of Gamma_hat(s, t) Omega[t, :].  The block's
    // t form one contiguous run of Omega's rows, so thread (group, column c) walks
    // every ng-th of them with coalesced loads; the ng partials of a column are
    // then added in shared memory (which reuses the mid rows: phase 3 reads only
    // the slots).  EMPTY and escalated points carry 0.
    (void)xts;
    float* gsm = mid;             // [HT * C]
    float* part = mid + HT * C;   // [NTH]
#pragma unroll
    for (int j = 0; j < PPT3; ++j) {
      const int e = threadIdx.x + j * NTH;
      if (e < HT * C) gsm[e] = gval[j];
    }
    __syncthreads();
    const int l = ep.l, ng = NTH / l;
    const int c = threadIdx.x % l, grp = threadIdx.x / l;
    float acc = 0.f;
    if (grp < ng) {
      const float* om = ep.omega + (long long)a0 * C * l + c;
      for (int t = grp; t < th * C; t += ng) acc = fmaf(gsm[t], om[(long long)t * l], acc);
    }
    part[threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.x < l) {
      float tot = 0.f;
      for (int gi = 0; gi < ng; ++gi) tot += part[gi * l + threadIdx.x];
      atomicAdd(ep.y + (long long)xs * l + threadIdx.x, tot);
    }
  }
}


// ---------------------------------------------------------------------------
// t-side sweep + solve with packed FP32 pairs (d = 2, FP32), persistent
// ---------------------------------------------------------------------------
// The same three phases as k_hsolve2 on tiles of one s-row x HT t1-rows, with
// every sliding sum carried out on a pair of independent sums by the paired FP32
// instructions of sm_100-class GPUs (one fma.rn.f32x2 performs two FMAs), so one
// issue slot feeds two FMA lanes.  The 15 mid arrays are grouped in 8 pairs
// (m, m'), stored interleaved per column ({mid m, mid m'}):
//   phase 1  item = (pair u, t2 column c): the t1 window of column c of the s-side
//            array(s) of m and m', weights {w_p, w_p'} -> HT rows of {m, m'};
//   phase 2  item = (unit (u, q), row i, SEG-column segment): the float2 window
//            along row i of pair u, weights {w_q, w_q} -> slots (m, q), (m', q);
//   phase 3  the per-point solve of k_hsolve2 (tside_phase3).
// Persistent CTAs (two per SM up to 9 taps) walk the tiles; each tile's input rows
// come in by TMA bulk copies, and the two CTAs of an SM start half a tile apart so
// that one's copy overlaps the other's arithmetic (the slots of phases 2-3 alias the
// input rows, so a CTA cannot fetch ahead of itself).  Tap counts are odd
// (2T + 1) and enter as template parameters up to TS_MAXT; every sum is formed
// in partials of at most TS_PART taps (plain FMAs) added with Kahan compensation
// when COMP is set.
constexpr int TS_PART = 12;
constexpr int TS_MAXT = 19;   // half-widths of the unrolled sweeps (taps <= 39)
constexpr int TS_PAIRS = 8;   // mid pairs
constexpr int TS_UNITS = 12;  // (mid pair, t2 power) units of phase 2
constexpr int TS_NT = 256;    // threads per CTA (two CTAs per SM)

// pair u -> (mid m, mid m'); m' = -1: none (its half is zero).  The pairs are
// chosen for phase 2: a unit is one stored pair at one t2 power, so a pair costs
// as many units as its mid with more t2 powers needs (m0: 3; m1, m3, m6, m10: 2;
// the rest 1).  Pairing the 2-power mids with each other and m0 with m1 gives
// 12 units -- 768 phase-2 items, three full rounds of the CTA's 256 threads --
// where pairing each mid with its array's neighbour gave 13 (a fourth round a
// quarter full).  Pairs of one s-side array (m0, m1; m10, m11) share their
// phase-1 window; the others load two.
static __constant__ int8_t c_ts_mid[TS_PAIRS][2] = {{0, 1}, {10, 11}, {3, 6}, {2, 4},
                                             {5, 7},  {8, 9},   {12, 13}, {14, -1}};
// phase-2 unit -> (pair, t2 power row, slot of .x, slot of .y; -1 = not needed)
static __constant__ int8_t c_ts_unit[TS_UNITS][4] = {
    {0, 0, 0, 3},   {0, 1, 4, 13}, {0, 2, 14, -1}, {1, 0, 15, 18}, {1, 1, 19, -1}, {2, 0, 1, 2},
    {2, 1, 8, 11},  {3, 0, 12, 7}, {4, 0, 5, 10},  {5, 0, 6, 9},   {6, 0, 16, 17}, {7, 3, 20, -1}};

struct TsGeom {
  int P, R, C;
  int Tr, Tc;      // tap half-widths (t1, t2)
  int nrp;         // input rows held per tile: HT + 2 Tr
  int off;         // first output column of a mid row: Tc rounded up to even
  int RS2;         // mid-pair row stride in float2 (odd, >= off + C + Tc)
  int SC;          // slot row stride (floats)
  int half;
  int ntiles;      // t1 blocks x P s-rows
};

__device__ __forceinline__ float2 f2neg(float2 a) { return make_float2(-a.x, -a.y); }

template <bool COMP>
__device__ __forceinline__ void kahan2(float2& s, float2& c, float2 p) {
  if constexpr (COMP) {
    const float2 y = __fadd2_rn(p, f2neg(c));
    const float2 t = __fadd2_rn(s, y);
    c = __fadd2_rn(__fadd2_rn(t, f2neg(s)), f2neg(y));
    s = t;
  } else {
    s = __fadd2_rn(s, p);
  }
}

// NO sums along a line of float2 from one window of NO + NTAP - 1 elements:
//   out[j] = sum_{k < NTAP} w[k] * x[(j + k) * stride]   (pairwise),
// w[k] given as float2 pairs, two taps per float4.
template <int NO, int NTAP, bool COMP>
__device__ __forceinline__ void slide2(const float2 (&win)[NO + NTAP - 1],
                                       const float4* __restrict__ w4, float2 (&out)[NO]) {
  float2 cmp[NO];
#pragma unroll
  for (int k0 = 0; k0 < NTAP; k0 += TS_PART) {
    float2 part[NO];
#pragma unroll
    for (int k = k0; k < (k0 + TS_PART < NTAP ? k0 + TS_PART : NTAP); ++k) {
      const float4 wq = w4[k >> 1];
      const float2 wk = (k & 1) ? make_float2(wq.z, wq.w) : make_float2(wq.x, wq.y);
#pragma unroll
      for (int j = 0; j < NO; ++j)
        part[j] = (k == k0) ? __fmul2_rn(wk, win[j + k]) : __ffma2_rn(wk, win[j + k], part[j]);
    }
#pragma unroll
    for (int j = 0; j < NO; ++j) {
      if (k0 == 0) {
        out[j] = part[j];
        cmp[j] = make_float2(0.f, 0.f);
      } else {
        kahan2<COMP>(out[j], cmp[j], part[j]);
      }
    }
  }
}

// weights of half-width T in pairs: row stride ntp = 2T + 1 rounded up to even
__host__ __device__ constexpr int ts_ntp(int T) { return (2 * T + 2) & ~1; }

// Weights {w, w} per table row (K, K u, K u^2, box) at offset k - T, for the t1
// (w1, from tabr) and the t2 (w2, from tabc) sweeps.
__device__ __forceinline__ void ts_load_weights(const double* __restrict__ tabr, int Tr,
                                                const double* __restrict__ tabc, int Tc,
                                                float2* __restrict__ w1, float2* __restrict__ w2) {
  const int n1 = ts_ntp(Tr), n2 = ts_ntp(Tc);
  for (int e = threadIdx.x; e < TROWS * n1; e += blockDim.x) {
    const int row = e / n1, k = e - (e / n1) * n1;
    const float w = k <= 2 * Tr ? (float)tabr[row * TW + TMAX + (k - Tr)] : 0.f;
    w1[e] = make_float2(w, w);
  }
  for (int e = threadIdx.x; e < TROWS * n2; e += blockDim.x) {
    const int row = e / n2, k = e - (e / n2) * n2;
    const float w = k <= 2 * Tc ? (float)tabc[row * TW + TMAX + (k - Tc)] : 0.f;
    w2[e] = make_float2(w, w);
  }
}

template <int C, int TR, bool COMP>
__device__ __forceinline__ void ts_phase1(const TsGeom& g, const float* __restrict__ in,
                                          const float2* __restrict__ w1, float2* __restrict__ mid2) {
  // item = (pair u, t2-column pair cp): float2 windows {column 2cp, column 2cp+1} of
  // the s-side arrays of m and m' (one window when they share their array) give the
  // HT rows of m and m' at both columns, stored interleaved ({m, m'} per column).
  constexpr int NTAP = 2 * TR + 1;
  constexpr int NW = HT + NTAP - 1;
  constexpr int NTP = (2 * TR + 2) & ~1;
  constexpr int CP = C / 2;
  for (int it = threadIdx.x; it < TS_PAIRS * CP; it += TS_NT) {
    const int u = it / CP, cp = it - (it / CP) * CP;
    const int m0 = c_ts_mid[u][0], m1 = c_ts_mid[u][1];
    const int a0 = c_mid_array[m0];
    float2 o0[HT], o1[HT];
    {
      const float2* x = reinterpret_cast<const float2*>(in + (size_t)a0 * g.nrp * C) + cp;
      float2 win[NW];
#pragma unroll
      for (int r = 0; r < NW; ++r) win[r] = x[r * CP];
      slide2<HT, NTAP, COMP>(win, reinterpret_cast<const float4*>(w1 + c_mid_pow[m0] * NTP), o0);
      if (m1 >= 0 && c_mid_array[m1] == a0)
        slide2<HT, NTAP, COMP>(win, reinterpret_cast<const float4*>(w1 + c_mid_pow[m1] * NTP), o1);
    }
    if (m1 >= 0 && c_mid_array[m1] != a0) {
      const float2* x = reinterpret_cast<const float2*>(in + (size_t)c_mid_array[m1] * g.nrp * C) + cp;
      float2 win[NW];
#pragma unroll
      for (int r = 0; r < NW; ++r) win[r] = x[r * CP];
      slide2<HT, NTAP, COMP>(win, reinterpret_cast<const float4*>(w1 + c_mid_pow[m1] * NTP), o1);
    } else if (m1 < 0) {
#pragma unroll
      for (int j = 0; j < HT; ++j) o1[j] = make_float2(0.f, 0.f);
    }
    float2* dst = mid2 + (size_t)u * HT * g.RS2 + g.off + 2 * cp;
#pragma unroll
    for (int j = 0; j < HT; ++j) {
      dst[j * g.RS2] = make_float2(o0[j].x, o1[j].x);
      dst[j * g.RS2 + 1] = make_float2(o0[j].y, o1[j].y);
    }
  }
}

template <int C, int TC, bool COMP>
__device__ __forceinline__ void ts_phase2(const TsGeom& g, const float2* __restrict__ mid2,
                                          const float2* __restrict__ w2, float* __restrict__ slots) {
  constexpr int NTAP = 2 * TC + 1;
  constexpr int NW = SEG + NTAP - 1;
  constexpr int NTP = (2 * TC + 2) & ~1;
  constexpr int NSEG = C / SEG;
  constexpr int PER = HT * NSEG;  // items per unit
  for (int it = threadIdx.x; it < TS_UNITS * PER; it += TS_NT) {
    const int un = it / PER, e = it - (it / PER) * PER;
    const int i = e % HT, sg = e / HT;  // 8 rows x 2 segments per half-warp
    const int u = c_ts_unit[un][0], pw = c_ts_unit[un][1];
    const int sx = c_ts_unit[un][2], sy = c_ts_unit[un][3];
    const float2* x = mid2 + ((size_t)u * HT + i) * g.RS2 + (g.off - TC) + sg * SEG;
    float2 win[NW];
#pragma unroll
    for (int r = 0; r < NW; ++r) win[r] = x[r];
    float2 o[SEG];
    slide2<SEG, NTAP, COMP>(win, reinterpret_cast<const float4*>(w2 + pw * NTP), o);
    float* dx = slots + ((size_t)sx * HT + i) * g.SC + sg * SEG;
#pragma unroll
    for (int j = 0; j < SEG; ++j) dx[j] = o[j].x;
    if (sy >= 0) {
      float* dy = slots + ((size_t)sy * HT + i) * g.SC + sg * SEG;
#pragma unroll
      for (int j = 0; j < SEG; ++j) dy[j] = o[j].y;
    }
  }
}

// Tile t -> (s-row xs, first t1-row a0); whether it has work in half mode.  Tiles
// run s-row-major (the tiles of one s-row share input rows, which then stay in
// L2); the grid size is odd, so that each CTA, taking every gridDim.x-th tile,
// meets every t1-block (the half mode skips most tiles of the low t1-blocks).
__device__ __forceinline__ bool ts_tile(const TsGeom& g, int t, int& xs, int& a0) {
  const int nb = (g.R + HT - 1) / HT;
  xs = t / nb;
  a0 = (t - xs * nb) * HT;
  const int th = min(HT, g.R - a0);
  return !(g.half && (a0 + th) * g.C <= xs);
}

__device__ __forceinline__ int ts_next(const TsGeom& g, int t) {
  int xs, a0;
  for (; t < g.ntiles; t += gridDim.x)
    if (ts_tile(g, t, xs, a0)) return t;
  return g.ntiles;
}

// Issue the bulk copies of tile t's in-grid input rows (thread 0) and zero its
// padding rows (all threads; disjoint from the copied rows).
template <int C>
__device__ __forceinline__ void ts_fetch(const TsGeom& g, const float* __restrict__ varr, int t,
                                         float* __restrict__ in, uint32_t bar) {
  int xs, a0;
  ts_tile(g, t, xs, a0);
  const long long PP = (long long)g.P * g.P;
  const int rlo = max(0, a0 - g.Tr), rhi = min(g.R, a0 - g.Tr + g.nrp);
  const int skip = rlo - (a0 - g.Tr);
  const int nrow = max(0, rhi - rlo);
  const uint32_t bytes = (uint32_t)(nrow * C * sizeof(float));
  if (threadIdx.x == 0) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    ptx::mbar_arrive_expect_tx(bar, 10 * bytes);
    if (bytes > 0)
      for (int a = 0; a < 10; ++a)
        ptx::bulk_load(ptx::smem_u32(in + ((size_t)a * g.nrp + skip) * C),
                       varr + a * PP + (long long)xs * g.P + (long long)rlo * C, bytes, bar);
  }
  constexpr int C4 = C / 4;
  const int padrows = g.nrp - nrow;
  for (int e = threadIdx.x; e < 10 * padrows * C4; e += TS_NT) {
    const int a = e / (padrows * C4);
    const int rem = e - a * padrows * C4;
    const int pr = rem / C4, c4 = rem % C4;
    const int r = pr < skip ? pr : nrow + pr;
    *reinterpret_cast<float4*>(in + ((size_t)a * g.nrp + r) * C + 4 * c4) =
        make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

// Two CTAs fit an SM up to 9 taps each side (shared memory); wider windows run one
// CTA per SM and may use every register.
template <bool COMP, int C, int TR, int TC>
__global__ void __launch_bounds__(TS_NT, (TR <= 9 && TC <= 9) ? 2 : 1)
    k_tsweep(const float* __restrict__ varr, TsGeom g, const double* __restrict__ tabr,
             const double* __restrict__ tabc, const double* __restrict__ mu_raw,
             float* __restrict__ gamma, uint8_t* __restrict__ status, Epilogue<float> ep,
             int* __restrict__ err) {
  static_assert(C % SEG == 0 && C <= 64, "t-plane width");
  extern __shared__ __align__(128) unsigned char tsm[];
  __shared__ double red[TS_NT / 32];
  __shared__ __align__(8) uint64_t tile_bar;
  constexpr int NTPR = (2 * TR + 2) & ~1, NTPC = (2 * TC + 2) & ~1;
  float2* w1 = reinterpret_cast<float2*>(tsm);               // [TROWS][NTPR]
  float2* w2 = w1 + TROWS * NTPR;                             // [TROWS][NTPC]
  float2* mid2 = w2 + TROWS * NTPC;                           // [TS_PAIRS][HT][RS2]
  float* in = reinterpret_cast<float*>(mid2 + (size_t)TS_PAIRS * HT * g.RS2);  // [10][nrp][C]
  float* slots = in;                                          // [NSL][HT][SC] (after phase 1)
  const uint32_t bar = ptx::smem_u32(&tile_bar);
  if (threadIdx.x == 0) {
    ptx::mbar_init(bar, 1);
    ptx::fence_mbar_init();
  }
  ts_load_weights(tabr, TR, tabc, TC, w1, w2);
  // zero the column halo of the mid rows once: [0, off) and [off + C, RS2)
  {
    const int padw = g.RS2 - C;
    for (int e = threadIdx.x; e < TS_PAIRS * HT * padw; e += TS_NT) {
      const int line = e / padw, k = e - (e / padw) * padw;
      const int cp = k < g.off ? k : C + k;
      mid2[(size_t)line * g.RS2 + cp] = make_float2(0.f, 0.f);
    }
  }
  __syncthreads();
  // The two CTAs of an SM run the same phases on tiles of equal cost; the second
  // half of the grid starts half a tile later, so that one CTA's input copy
  // overlaps the other's arithmetic instead of coinciding with it.
  if (blockIdx.x >= gridDim.x / 2) __nanosleep(3000);
  uint32_t parity = 0;
  __shared__ CvShared cvs;  // this CTA's CV terms over its tiles
  if (threadIdx.x == 0) cvs.v[0] = cvs.v[1] = cvs.v[2] = 0.0;
  __syncthreads();
  for (int t = ts_next(g, blockIdx.x); t < g.ntiles; parity ^= 1u) {
    int xs, a0;
    ts_tile(g, t, xs, a0);
    const int th = min(HT, g.R - a0);
    ts_fetch<C>(g, varr, t, in, bar);
    const bool landed = ptx::mbar_wait(bar, parity, err);
    if (__syncthreads_or(!landed)) return;
    ts_phase1<C, TR, COMP>(g, in, w1, mid2);
    __syncthreads();
    const int tn = ts_next(g, t + gridDim.x);
    ts_phase2<C, TC, COMP>(g, mid2, w2, slots);
    __syncthreads();
    tside_phase3<C, TS_NT>(slots, g.SC, g.half, g.P, xs, a0, th, mu_raw, gamma, status, ep, red,
                           reinterpret_cast<float*>(mid2), &cvs);
    // the y epilogue used the mid rows as scratch: restore their zero halo
    if (ep.y) {
      __syncthreads();
      const int padw = g.RS2 - C;
      for (int e = threadIdx.x; e < TS_PAIRS * HT * padw; e += TS_NT) {
        const int line = e / padw, k = e - (e / padw) * padw;
        const int cp = k < g.off ? k : C + k;
        mid2[(size_t)line * g.RS2 + cp] = make_float2(0.f, 0.f);
      }
    }
    __syncthreads();  // phase 3 read the slots, which alias the next tile's input rows
    t = tn;
  }
  if (ep.cvacc) cv_flush(&cvs, ep.cvacc);
}

inline TsGeom ts_geometry(int P, int M1, int M2, int Tr, int Tc) {
  TsGeom g{};
  g.P = P;
  g.R = M1;
  g.C = M2;
  g.Tr = Tr;
  g.Tc = Tc;
  g.nrp = HT + 2 * Tr;
  g.off = (Tc + 1) & ~1;
  g.RS2 = (g.off + M2 + Tc) | 1;
  g.SC = M2 + 3;
  g.ntiles = ((M1 + HT - 1) / HT) * P;
  return g;
}

inline size_t ts_smem(const TsGeom& g) {
  const size_t in_f = (size_t)10 * g.nrp * g.C;
  const size_t slot_f = (size_t)NSL * HT * g.SC;
  return sizeof(float2) * ((size_t)TROWS * ts_ntp(g.Tr) + (size_t)TROWS * ts_ntp(g.Tc) +
                           (size_t)TS_PAIRS * HT * g.RS2) +
         sizeof(float) * (in_f > slot_f ? in_f : slot_f);
}

// Launches k_tsweep for the half-width T: two CTAs per SM walk the tiles.
template <bool COMP, int C, int T>
void tsweep_launch_t(fpca_ctx* ctx, size_t smem, const float* varr, const TsGeom& g,
                     const double* tabr, const double* tabc, const double* mu_raw, float* gamma,
                     uint8_t* status, const Epilogue<float>& ep) {
  static int attr = 0;  // dynamic shared memory the kernel is configured for
  if ((int)smem > attr) {
    cudaFuncSetAttribute(k_tsweep<COMP, C, T, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    attr = (int)smem;
  }
  const int nb = g.ntiles < 2 * ctx->num_sms - 1 ? g.ntiles : 2 * ctx->num_sms - 1;
  k_tsweep<COMP, C, T, T><<<nb > 0 ? nb : 1, TS_NT, smem, ctx->stream>>>(
      varr, g, tabr, tabc, mu_raw, gamma, status, ep, ctx->d_err);
}

#define FPCA_TSWEEP_PARAMS                                                                     \
  fpca_ctx *ctx, bool comp, int T, size_t smem, const float *varr, const TsGeom &g,          \
      const double *tabr, const double *tabc, const double *mu_raw, float *gamma,            \
      uint8_t *status, const Epilogue<float> &ep
#define FPCA_TSWEEP_ARGS ctx, comp, T, smem, varr, g, tabr, tabc, mu_raw, gamma, status, ep

// The kernels for half-widths TLO..THI (true if T is among them and was launched).
template <int C, int TLO, int THI>
bool tsweep_launch_range(FPCA_TSWEEP_PARAMS) {
  if constexpr (TLO > THI) {
    return false;
  } else {
    if (T == TLO) {
      if (comp)
        tsweep_launch_t<true, C, TLO>(ctx, smem, varr, g, tabr, tabc, mu_raw, gamma, status, ep);
      else
        tsweep_launch_t<false, C, TLO>(ctx, smem, varr, g, tabr, tabc, mu_raw, gamma, status, ep);
      return true;
    }
    return tsweep_launch_range<C, TLO + 1, THI>(FPCA_TSWEEP_ARGS);
  }
}

// Each range is instantiated in a translation unit of its own (tsweep_*.cu), so
// that the unrolled kernels compile in parallel.
bool tsweep_c64_a(FPCA_TSWEEP_PARAMS);  // T 1..6
bool tsweep_c64_b(FPCA_TSWEEP_PARAMS);  // T 7..10
bool tsweep_c64_c(FPCA_TSWEEP_PARAMS);  // T 11..13
bool tsweep_c64_d(FPCA_TSWEEP_PARAMS);  // T 14..16
bool tsweep_c64_e(FPCA_TSWEEP_PARAMS);  // T 17..19
bool tsweep_c32_a(FPCA_TSWEEP_PARAMS);  // T 1..6
bool tsweep_c32_b(FPCA_TSWEEP_PARAMS);  // T 7..12

// Is the packed-pair t-side sweep built for this t-plane width and these windows?
inline bool tsweep_built(int C, int Tr, int Tc) {
  if (Tr != Tc || Tr < 1) return false;
  return (C == 64 && Tr <= 19) || (C == 32 && Tr <= 12);
}

// Launches the packed sweep for t-planes C wide and half-width T on both t axes.
inline bool tsweep_launch(int C, FPCA_TSWEEP_PARAMS) {
  if (C == 64)
    return tsweep_c64_a(FPCA_TSWEEP_ARGS) || tsweep_c64_b(FPCA_TSWEEP_ARGS) ||
           tsweep_c64_c(FPCA_TSWEEP_ARGS) || tsweep_c64_d(FPCA_TSWEEP_ARGS) ||
           tsweep_c64_e(FPCA_TSWEEP_ARGS);
  if (C == 32) return tsweep_c32_a(FPCA_TSWEEP_ARGS) || tsweep_c32_b(FPCA_TSWEEP_ARGS);
  return false;
}

}  // namespace fpca_sweep
