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
#include <array>
#include <vector>
#include <cmath>

#include "fpca_internal.cuh"
#include "ptx.cuh"
#include "ff.cuh"
#include "tside.cuh"

namespace {

using namespace fpca_sweep;

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
// mean smoother by separable sums (Eq. 2.3, FP64): the moments
//   S_e = sum_b K(c_b - x) u^e W_b (|e| <= 2),  T_e = sum_b K u^e V_b (|e| <= 1)
// and the window count of non-empty bins are products of 1-D kernels, so they
// are built one axis at a time (the last axis first), each pass applying
// K u^power (or the box of the window, for the count) along one axis to the
// arrays of the previous pass; then one (d+1)-dimensional solve per node.
// ---------------------------------------------------------------------------
constexpr int MJ_MAX = 16;  // jobs per pass (d = 3: 6, 10, 15)

struct MeanPass {
  int axis, stride, T, njobs;
  int src[MJ_MAX], row[MJ_MAX];  // row: 0 K, 1 K u, 2 K u^2, 3 box
};

__global__ void k_mean_prep(int P, const int32_t* __restrict__ cnt, const double* __restrict__ w,
                            const double* __restrict__ v, double* __restrict__ out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  out[p] = w[p];
  out[P + p] = v[p];
  out[2 * P + p] = cnt[p] > 0 ? 1.0 : 0.0;
}

// One thread per (node, job): the jobs of a pass run side by side and each tap
// sum is split into two interleaved FP64 chains (even and odd offsets), since
// dependent FP64 operations have a long latency on this GPU.
__global__ void k_mean_pass(int P, int M, MeanPass mp, const double* __restrict__ tab,
                            const double* __restrict__ in, double* __restrict__ out) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)P * mp.njobs) return;
  const int j = (int)(e / P), p = (int)(e - (long long)j * P);
  const int c = (p / mp.stride) % M;
  const int lo = max(-mp.T, -c), hi = min(mp.T, M - 1 - c);
  const double* w = tab + (size_t)mp.axis * TROWS * TW + TMAX + mp.row[j] * TW;
  const double* src = in + (size_t)mp.src[j] * P;
  double s0 = 0.0, s1 = 0.0;
  int r = lo;
  for (; r + 1 <= hi; r += 2) {
    s0 = fma(w[r], src[p + r * mp.stride], s0);
    s1 = fma(w[r + 1], src[p + (r + 1) * mp.stride], s1);
  }
  if (r <= hi) s0 = fma(w[r], src[p + r * mp.stride], s0);
  out[(size_t)j * P + p] = s0 + s1;
}

struct MeanIdx {
  int a[16], r[4], n;  // array of each normal-matrix entry, right-hand side entry, count
};

template <int DIM>
__global__ void k_mean_solve(int P, const double* __restrict__ mom, MeanIdx ix,
                             double* __restrict__ mu, uint8_t* __restrict__ status) {
  constexpr int D = DIM + 1;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  double A[D][D], r[D];
#pragma unroll
  for (int i = 0; i < D; ++i) {
    r[i] = mom[(size_t)ix.r[i] * P + p];
#pragma unroll
    for (int j = 0; j < D; ++j) A[i][j] = mom[(size_t)ix.a[i * D + j] * P + p];
  }
  uint8_t st;
  mu[p] = fit_point<D, double>(A, r, mom[(size_t)ix.n * P + p], st);
  if (status) status[p] = st;
}

// sigma2(t) = b0(t) - Gamma_hat(t, t) - mu_hat(t)^2 in place of b0 (Eq. 2.5 with the
// sign reading of the mean term); EMPTY fits give NaN.
template <typename TG>
__global__ void k_sigma2_curve(int P, const double* __restrict__ mu, const TG* __restrict__ gd,
                               long long gstride, const uint8_t* __restrict__ st,
                               double* __restrict__ sig) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const double b0 = sig[p];
  const bool empty = st ? st[p] == FPCA_PT_EMPTY : isnan(b0);
  sig[p] = empty ? __longlong_as_double(0x7ff8000000000000ll)
                 : b0 - (double)gd[(long long)p * gstride] - mu[p] * mu[p];
}

// Eq. (2.6): the mean of sigma2(t) over the domain nodes with a value (one block).
__global__ void k_sigma2_mean(int P, const double* __restrict__ sig, const int32_t* __restrict__ dom,
                              double* __restrict__ out) {
  __shared__ double rs[32], rc[32];
  double s = 0.0, c = 0.0;
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    const double v = sig[p];
    if ((!dom || dom[p] > 0) && !isnan(v)) {
      s += v;
      c += 1.0;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  if ((threadIdx.x & 31) == 0) {
    rs[threadIdx.x >> 5] = s;
    rc[threadIdx.x >> 5] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ts = 0.0, tc = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      ts += rs[w];
      tc += rc[w];
    }
    out[0] = tc > 0.0 ? ts / tc : __longlong_as_double(0x7ff8000000000000ll);
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

// ---------------------------------------------------------------------------
// t-side sweep + solve, register-blocked (d = 2, FP32)
// ---------------------------------------------------------------------------
// The 10 s-side arrays of row x_s are summed along t1 into 15 "mid" arrays
// (array a, t1-power a1) and along t2 into the 21 moment slots; the slots
// then feed the per-point solve.  One block handles HT rows of the t-plane:
//   phase 1  item = (mid array, column): HT outputs down one column from a
//            sliding window of input rows; tap weights read 4 at a time;
//   phase 2  item = (slot, row, SEG-column segment): SEG outputs along a row
//            of a mid array from a sliding window;
//   phase 3  one point per thread at a time: 21 slots -> A, r -> solve.
// Tap lists are zero-padded to a multiple of 4 (out-of-grid rows and
// columns are zero in shared memory), so the inner loops carry no bounds
// checks.  With COMP, every 4-tap partial is added to the running sum with
// Kahan compensation.
struct Hs2Geom {
  int P, R, C;
  int Tr, Tc;        // tap half-widths (t1, t2)
  int ntr, ntc;      // padded tap counts (multiples of 4)
  int nrp;           // input rows held per block: HT + ntr (the window preloads one spare row)
  int RS;            // mid row stride (odd, >= C + ntc)
  int SC;            // slot row stride (odd, >= C)
  int half;          // evaluate only t >= s (flat node order); see k_mirror_lower
};

template <bool COMP>
__device__ __forceinline__ void chunk_add(float& s, float& c, float p) {
  if constexpr (COMP) {
    const float y = p - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  } else {
    s += p;
  }
}

// NO outputs along a line: out[j] = sum_{k < nt} w[k] * x[(j + k) * stride].
// The next 4-tap chunk (inputs and weights) is loaded before the current one
// is summed, so shared-memory latency overlaps the FMAs.
template <int NO, bool COMP>
__device__ __forceinline__ void slide_sum(const float* __restrict__ x, int stride,
                                          const float4* __restrict__ w4, int nt, float (&out)[NO]) {
  float win[NO + 4];
#pragma unroll
  for (int j = 0; j < NO; ++j) win[j] = x[j * stride];
  float nxt[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) nxt[u] = x[(NO + u) * stride];
  float4 wn = w4[0];
  float sum[NO], cmp[NO];
#pragma unroll
  for (int j = 0; j < NO; ++j) {
    sum[j] = 0.f;
    cmp[j] = 0.f;
  }
#pragma unroll 2
  for (int kc = 0; kc < nt; kc += 4) {
    const float4 w = wn;
#pragma unroll
    for (int u = 0; u < 4; ++u) win[NO + u] = nxt[u];
    if (kc + 4 < nt) {
#pragma unroll
      for (int u = 0; u < 4; ++u) nxt[u] = x[(NO + kc + 4 + u) * stride];
      wn = w4[(kc >> 2) + 1];
    }
    if constexpr (COMP) {
#pragma unroll
      for (int j = 0; j < NO; ++j) {
        float p = w.x * win[j];
        p = fmaf(w.y, win[j + 1], p);
        p = fmaf(w.z, win[j + 2], p);
        p = fmaf(w.w, win[j + 3], p);
        chunk_add<true>(sum[j], cmp[j], p);
      }
    } else {
#pragma unroll
      for (int j = 0; j < NO; ++j) {
        sum[j] = fmaf(w.x, win[j], sum[j]);
        sum[j] = fmaf(w.y, win[j + 1], sum[j]);
        sum[j] = fmaf(w.z, win[j + 2], sum[j]);
        sum[j] = fmaf(w.w, win[j + 3], sum[j]);
      }
    }
#pragma unroll
    for (int j = 0; j < NO; ++j) win[j] = win[j + 4];
  }
#pragma unroll
  for (int j = 0; j < NO; ++j) out[j] = sum[j];
}

// 8-tap partial (4 when only one chunk is left) of a compensated sliding sum:
// plain FMAs inside the partial, then a Kahan add into the running sum (the
// first partial starts it).
template <int NO>
__device__ __forceinline__ void comp_partial8(const float* win, int b, float4 w, float4 w2,
                                              bool two, bool first, float (&sum)[NO],
                                              float (&cmp)[NO]) {
#pragma unroll
  for (int j = 0; j < NO; ++j) {
    float p = w.x * win[b + j];
    p = fmaf(w.y, win[b + j + 1], p);
    p = fmaf(w.z, win[b + j + 2], p);
    p = fmaf(w.w, win[b + j + 3], p);
    if (two) {
      p = fmaf(w2.x, win[b + j + 4], p);
      p = fmaf(w2.y, win[b + j + 5], p);
      p = fmaf(w2.z, win[b + j + 6], p);
      p = fmaf(w2.w, win[b + j + 7], p);
    }
    if (first) {
      sum[j] = p;
      cmp[j] = 0.f;
    } else {
      chunk_add<true>(sum[j], cmp[j], p);
    }
  }
}

// slide_sum with the chunk count NCH = nt / 4 fixed at compile time: the tap
// loop unrolls completely, so the sliding window needs no register shifts and
// no loop bookkeeping.  With COMP the partials span 8 taps (two chunks).
template <int NO, int NCH, bool COMP>
__device__ __forceinline__ void slide_sum_fixed(const float* __restrict__ x, int stride,
                                                const float4* __restrict__ w4, float (&out)[NO]) {
  constexpr int NW = NO + 4 * NCH;
  float win[NW];
#pragma unroll
  for (int j = 0; j < NW; ++j) win[j] = x[j * stride];
  float sum[NO], cmp[NO];
#pragma unroll
  for (int j = 0; j < NO; ++j) {
    sum[j] = 0.f;
    cmp[j] = 0.f;
  }
  if constexpr (COMP) {
#pragma unroll
    for (int kc = 0; kc < NCH; kc += 2) {
      const bool two = kc + 1 < NCH;
      comp_partial8<NO>(win, 4 * kc, w4[kc], two ? w4[kc + 1] : make_float4(0.f, 0.f, 0.f, 0.f),
                        two, kc == 0, sum, cmp);
    }
  }
#pragma unroll
  for (int kc = 0; kc < NCH; ++kc) {
    const float4 w = w4[kc];
    const int b = 4 * kc;
    if constexpr (!COMP) {
#pragma unroll
      for (int j = 0; j < NO; ++j) {
        sum[j] = fmaf(w.x, win[b + j], sum[j]);
        sum[j] = fmaf(w.y, win[b + j + 1], sum[j]);
        sum[j] = fmaf(w.z, win[b + j + 2], sum[j]);
        sum[j] = fmaf(w.w, win[b + j + 3], sum[j]);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < NO; ++j) out[j] = sum[j];
}

// slide_sum for any padded tap count: the fully unrolled form up to 40 taps
// (every bandwidth with h M < 20), the looped form beyond.
template <int NO, bool COMP>
__device__ __forceinline__ void slide_sum_any(const float* __restrict__ x, int stride,
                                              const float4* __restrict__ w4, int nt,
                                              float (&out)[NO]) {
  switch (nt >> 2) {
    case 1: slide_sum_fixed<NO, 1, COMP>(x, stride, w4, out); return;
    case 2: slide_sum_fixed<NO, 2, COMP>(x, stride, w4, out); return;
    case 3: slide_sum_fixed<NO, 3, COMP>(x, stride, w4, out); return;
    case 4: slide_sum_fixed<NO, 4, COMP>(x, stride, w4, out); return;
    case 5: slide_sum_fixed<NO, 5, COMP>(x, stride, w4, out); return;
    case 6: slide_sum_fixed<NO, 6, COMP>(x, stride, w4, out); return;
    case 7: slide_sum_fixed<NO, 7, COMP>(x, stride, w4, out); return;
    case 8: slide_sum_fixed<NO, 8, COMP>(x, stride, w4, out); return;
    case 9: slide_sum_fixed<NO, 9, COMP>(x, stride, w4, out); return;
    case 10: slide_sum_fixed<NO, 10, COMP>(x, stride, w4, out); return;
    default: slide_sum<NO, COMP>(x, stride, w4, nt, out); return;
  }
}

// weights in padded form: wp[row][k], k = 0..nt-1 <-> offset k - T (zero beyond 2T)
__device__ __forceinline__ void load_padded_weights(const double* __restrict__ tab, int T, int nt,
                                                    float* __restrict__ wp) {
  for (int e = threadIdx.x; e < TROWS * nt; e += blockDim.x) {
    const int row = e / nt, k = e - (e / nt) * nt;
    wp[e] = k <= 2 * T ? (float)tab[row * TW + TMAX + (k - T)] : 0.f;
  }
}

// One tile of the scalar t-side sweep: s-row xs, t-plane rows [a0, a0 + HT), the
// three phases of k_hsolve2 on the shared-memory layout below (sized by g; the
// weights wr, wc are loaded by the caller).  `parity` is the phase of the tile
// barrier to wait for.  Returns false if the bounded wait for the copies gave up
// (every thread returns the same value).
template <bool COMP, int C>
__device__ __forceinline__ bool hsolve2_tile(const float* __restrict__ varr, const Hs2Geom& g,
                                             int xs, int a0, const float* wr, const float* wc,
                                             float* mid, float* in, uint32_t bar, uint32_t parity,
                                             const double* __restrict__ mu_raw,
                                             float* __restrict__ gamma,
                                             uint8_t* __restrict__ status,
                                             const Epilogue<float>& ep, double* red,
                                             int* __restrict__ err, CvShared* cvs = nullptr) {
  const int P = g.P, R = g.R;
  float* slots = in;                                    // [NSL][HT][SC]
  const int th = min(HT, R - a0);
  const long long PP = (long long)P * P;
  // input rows a0 - Tr .. a0 - Tr + nrp - 1 of the t-plane, zero outside [0, R):
  // the in-grid rows of each array are one contiguous run in global memory,
  // fetched by the TMA engine (one bulk copy per array) while the threads
  // fill the padding rows.
  const int rlo = max(0, a0 - g.Tr), rhi = min(R, a0 - g.Tr + g.nrp);
  const int skip = rlo - (a0 - g.Tr);  // padding rows above the grid
  const uint32_t bytes = (uint32_t)((rhi - rlo) * C * sizeof(float));
  if (threadIdx.x == 0) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    ptx::mbar_arrive_expect_tx(bar, 10 * bytes);
    for (int a = 0; a < 10; ++a)
      ptx::bulk_load(ptx::smem_u32(in + ((size_t)a * g.nrp + skip) * C),
                     varr + a * PP + (long long)xs * P + (long long)rlo * C, bytes, bar);
  }
  {
    constexpr int C4 = C / 4;
    const int padrows = g.nrp - (rhi - rlo);
    for (int e = threadIdx.x; e < 10 * padrows * C4; e += NT2) {
      const int a = e / (padrows * C4);
      const int rem = e - a * padrows * C4;
      const int pr = rem / C4, c4 = rem % C4;
      const int r = pr < skip ? pr : (rhi - rlo) + pr;  // above, then below the copied rows
      *reinterpret_cast<float4*>(in + ((size_t)a * g.nrp + r) * C + 4 * c4) =
          make_float4(0.f, 0.f, 0.f, 0.f);
    }
    // zero the column padding of the mid rows
    const int padw = g.RS - C;
    for (int e = threadIdx.x; e < NMID * HT * padw; e += NT2) {
      const int line = e / padw, k = e - (e / padw) * padw;
      const int cp = k < g.Tc ? k : C + k;
      mid[(size_t)line * g.RS + cp] = 0.f;
    }
  }
  // bounded wait for the copies; the block leaves together if any thread gave up
  const bool landed = ptx::mbar_wait(bar, parity, err);
  if (__syncthreads_or(!landed)) return false;

  // phase 1: sums across t-plane rows
  for (int it = threadIdx.x; it < NMID * C; it += NT2) {
    const int m = it / C, c = it - (it / C) * C;
    const int a = c_mid_array[m], pw = c_mid_pow[m];
    float out[HT];
    slide_sum_any<HT, COMP>(in + (size_t)a * g.nrp * C + c, C,
                            reinterpret_cast<const float4*>(wr + pw * g.ntr), g.ntr, out);
    float* dst = mid + (size_t)m * HT * g.RS + g.Tc + c;
#pragma unroll
    for (int j = 0; j < HT; ++j) dst[j * g.RS] = out[j];
  }
  __syncthreads();

  // phase 2: sums along t-plane rows into the moment slots (aliasing `in`).
  // A warp covers 8 rows x 4 segments of one slot: with odd row strides its
  // loads and stores fall in 32 distinct banks.
  constexpr int NSEG = C / SEG;
  constexpr int SLO = NSEG < 4 ? NSEG : 4;
  for (int it = threadIdx.x; it < NSL * HT * NSEG; it += NT2) {
    const int s = it / (HT * NSEG);
    const int rem = it % (HT * NSEG);
    const int sg = (rem % SLO) + SLO * (rem / (SLO * HT));
    const int i = (rem / SLO) % HT;
    const int m = c_slot_mid[s], pw = c_slot_pow[s];
    float out[SEG];
    slide_sum_any<SEG, COMP>(mid + ((size_t)m * HT + i) * g.RS + sg * SEG, 1,
                             reinterpret_cast<const float4*>(wc + pw * g.ntc), g.ntc, out);
    float* dst = slots + ((size_t)s * HT + i) * g.SC + sg * SEG;
#pragma unroll
    for (int j = 0; j < SEG; ++j) dst[j] = out[j];
  }
  __syncthreads();

  tside_phase3<C, NT2>(slots, g.SC, g.half, g.P, xs, a0, th, mu_raw, gamma, status, ep, red, mid,
                       cvs);
  return true;
}

template <bool COMP, int C>
__global__ void __launch_bounds__(NT2, 2)
    k_hsolve2(const float* __restrict__ varr, Hs2Geom g, const double* __restrict__ tabr,
              const double* __restrict__ tabc, const double* __restrict__ mu_raw,
              float* __restrict__ gamma, uint8_t* __restrict__ status, Epilogue<float> ep,
              int* __restrict__ err) {
  static_assert(C % SEG == 0 && C <= 64, "t-plane width");
  extern __shared__ __align__(128) unsigned char hs2[];
  __shared__ double red[NT2 / 32];
  __shared__ __align__(8) uint64_t tile_bar;
  float* wr = reinterpret_cast<float*>(hs2);          // [TROWS][ntr]
  float* wc = wr + TROWS * g.ntr;                       // [TROWS][ntc]
  float* mid = wc + TROWS * g.ntc;                      // [NMID][HT][RS]
  float* in = mid + (size_t)NMID * HT * g.RS;           // [10][nrp][C]; later the slots
  // (the sliding windows read input rows < HT + ntr = nrp and mid columns
  //  < C + ntc <= RS, so every load stays inside these arrays)
  const int xs = blockIdx.y;
  const int a0 = blockIdx.x * HT;
  const int th = min(HT, g.R - a0);
  // Gamma_hat(s, t) = Gamma_hat(t, s) exactly (one bandwidth for s and t, symmetric
  // bins), so in half mode a block whose t-rows all lie before s has nothing to do
  if (g.half && (a0 + th) * C <= xs) return;
  const uint32_t bar = ptx::smem_u32(&tile_bar);
  if (threadIdx.x == 0) {
    ptx::mbar_init(bar, 1);
    ptx::fence_mbar_init();
  }
  load_padded_weights(tabr, g.Tr, g.ntr, wr);
  load_padded_weights(tabc, g.Tc, g.ntc, wc);
  __syncthreads();
  hsolve2_tile<COMP, C>(varr, g, xs, a0, wr, wc, mid, in, bar, 0, mu_raw, gamma, status, ep, red,
                        err);
}

// The CV grid's (bandwidth, fold) items through the scalar sweep in one
// persistent launch: CTAs pull tiles (item-major, then s-row, then t1 block)
// from a counter and run hsolve2_tile on each; the shared memory is sized for the
// widest window of the grid.  Per item: its s-side arrays, tap tables and geometry,
// and the epilogue of its fold (CV terms into its own accumulators).
struct CvGridItem {
  const float* varr;
  const double* tab;   // per-axis tables (TROWS x TW each) of the item's bandwidth
  Hs2Geom g;
  Epilogue<float> ep;
  int item;            // index of the item (escalation queue)
};

template <bool COMP, int C>
__global__ void __launch_bounds__(NT2, 2)
    k_hsolve2_grid(const CvGridItem* __restrict__ items, int nitems, int nblk,
                   unsigned* __restrict__ counter, int ntr_max, int ntc_max, int rs_max,
                   int* __restrict__ esc_item, int* __restrict__ err) {
  static_assert(C % SEG == 0 && C <= 64, "t-plane width");
  extern __shared__ __align__(128) unsigned char hs2g[];
  __shared__ double red[NT2 / 32];
  __shared__ __align__(8) uint64_t tile_bar;
  __shared__ int work;
  float* wr = reinterpret_cast<float*>(hs2g);           // [TROWS][ntr_max]
  float* wc = wr + TROWS * ntr_max;                       // [TROWS][ntc_max]
  float* mid = wc + TROWS * ntc_max;                      // [NMID][HT][rs_max]
  float* in = mid + (size_t)NMID * HT * rs_max;           // [10][nrp][C]; later the slots
  const uint32_t bar = ptx::smem_u32(&tile_bar);
  if (threadIdx.x == 0) {
    ptx::mbar_init(bar, 1);
    ptx::fence_mbar_init();
  }
  __syncthreads();
  int cur = -1;  // item whose weights are in shared memory
  uint32_t parity = 0;
  const int total = nitems * nblk;
  // CV terms of the current item gathered in shared memory, added to its accumulators
  // when the CTA moves on to another item (one flush per item, not a reduction per tile)
  __shared__ CvShared cvs;
  if (threadIdx.x == 0) cvs.v[0] = cvs.v[1] = cvs.v[2] = 0.0;
  __syncthreads();
  auto flush = [&]() {
    if (cur >= 0) cv_flush(&cvs, items[cur].ep.cvacc);
  };
  while (true) {
    if (threadIdx.x == 0) {
      int w = (int)atomicAdd(counter, 1u);
      // skip tiles with nothing to do (half mode) without a barrier each
      while (w < total) {
        const int it = w / nblk, r = w - it * nblk;
        const Hs2Geom& g = items[it].g;
        const int nb = (g.R + HT - 1) / HT;
        const int xs = r / nb, a0 = (r - xs * nb) * HT;
        const int th = min(HT, g.R - a0);
        if (!(g.half && (a0 + th) * C <= xs)) break;
        w = (int)atomicAdd(counter, 1u);
      }
      work = w;
    }
    __syncthreads();
    const int w = work;
    if (w >= total) break;
    const int it = w / nblk, r = w - it * nblk;
    const CvGridItem& I = items[it];
    const int nb = (I.g.R + HT - 1) / HT;
    const int xs = r / nb, a0 = (r - xs * nb) * HT;
    if (it != cur) {
      flush();
      load_padded_weights(I.tab, I.g.Tr, I.g.ntr, wr);
      load_padded_weights(I.tab + TROWS * TW, I.g.Tc, I.g.ntc, wc);
      cur = it;
    }
    Epilogue<float> ep = I.ep;
    if (ep.esc_count) ep.esc_idx_item = esc_item, ep.esc_item_id = I.item;
    if (!hsolve2_tile<COMP, C>(I.varr, I.g, xs, a0, wr, wc, mid, in, bar, parity, nullptr,
                               nullptr, nullptr, ep, red, err, &cvs))
      return;
    parity ^= 1u;
    __syncthreads();  // the slots alias the next tile's input rows
  }
  flush();
}

// NO outputs x NP powers along a line from one sliding window:
// out[p][j] = sum_{k < nt} w_p[k] * x[(j + k) * stride].
template <int NO, int NP, bool COMP>
__device__ __forceinline__ void slide_sum_multi(const float* __restrict__ x, int stride,
                                                const float4* const (&w4)[NP], int nt,
                                                float (&out)[NP][NO]) {
  float win[NO + 4];
#pragma unroll
  for (int j = 0; j < NO; ++j) win[j] = x[j * stride];
  float nxt[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) nxt[u] = x[(NO + u) * stride];
  float sum[NP][NO], cmp[NP][NO];
#pragma unroll
  for (int q = 0; q < NP; ++q)
#pragma unroll
    for (int j = 0; j < NO; ++j) {
      sum[q][j] = 0.f;
      cmp[q][j] = 0.f;
    }
#pragma unroll 2
  for (int kc = 0; kc < nt; kc += 4) {
#pragma unroll
    for (int u = 0; u < 4; ++u) win[NO + u] = nxt[u];
    if (kc + 4 < nt) {
#pragma unroll
      for (int u = 0; u < 4; ++u) nxt[u] = x[(NO + kc + 4 + u) * stride];
    }
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      const float4 w = w4[q][kc >> 2];
      if constexpr (COMP) {
#pragma unroll
        for (int j = 0; j < NO; ++j) {
          float pp = w.x * win[j];
          pp = fmaf(w.y, win[j + 1], pp);
          pp = fmaf(w.z, win[j + 2], pp);
          pp = fmaf(w.w, win[j + 3], pp);
          chunk_add<true>(sum[q][j], cmp[q][j], pp);
        }
      } else {
#pragma unroll
        for (int j = 0; j < NO; ++j) {
          sum[q][j] = fmaf(w.x, win[j], sum[q][j]);
          sum[q][j] = fmaf(w.y, win[j + 1], sum[q][j]);
          sum[q][j] = fmaf(w.z, win[j + 2], sum[q][j]);
          sum[q][j] = fmaf(w.w, win[j + 3], sum[q][j]);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < NO; ++j) win[j] = win[j + 4];
  }
#pragma unroll
  for (int q = 0; q < NP; ++q)
#pragma unroll
    for (int j = 0; j < NO; ++j) out[q][j] = sum[q][j];
}

// slide_sum_multi with NCH = nt / 4 fixed at compile time (12-tap partials with COMP).
template <int NO, int NP, int NCH, bool COMP>
__device__ __forceinline__ void slide_sum_multi_fixed(const float* __restrict__ x, int stride,
                                                      const float4* const (&w4)[NP],
                                                      float (&out)[NP][NO]) {
  constexpr int NW = NO + 4 * NCH;
  float win[NW];
#pragma unroll
  for (int j = 0; j < NW; ++j) win[j] = x[j * stride];
  float sum[NP][NO], cmp[NP][NO];
#pragma unroll
  for (int q = 0; q < NP; ++q)
#pragma unroll
    for (int j = 0; j < NO; ++j) {
      sum[q][j] = 0.f;
      cmp[q][j] = 0.f;
    }
  if constexpr (COMP) {
    // partials of up to 12 taps (three chunks), Kahan-added: one compensation step per
    // output for windows up to 24 taps, where 8-tap partials need two from 17 taps on
    // (these passes are bound by their instruction count)
#pragma unroll
    for (int kc = 0; kc < NCH; kc += 3) {
      const int nch = NCH - kc < 3 ? NCH - kc : 3;
#pragma unroll
      for (int q = 0; q < NP; ++q) {
#pragma unroll
        for (int j = 0; j < NO; ++j) {
          float p = 0.f;
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            if (c >= nch) break;
            const float4 w = w4[q][kc + c];
            const int b = 4 * (kc + c) + j;
            p = (c == 0) ? w.x * win[b] : fmaf(w.x, win[b], p);
            p = fmaf(w.y, win[b + 1], p);
            p = fmaf(w.z, win[b + 2], p);
            p = fmaf(w.w, win[b + 3], p);
          }
          if (kc == 0) {
            sum[q][j] = p;
          } else {
            chunk_add<true>(sum[q][j], cmp[q][j], p);
          }
        }
      }
    }
  }
#pragma unroll
  for (int kc = 0; kc < NCH; ++kc) {
    const int b = 4 * kc;
#pragma unroll
    for (int q = 0; q < NP; ++q) {
      const float4 w = w4[q][kc];
      if constexpr (!COMP) {
#pragma unroll
        for (int j = 0; j < NO; ++j) {
          sum[q][j] = fmaf(w.x, win[b + j], sum[q][j]);
          sum[q][j] = fmaf(w.y, win[b + j + 1], sum[q][j]);
          sum[q][j] = fmaf(w.z, win[b + j + 2], sum[q][j]);
          sum[q][j] = fmaf(w.w, win[b + j + 3], sum[q][j]);
        }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < NP; ++q)
#pragma unroll
    for (int j = 0; j < NO; ++j) out[q][j] = sum[q][j];
}

template <int NO, int NP, bool COMP>
__device__ __forceinline__ void slide_sum_multi_any(const float* __restrict__ x, int stride,
                                                    const float4* const (&w4)[NP], int nt,
                                                    float (&out)[NP][NO]) {
  switch (nt >> 2) {
    case 1: slide_sum_multi_fixed<NO, NP, 1, COMP>(x, stride, w4, out); return;
    case 2: slide_sum_multi_fixed<NO, NP, 2, COMP>(x, stride, w4, out); return;
    case 3: slide_sum_multi_fixed<NO, NP, 3, COMP>(x, stride, w4, out); return;
    case 4: slide_sum_multi_fixed<NO, NP, 4, COMP>(x, stride, w4, out); return;
    case 5: slide_sum_multi_fixed<NO, NP, 5, COMP>(x, stride, w4, out); return;
    case 6: slide_sum_multi_fixed<NO, NP, 6, COMP>(x, stride, w4, out); return;
    case 7: slide_sum_multi_fixed<NO, NP, 7, COMP>(x, stride, w4, out); return;
    case 8: slide_sum_multi_fixed<NO, NP, 8, COMP>(x, stride, w4, out); return;
    case 9: slide_sum_multi_fixed<NO, NP, 9, COMP>(x, stride, w4, out); return;
    case 10: slide_sum_multi_fixed<NO, NP, 10, COMP>(x, stride, w4, out); return;
    default: slide_sum_multi<NO, NP, COMP>(x, stride, w4, nt, out); return;
  }
}

// s-side pass (FP32): one block = one line (Ma rows along the pass axis) x
// 128 columns of one input array; rows padded with zeros above and below.
constexpr int VROWS = 8;  // outputs per sliding window
template <int NP, bool COMP>
__device__ __forceinline__ void vpass2_line(const VJob& jb, const float* tile, const float* wp,
                                            int ntp, int Ma, int stride, long long base, int P,
                                            int col) {
  // Ma: the rows of the line computed here (a prefix of it, see SBand)
  const float4* w4[NP];
#pragma unroll
  for (int q = 0; q < NP; ++q) w4[q] = reinterpret_cast<const float4*>(wp + jb.row[q] * ntp);
  for (int x0 = 0; x0 < Ma; x0 += VROWS) {
    float out[NP][VROWS];
    slide_sum_multi_any<VROWS, NP, COMP>(tile + (size_t)x0 * VCOLS + threadIdx.x, VCOLS, w4, ntp,
                                         out);
#pragma unroll
    for (int j = 0; j < VROWS; ++j) {
      const int x = x0 + j;
      if (x < Ma) {
        const long long o = (base + (long long)x * stride) * P + col;
#pragma unroll
        for (int q = 0; q < NP; ++q) static_cast<float*>(jb.out[q])[o] = out[q][j];
      }
    }
  }
}

// The part of the s-side outputs that a half-mode t-side sweep (t >= s) reads, for
// d = 2: entry (s1, s2; t1, t2) is read iff t1 >= HT floor(s1 / HT) - T0 (the blocks
// of t-rows that reach past s, widened by the t1 window).  For a column block whose
// largest t1 is t1max that means s1 < need = HT (floor((t1max + T0) / HT) + 1).
// mode 1 (the s2 pass, one line per s1): a line is skipped when s1 >= need + T0 (the
// s1 pass reads s1 +- T0); mode 2 (the s1 pass, lines along s1): rows s1 < need are
// computed from the rows s1 < need + T0.
struct SBand {
  int mode;  // 0: every row
  int R, C, T0;
};

template <bool COMP>
__global__ void __launch_bounds__(VCOLS)
    k_vpass2(VJobs jobs, int P, int Ma, int stride, int taps, int ntp,
             const double* __restrict__ tab, int bulk, SBand band, int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char vsm2[];
  __shared__ __align__(8) uint64_t vbar;
  float* wp = reinterpret_cast<float*>(vsm2);  // [TROWS][ntp]
  float* tile = wp + TROWS * ntp;              // [Ma + ntp + VROWS][VCOLS], row r <-> x = r - taps
  const int nrow = ((Ma + VROWS - 1) / VROWS) * VROWS + ntp;
  float* subt = tile + (size_t)nrow * VCOLS;   // [Ma][VCOLS] when a job subtracts a fold
  const VJob& jb = jobs.j[blockIdx.z];
  const int col0 = blockIdx.x * VCOLS;
  const int col = col0 + threadIdx.x;
  const int L = blockIdx.y;
  const long long base = (long long)(L / stride) * Ma * stride + (L % stride);
  int Mcomp = Ma, Mload = Ma;  // rows computed, rows read
  if (band.mode) {
    const int t1max = min(band.R - 1, (min(P, col0 + VCOLS) - 1) / band.C);
    const int need = min(band.R, ((t1max + band.T0) / HT + 1) * HT);
    if (band.mode == 1) {
      if (L >= min(band.R, need + band.T0)) return;  // this line's s1 is never read
    } else {
      Mcomp = min(Ma, need);
      Mload = min(Ma, need + band.T0);
    }
  }
  if (bulk) {
    // one bulk copy per tile row (and per fold row), all on one mbarrier
    const int ncols = min(VCOLS, P - col0);
    const uint32_t rbytes = (uint32_t)ncols * 4u;
    const uint32_t bar = ptx::smem_u32(&vbar);
    if (threadIdx.x == 0) {
      ptx::mbar_init(bar, 1);
      ptx::fence_mbar_init();
    }
    __syncthreads();
    const int nsrc = jb.sub ? 2 : 1;
    if (threadIdx.x == 0) ptx::mbar_arrive_expect_tx(bar, rbytes * (uint32_t)(Mload * nsrc));
    __syncwarp();
    if (threadIdx.x < 32) {
      for (int x = threadIdx.x; x < Mload; x += 32) {
        const long long e = (base + (long long)x * stride) * P + col0;
        ptx::bulk_load(ptx::smem_u32(tile + (size_t)(x + taps) * VCOLS),
                       static_cast<const float*>(jb.in) + e, rbytes, bar);
        if (jb.sub)
          ptx::bulk_load(ptx::smem_u32(subt + (size_t)x * VCOLS),
                         static_cast<const float*>(jb.sub) + e, rbytes, bar);
      }
    }
    load_padded_weights(tab, taps, ntp, wp);
    for (int r = 0; r < nrow; ++r)
      if (r < taps || r >= taps + Mload) tile[(size_t)r * VCOLS + threadIdx.x] = 0.f;
    const bool landed = ptx::mbar_wait(bar, 0, err);
    if (__syncthreads_or(!landed)) return;
    if (jb.in_int || jb.sub) {
      for (int x = 0; x < Mload; ++x) {
        float* tv = tile + (size_t)(x + taps) * VCOLS + threadIdx.x;
        if (jb.in_int) {
          int c = __float_as_int(*tv);
          if (jb.sub) c -= __float_as_int(subt[(size_t)x * VCOLS + threadIdx.x]);
          *tv = c > 0 ? 1.f : 0.f;
        } else {
          *tv -= subt[(size_t)x * VCOLS + threadIdx.x];
        }
      }
    }
  } else {
    load_padded_weights(tab, taps, ntp, wp);
    // rows in batches of 8 so that eight global loads are in flight per thread
    for (int r0 = 0; r0 < nrow; r0 += 8) {
      float vals[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int x = r0 + u - taps;
        float val = 0.f;
        if (col < P && x >= 0 && x < Mload && r0 + u < nrow) {
          const long long e = (base + (long long)x * stride) * P + col;
          if (jb.in_int) {
            int c = __ldg(static_cast<const int32_t*>(jb.in) + e);
            if (jb.sub) c -= __ldg(static_cast<const int32_t*>(jb.sub) + e);
            val = c > 0 ? 1.f : 0.f;
          } else {
            val = __ldg(static_cast<const float*>(jb.in) + e);
            if (jb.sub) val -= __ldg(static_cast<const float*>(jb.sub) + e);
          }
        }
        vals[u] = val;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (r0 + u < nrow) tile[(size_t)(r0 + u) * VCOLS + threadIdx.x] = vals[u];
    }
  }
  __syncthreads();
  if (col >= P) return;
  if (jb.npow == 3)
    vpass2_line<3, COMP>(jb, tile, wp, ntp, Mcomp, stride, base, P, col);
  else if (jb.npow == 2)
    vpass2_line<2, COMP>(jb, tile, wp, ntp, Mcomp, stride, base, P, col);
  else
    vpass2_line<1, COMP>(jb, tile, wp, ntp, Mcomp, stride, base, P, col);
}

size_t vpass2_smem(int Ma, int ntp, bool with_sub) {
  const int nrow = ((Ma + VROWS - 1) / VROWS) * VROWS + ntp;
  return sizeof(float) * ((size_t)TROWS * ntp + (size_t)nrow * VCOLS +
                          (with_sub ? (size_t)Ma * VCOLS : 0));
}

// Float-float fits of the queued (escalated) points, whose FP32 elimination met a
// pivot below ESCALATE_F32 of its diagonal: one thread per point; writes
// Gamma_hat, status and the epilogue terms the t-side kernel skipped.
__global__ void __launch_bounds__(256)
    k_escalated(int P, const float* __restrict__ esc_slots, const int2* __restrict__ esc_idx,
                const unsigned* __restrict__ esc_count, int cap, const double* __restrict__ mu_raw,
                float* __restrict__ gamma, uint8_t* __restrict__ status, Epilogue<float> ep0,
                int half, const CvGridItem* __restrict__ items = nullptr,
                const int* __restrict__ esc_item = nullptr) {
  const unsigned n = min(*esc_count, (unsigned)cap);
  for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const float* sl = esc_slots + (size_t)e * NSL;
    const int2 id = esc_idx[e];
    // batched CV grid: the queued point's own item (its fold's epilogue)
    const Epilogue<float>& ep = items ? items[esc_item[e]].ep : ep0;
    // the 5 x 5 system in float-float: symmetric elimination in the order of
    // elim_solve, pivot ratios against the original diagonal, inverses of the
    // pivots reused by the back substitution
    ff::F2 A[5][5], r[5], inv[5];
    float diag[5];
#pragma unroll
    for (int i2 = 0; i2 < 5; ++i2) {
      r[i2] = ff::make(sl[rslot(2, i2)]);
#pragma unroll
      for (int j2 = i2; j2 < 5; ++j2) {
        A[i2][j2] = ff::make(sl[aslot(2, i2, j2)]);
        A[j2][i2] = A[i2][j2];
      }
      diag[i2] = A[i2][i2].hi;
    }
    const double lc = (double)r[0].hi / (double)A[0][0].hi;
    float minratio = 1e30f;
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      const ff::F2 piv = A[k][k];
      const float ratio = diag[k] > 0.f ? piv.hi / diag[k] : -1.f;
      minratio = fminf(minratio, ratio);
      if (!(piv.hi > 0.f)) {
        ok = false;
        break;
      }
      inv[k] = ff::recip(piv);
#pragma unroll
      for (int i = k + 1; i < 5; ++i) {
        const ff::F2 l = ff::mul(A[k][i], inv[k]);
#pragma unroll
        for (int j = i; j < 5; ++j) A[i][j] = ff::sub_mul(A[i][j], l, A[k][j]);
        r[i] = ff::sub_mul(r[i], l, r[k]);
      }
    }
    double g = lc;
    uint8_t st = FPCA_PT_FALLBACK;
    if (ok && (double)minratio > PIVOT_RTOL_F32) {
      ff::F2 x[5];
#pragma unroll
      for (int k = 4; k >= 0; --k) {
        ff::F2 sacc = r[k];
#pragma unroll
        for (int j = k + 1; j < 5; ++j) sacc = ff::sub_mul(sacc, A[k][j], x[j]);
        x[k] = ff::mul(sacc, inv[k]);
      }
      g = ff::to_double(x[0]);
      st = FPCA_PT_OK;
    }
    if (mu_raw) g -= mu_raw[id.x] * mu_raw[id.y];
    const long long o = (long long)id.x * P + id.y;
    const float gv = (float)g;
    if (gamma) gamma[o] = gv;
    if (status) status[o] = st;
    if (ep.cvacc) {
      const double mul = (half && id.y != id.x) ? 2.0 : 1.0;  // (s, t) stands for (t, s) too
      const double wf = (double)ep.wf[o];
      atomicAdd(ep.cvacc + 0, mul * ((double)ep.qf[o] - 2.0 * g * (double)ep.vf[o] + g * g * wf));
      atomicAdd(ep.cvacc + 1, mul * wf);
    }
    if (ep.y)
      for (int c = 0; c < ep.l; ++c)
        atomicAdd(ep.y + (long long)id.x * ep.l + c, gv * ep.omega[(long long)id.y * ep.l + c]);
  }
}

// Lower triangle (t < s in flat node order) of Gamma_hat and of its status from
// the upper one after a half-mode t-side sweep (Gamma_hat(t, s) = Gamma_hat(s, t)):
// one block per lower 64 x 64 tile pair, its source tile loaded with every load in
// flight at once, then transposed through shared memory.
constexpr int MIR_T = 64;  // mirror tile edge
__global__ void __launch_bounds__(256)
    k_mirror_lower(int P, float* __restrict__ gamma, uint8_t* __restrict__ status) {
  __shared__ float tg[MIR_T][MIR_T + 1];
  __shared__ uint8_t ts[MIR_T][MIR_T + 4];
  // lower tile pair L -> destination rows bi*64.., columns bj*64.., bj <= bi
  const int L = blockIdx.x;
  int bi = 0;
  while ((bi + 1) * (bi + 2) / 2 <= L) ++bi;
  const int bj = L - bi * (bi + 1) / 2;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  // all loads of the source tile (bj, bi) first: 8 rows x 2 columns per thread
  float gv[8][2];
  uint8_t sv[8][2];
#pragma unroll
  for (int k = 0; k < 8; ++k)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int sr = bj * MIR_T + ty + 8 * k, sc = bi * MIR_T + tx + 32 * h;
      const bool in = sr < P && sc < P;
      const long long o = (long long)sr * P + sc;
      gv[k][h] = (gamma && in) ? gamma[o] : 0.f;
      sv[k][h] = (status && in) ? status[o] : 0;
    }
#pragma unroll
  for (int k = 0; k < 8; ++k)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      tg[ty + 8 * k][tx + 32 * h] = gv[k][h];
      ts[ty + 8 * k][tx + 32 * h] = sv[k][h];
    }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 8; ++k)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = ty + 8 * k, c = tx + 32 * h;
      const int dr = bi * MIR_T + r, dc = bj * MIR_T + c;
      if (dr < P && dc < dr) {
        const long long o = (long long)dr * P + dc;
        if (gamma) gamma[o] = tg[c][r];
        if (status) status[o] = ts[c][r];
      }
    }
}

// Geometry of k_hsolve2 for a d = 2 grid and tap half-widths (Tr on t1, Tc on t2).
Hs2Geom hs2_geometry(int P, int M1, int M2, int Tr, int Tc) {
  Hs2Geom g{};
  g.P = P;
  g.R = M1;
  g.C = M2;
  g.Tr = Tr;
  g.Tc = Tc;
  g.ntr = ((2 * Tr + 1) + 3) / 4 * 4;
  g.ntc = ((2 * Tc + 1) + 3) / 4 * 4;
  g.nrp = HT + g.ntr;
  g.RS = (M2 + g.ntc) | 1;
  g.SC = M2 | 1;
  return g;
}

size_t hs2_smem(const Hs2Geom& g) {
  const size_t in_f = (size_t)10 * g.nrp * g.C;
  const size_t slot_f = (size_t)NSL * HT * g.SC;
  return sizeof(float) * ((size_t)TROWS * (g.ntr + g.ntc) + (size_t)NMID * HT * g.RS +
                          (in_f > slot_f ? in_f : slot_f));
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

template <bool COMP, int C>
void launch_hsolve2(fpca_ctx* ctx, dim3 grid, size_t smem, const float* varr, const Hs2Geom& g,
                    const double* tabr, const double* tabc, const double* mu_raw, float* gamma,
                    uint8_t* status, const Epilogue<float>& ep) {
  cudaFuncSetAttribute(k_hsolve2<COMP, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_hsolve2<COMP, C><<<grid, NT2, smem, ctx->stream>>>(varr, g, tabr, tabc, mu_raw, gamma, status,
                                                       ep, ctx->d_err);
}

// Launches one s-side pass: njobs input arrays, lines of Ma rows at row
// stride `stride`, `lines` lines.  FP32 uses the sliding-window kernel.
template <typename T, bool COMP>
bool launch_vpass(fpca_ctx* ctx, const VJobs& jobs, int njobs, int P, int Ma, int stride, int lines,
                  int taps, const double* tab, SBand band = SBand{}) {
  const dim3 grid((P + VCOLS - 1) / VCOLS, lines, njobs);
  if constexpr (sizeof(T) == 4) {
    const int ntp = ((2 * taps + 1) + 3) / 4 * 4;
    bool with_sub = false;
    for (int j = 0; j < njobs; ++j) with_sub = with_sub || jobs.j[j].sub != nullptr;
    const size_t sm = vpass2_smem(Ma, ntp, with_sub);
    // bulk row copies need 16-byte aligned rows: P a multiple of 4
    const int bulk = (P % 4 == 0) ? 1 : 0;
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_vpass2<COMP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)vpass2_smem(64, 128, true));
      attr = true;
    }
    k_vpass2<COMP><<<grid, VCOLS, sm, ctx->stream>>>(jobs, P, Ma, stride, taps, ntp, tab, bulk,
                                                     band, ctx->d_err);
  } else {
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute(k_vpass<T, COMP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(sizeof(T) * (TROWS * TW + (size_t)64 * VCOLS)));
      attr = true;
    }
    k_vpass<T, COMP><<<grid, VCOLS, sizeof(T) * (TROWS * TW + (size_t)Ma * VCOLS), ctx->stream>>>(
        jobs, P, Ma, stride, taps, tab);
  }
  return true;
}

// One smoothing pass of the P x P bins (optionally train = pooled - sub_*).
template <typename T, bool COMP>
fpca_status cov_smooth_one(fpca_ctx* ctx, const fpca_grid* g, const int32_t* cnt, const T* w,
                           const T* v, const int32_t* sub_cnt, const T* sub_w, const T* sub_v,
                           const double* h, const double* tab, T* mids, T* varr,
                           const double* mu_raw, T* gamma, uint8_t* status, Epilogue<T> ep,
                           bool symmetric, bool sside_only = false) {
  const int d = g->d;
  const int P = grid_P(g);
  const long long PP = (long long)P * P;
  const int Tax[2] = {host_taps(h[0], g->m[0]), d > 1 ? host_taps(h[1], g->m[1]) : 0};
  auto tabk = [&](int k) { return tab + (size_t)k * TROWS * TW; };
  // sside_only: the s-side passes into varr and nothing else (the batched CV grid
  // runs every item's t-side in one launch, in half mode)
  if (d == 2) {
    const int M1 = g->m[0], M2 = g->m[1];
    // Will the t-side run in half mode (FP32 sweep kernel, symmetric bins, no fused
    // y)?  Then the s-side passes only produce the band it reads (SBand).
    bool half2 = false;
    bool use_ts = false;
    if constexpr (sizeof(T) == 4) {
      use_ts = tsweep_built(M2, Tax[0], Tax[1]) &&
               ts_smem(ts_geometry(P, M1, M2, Tax[0], Tax[1])) <= ctx->smem_optin &&
               ctx->tside_kernel != 1;  // 1: the scalar sweep only
      if ((M2 == 8 || M2 == 16 || M2 == 32 || M2 == 64) && symmetric && !ep.y)
        half2 = use_ts || hs2_smem(hs2_geometry(P, M1, M2, Tax[0], Tax[1])) <= ctx->smem_optin;
    }
    const SBand band1{half2 ? 1 : 0, M1, M2, Tax[0]};
    const SBand band2{half2 ? 2 : 0, M1, M2, Tax[0]};
    // pass along s2 (axis 1): rows L*M2 + a
    VJobs j1{};
    j1.j[0] = VJob{w, sub_w, 0, 3, {0, 1, 2}, {mids + 0 * PP, mids + 1 * PP, mids + 2 * PP}};
    j1.j[1] = VJob{v, sub_v, 0, 2, {0, 1, 0}, {mids + 3 * PP, mids + 4 * PP, nullptr}};
    j1.j[2] = VJob{cnt, sub_cnt, 1, 1, {3, 0, 0}, {mids + 5 * PP, nullptr, nullptr}};
    if (!launch_vpass<T, COMP>(ctx, j1, 3, P, M2, 1, M1, Tax[1], tabk(1), band1))
      return fpca_check_launch(ctx, "cov_vpass_s2");
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
    if (!launch_vpass<T, COMP>(ctx, j2, 6, P, M1, M2, M2, Tax[0], tabk(0), band2))
      return fpca_check_launch(ctx, "cov_vpass_s1");
    FPCA_LAUNCHED(ctx, "cov_vpass_s1");
    if (sside_only) return FPCA_OK;
    // t-side + solve
    if constexpr (sizeof(T) == 4) {
      Hs2Geom hg = hs2_geometry(P, M1, M2, Tax[0], Tax[1]);
      const bool hs_ok = (M2 == 8 || M2 == 16 || M2 == 32 || M2 == 64) &&
                         hs2_smem(hg) <= ctx->smem_optin;
      if (use_ts || hs_ok) {
        TsGeom tg = ts_geometry(P, M1, M2, Tax[0], Tax[1]);
        // symmetric bins: t >= s only, the rest mirrored (the fused y = Gamma_hat Omega
        // needs every row); decided above with the s-side band
        tg.half = half2 ? 1 : 0;
        hg.half = half2 ? 1 : 0;
        const float* va = reinterpret_cast<const float*>(varr);
        float* gm = reinterpret_cast<float*>(gamma);
        const Epilogue<float>& ef = *reinterpret_cast<const Epilogue<float>*>(&ep);
        auto run_ts = [&](const Epilogue<float>& e) {
          return tsweep_launch(M2, ctx, COMP, Tax[0], ts_smem(tg), va, tg, tabk(0), tabk(1),
                               mu_raw, gm, status, e);
        };
        auto run_hs = [&](const Epilogue<float>& e) {
          const dim3 grid((M1 + HT - 1) / HT, P);
          const size_t sm2 = hs2_smem(hg);
          switch (M2) {
            case 8: launch_hsolve2<COMP, 8>(ctx, grid, sm2, va, hg, tabk(0), tabk(1), mu_raw, gm, status, e); break;
            case 16: launch_hsolve2<COMP, 16>(ctx, grid, sm2, va, hg, tabk(0), tabk(1), mu_raw, gm, status, e); break;
            case 32: launch_hsolve2<COMP, 32>(ctx, grid, sm2, va, hg, tabk(0), tabk(1), mu_raw, gm, status, e); break;
            default: launch_hsolve2<COMP, 64>(ctx, grid, sm2, va, hg, tabk(0), tabk(1), mu_raw, gm, status, e); break;
          }
          return true;
        };
        bool packed = use_ts;
        if (use_ts && hs_ok && ctx->tside_kernel == 0) {
          // autotune: both sweeps built for this grid and these windows; time each
          // once (twice, keeping the faster run) and remember the faster in the context
          const std::array<int, 6> key = {M1, M2, Tax[0], Tax[1], COMP ? 1 : 0, tg.half};
          auto it = ctx->tside_choice.find(key);
          if (it == ctx->tside_choice.end()) {
            if (fpca_no_capture(ctx, "timing the t-side sweeps") != FPCA_OK)
              return FPCA_E_UNSUPPORTED;
            Epilogue<float> e = ef;  // no accumulating epilogues, escalations solved in place
            e.cvacc = nullptr;
            e.y = nullptr;
            e.esc_count = nullptr;
            cudaEvent_t ev[5];
            for (auto& x : ev) cudaEventCreate(&x);
            cudaEventRecord(ev[0], ctx->stream);
            for (int rep = 0; rep < 2; ++rep) {
              run_ts(e);
              cudaEventRecord(ev[1 + 2 * rep], ctx->stream);
              run_hs(e);
              cudaEventRecord(ev[2 + 2 * rep], ctx->stream);
            }
            ctx->launches += 4;
            fpca_status st = fpca_check_launch(ctx, "t-side autotune");
            if (st == FPCA_OK && cudaEventSynchronize(ev[4]) != cudaSuccess)
              st = fpca_check_launch(ctx, "t-side autotune");
            float t[4] = {0.f, 0.f, 0.f, 0.f};
            for (int q = 0; q < 4; ++q) cudaEventElapsedTime(&t[q], ev[q], ev[q + 1]);
            for (auto& x : ev) cudaEventDestroy(x);
            if (st != FPCA_OK) return st;
            const float tts = std::min(t[0], t[2]), ths = std::min(t[1], t[3]);
            it = ctx->tside_choice.emplace(key, tts <= ths ? 2 : 1).first;
          }
          packed = it->second == 2;
        }
        if (ef.esc_count) cudaMemsetAsync(ef.esc_count, 0, sizeof(unsigned), ctx->stream);
        if (packed) {
          if (!run_ts(ef))
            return fpca_fail(ctx, FPCA_E_UNSUPPORTED, "t-side sweep: no kernel for T = %d", Tax[0]);
          FPCA_LAUNCHED(ctx, "cov_tsweep");
        } else {
          run_hs(ef);
          FPCA_LAUNCHED(ctx, "cov_hpass_solve");
        }
        if (ef.esc_count) {
          k_escalated<<<ctx->num_sms * 8, 256, 0, ctx->stream>>>(
              P, ef.esc_slots, ef.esc_idx, ef.esc_count, ef.esc_cap, mu_raw, gm, status, ef,
              tg.half);
          FPCA_LAUNCHED(ctx, "cov_escalated");
        }
        if (tg.half && (gm || status)) {
          const int nt = (P + MIR_T - 1) / MIR_T;
          k_mirror_lower<<<nt * (nt + 1) / 2, 256, 0, ctx->stream>>>(P, gm, status);
          FPCA_LAUNCHED(ctx, "cov_mirror");
        }
        return FPCA_OK;
      }
    }
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
  if (!launch_vpass<T, COMP>(ctx, j1, 3, P, M1, 1, 1, Tax[0], tabk(0)))
    return fpca_check_launch(ctx, "cov_vpass_s1");
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

// Shared memory of the batched CV-grid sweep: sized for the widest window of the grid.
size_t cv_grid_smem(const fpca_grid* g, const double* h, int nh) {
  const int P = grid_P(g), M1 = g->m[0], M2 = g->m[1];
  int ntr = 0, ntc = 0, nrp = 0, rs = 0;
  for (int ih = 0; ih < nh; ++ih) {
    const Hs2Geom hg = hs2_geometry(P, M1, M2, host_taps(h[2 * ih], M1), host_taps(h[2 * ih + 1], M2));
    ntr = std::max(ntr, hg.ntr);
    ntc = std::max(ntc, hg.ntc);
    nrp = std::max(nrp, hg.nrp);
    rs = std::max(rs, hg.RS);
  }
  const int SC = M2 | 1;
  const size_t in_f = (size_t)10 * nrp * M2, slot_f = (size_t)NSL * HT * SC;
  return sizeof(float) * ((size_t)TROWS * (ntr + ntc) + (size_t)NMID * HT * rs +
                          (in_f > slot_f ? in_f : slot_f));
}

// The t-sides of all (bandwidth, fold) items of a CV grid in one persistent launch
// (k_hsolve2_grid), from the items' s-side arrays, then the escalated fits.
template <bool COMP>
fpca_status cv_grid_batched(fpca_ctx* ctx, const fpca_grid* g, const fpca_covbins* bins,
                            const double* h, int nh, int F, const double* tab_all,
                            const float* varr_all, double* cvacc, CvGridItem* items_d,
                            int* esc_item, unsigned* counter, float* esc_slots, int2* esc_idx,
                            unsigned* esc_count, int esc_cap) {
  const int P = grid_P(g), M1 = g->m[0], M2 = g->m[1];
  const long long PP = (long long)P * P;
  const int nitems = nh * F;
  const float* fw = static_cast<const float*>(bins->w);
  const float* fv = static_cast<const float*>(bins->v);
  const float* fq = static_cast<const float*>(bins->q);
  std::vector<CvGridItem> items(nitems);
  int ntr = 0, ntc = 0, rs = 0;
  for (int ih = 0; ih < nh; ++ih) {
    for (int f = 0; f < F; ++f) {
      CvGridItem& it = items[ih * F + f];
      it.varr = varr_all + (size_t)(ih * F + f) * 10 * PP;
      it.tab = tab_all + (size_t)ih * 3 * TROWS * TW;
      it.g = hs2_geometry(P, M1, M2, host_taps(h[2 * ih], M1), host_taps(h[2 * ih + 1], M2));
      it.g.half = 1;
      it.ep = Epilogue<float>{};
      it.ep.wf = fw + (size_t)f * PP;
      it.ep.vf = fv + (size_t)f * PP;
      it.ep.qf = fq + (size_t)f * PP;
      it.ep.cvacc = cvacc + 3 * ((size_t)ih * F + f);
      it.ep.esc_slots = esc_slots;
      it.ep.esc_idx = esc_idx;
      it.ep.esc_count = esc_count;
      it.ep.esc_cap = esc_cap;
      it.item = ih * F + f;
      ntr = std::max(ntr, it.g.ntr);
      ntc = std::max(ntc, it.g.ntc);
      rs = std::max(rs, it.g.RS);
    }
  }
  const size_t smem = cv_grid_smem(g, h, nh);
  // pageable source: the copy is staged before the call returns (so not capturable)
  if (fpca_no_capture(ctx, "the batched CV grid") != FPCA_OK) return FPCA_E_UNSUPPORTED;
  if (cudaMemcpyAsync(items_d, items.data(), sizeof(CvGridItem) * nitems, cudaMemcpyHostToDevice,
                      ctx->stream) != cudaSuccess)
    return fpca_check_launch(ctx, "cv grid items");
  cudaMemsetAsync(counter, 0, sizeof(unsigned), ctx->stream);
  cudaMemsetAsync(esc_count, 0, sizeof(unsigned), ctx->stream);
  const int nblk = ((M1 + HT - 1) / HT) * P;
  const int per_sm = smem * 2 <= ctx->smem_optin ? 2 : 1;
  const dim3 grid(ctx->num_sms * per_sm);
  auto launch = [&](auto kern) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    kern<<<grid, NT2, smem, ctx->stream>>>(items_d, nitems, nblk, counter, ntr, ntc, rs, esc_item,
                                           ctx->d_err);
  };
  switch (M2) {
    case 8: launch(k_hsolve2_grid<COMP, 8>); break;
    case 16: launch(k_hsolve2_grid<COMP, 16>); break;
    case 32: launch(k_hsolve2_grid<COMP, 32>); break;
    default: launch(k_hsolve2_grid<COMP, 64>); break;
  }
  FPCA_LAUNCHED(ctx, "cov_cv_grid");
  k_escalated<<<ctx->num_sms * 8, 256, 0, ctx->stream>>>(P, esc_slots, esc_idx, esc_count, esc_cap,
                                                          nullptr, nullptr, nullptr,
                                                          Epilogue<float>{}, 1, items_d, esc_item);
  FPCA_LAUNCHED(ctx, "cov_escalated");
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
  // queue of escalated FP32 fits (d = 2 FP32 kernel): up to 2^21 points
  const int esc_cap = (sizeof(T) == 4 && d == 2) ? (int)std::min<long long>(PP, 1ll << 21) : 0;
  const size_t need = WsCarve::round(sizeof(double) * 3 * TROWS * TW * (size_t)nh) +
                      WsCarve::round(sizeof(T) * PP * (size_t)(nmid + narr(d))) +
                      (F > 1 ? WsCarve::round(sizeof(T) * PP) * 2 + WsCarve::round(4 * PP) : 0) +
                      WsCarve::round(sizeof(double) * 3 * (size_t)nh * F) +
                      WsCarve::round(sizeof(float) * 21 * (size_t)esc_cap) +
                      WsCarve::round(sizeof(int2) * (size_t)esc_cap) + 8192;
  // The CV grid batched: every (bandwidth, fold) item keeps its s-side arrays and
  // one persistent launch runs all their t-sides (FP32, d = 2, symmetric bins,
  // the scalar sweep's shapes, and the items' arrays fit in free device memory).
  const int nitems = nh * F;
  bool batched = false;
  size_t need_b = 0;
  if constexpr (sizeof(T) == 4) {
    const int M2 = d == 2 ? g->m[1] : 0;
    if (cv && ctx->cv_batch != 0 && d == 2 && F >= 2 && bins->asym == 0 && !mu_raw &&
        ctx->tside_kernel != 2 && (M2 == 8 || M2 == 16 || M2 == 32 || M2 == 64)) {
      batched = cv_grid_smem(g, h, nh) <= ctx->smem_optin;
      need_b = WsCarve::round(sizeof(float) * 10 * (size_t)PP * nitems) +
               WsCarve::round(sizeof(CvGridItem) * (size_t)nitems) +
               WsCarve::round(sizeof(int) * (size_t)esc_cap) + 1024;
      size_t fr = 0, tot = 0;
      if (batched && need + need_b > ctx->ws_bytes) {
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
          cudaGetLastError();
          fr = 0;
        }
        // leave room: grow only into at most 80% of what is free
        batched = need + need_b <= ctx->ws_bytes + (size_t)(0.8 * (double)fr);
      }
    }
  }
  void* ws = fpca_workspace(ctx, need + (batched ? need_b : 0));
  if (!ws && batched) {
    batched = false;
    ws = fpca_workspace(ctx, need);
  }
  if (!ws) return fpca_fail(ctx, FPCA_E_OOM, "workspace (%zu bytes)", need);
  WsCarve carve(ws);
  // tap tables of every bandwidth (TROWS x TW per axis, 3 axes)
  double* tab_all = carve.take<double>(3 * TROWS * TW * (size_t)nh);
  T* mids = carve.take<T>((size_t)PP * nmid);
  T* varr = carve.take<T>((size_t)PP * narr(d));
  double* cvacc = carve.take<double>((size_t)3 * nh * F);
  float* esc_slots = carve.take<float>((size_t)21 * esc_cap);
  int2* esc_idx = carve.take<int2>((size_t)esc_cap);
  unsigned* esc_count = carve.take<unsigned>(1);
  float* varr_all = nullptr;
  CvGridItem* items_d = nullptr;
  int* esc_item = nullptr;
  unsigned* counter = nullptr;
  if (batched) {
    varr_all = carve.take<float>(10 * (size_t)PP * nitems);
    items_d = carve.take<CvGridItem>(nitems);
    esc_item = carve.take<int>(esc_cap);
    counter = carve.take<unsigned>(4);
  }
  auto with_queue = [&](Epilogue<T>& ep) {
    if (esc_cap > 0) {
      ep.esc_slots = reinterpret_cast<float*>(esc_slots);
      ep.esc_idx = esc_idx;
      ep.esc_count = esc_count;
      ep.esc_cap = esc_cap;
    }
  };
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
  for (int ih = 0; ih < nh; ++ih) {
    const double* hh = h + (size_t)ih * d;
    TapParams tp{};
    tp.d = d;
    for (int k = 0; k < 3; ++k) {
      tp.m[k] = k < d ? g->m[k] : 1;
      tp.h[k] = k < d ? hh[k] : 1.0;
    }
    double* tabh = tab_all + (size_t)ih * 3 * TROWS * TW;
    k_taps<<<d, 128, 0, ctx->stream>>>(tp, tabh);
    FPCA_LAUNCHED(ctx, "taps");
    // the fit on all bins: Gamma_hat, status, projection
    if (gamma || status || y) {
      Epilogue<T> ep{};
      with_queue(ep);
      if (y) {
        ep.omega = omega;
        ep.l = l;
        ep.y = y + (size_t)ih * P * l;
      }
      fpca_status s = cov_smooth_one<T, COMP>(
          ctx, g, cnt, w, v, nullptr, nullptr, nullptr, hh, tabh, mids, varr, mu_raw,
          gamma ? gamma + (size_t)ih * PP : nullptr, status ? status + (size_t)ih * PP : nullptr,
          ep, bins->asym == 0);
      if (s != FPCA_OK) return s;
    }
  }
  // K-fold CV: for each (bandwidth, fold) item, fit on the other folds and score
  // the held-out fold; item by item, or batched (all s-sides, then one t-side launch)
  auto run_items = [&]() -> fpca_status {
    cudaMemsetAsync(cvacc, 0, sizeof(double) * 3 * (size_t)nh * F, ctx->stream);
    const T* fw = static_cast<const T*>(bins->w);
    const T* fv = static_cast<const T*>(bins->v);
    const T* fq = static_cast<const T*>(bins->q);
    for (int ih = 0; ih < nh; ++ih) {
      for (int f = 0; f < F; ++f) {
        Epilogue<T> ep{};
        with_queue(ep);
        ep.wf = fw + (size_t)f * PP;
        ep.vf = fv + (size_t)f * PP;
        ep.qf = fq + (size_t)f * PP;
        ep.cvacc = cvacc + 3 * ((size_t)ih * F + f);
        fpca_status s = cov_smooth_one<T, COMP>(
            ctx, g, cnt, w, v, bins->cnt + (size_t)f * PP, fw + (size_t)f * PP,
            fv + (size_t)f * PP, h + (size_t)ih * d, tab_all + (size_t)ih * 3 * TROWS * TW, mids,
            varr, mu_raw, nullptr, nullptr, ep, bins->asym == 0);
        if (s != FPCA_OK) return s;
      }
    }
    return FPCA_OK;
  };
  auto run_batched = [&]() -> fpca_status {
    if constexpr (sizeof(T) == 4) {
      cudaMemsetAsync(cvacc, 0, sizeof(double) * 3 * (size_t)nh * F, ctx->stream);
      const T* fw = static_cast<const T*>(bins->w);
      const T* fv = static_cast<const T*>(bins->v);
      for (int ih = 0; ih < nh; ++ih) {
        for (int f = 0; f < F; ++f) {
          T* vi = reinterpret_cast<T*>(varr_all) + (size_t)(ih * F + f) * 10 * PP;
          fpca_status s = cov_smooth_one<T, COMP>(
              ctx, g, cnt, w, v, bins->cnt + (size_t)f * PP, fw + (size_t)f * PP,
              fv + (size_t)f * PP, h + (size_t)ih * d, tab_all + (size_t)ih * 3 * TROWS * TW,
              mids, vi, nullptr, nullptr, nullptr, Epilogue<T>{}, true, true);
          if (s != FPCA_OK) return s;
        }
      }
      return cv_grid_batched<COMP>(ctx, g, bins, h, nh, F, tab_all, varr_all, cvacc, items_d,
                                   esc_item, counter, esc_slots, esc_idx, esc_count, esc_cap);
    }
    return FPCA_OK;
  };
  if (cv) {
    fpca_status st = FPCA_OK;
    if (!batched) {
      st = run_items();
    } else if (ctx->cv_batch == 1) {
      st = run_batched();
    } else {
      // automatic: time both schedules once per (grid, folds, precision, number of
      // bandwidths, whether the widest window leaves room for two batched CTAs per
      // SM) -- after one untimed item-by-item pass, so the sweep choices those items
      // make are already settled -- and remember the faster in the context.  The
      // key leaves the windows themselves out: the checks of nearby bandwidths on
      // many datasets share one decision instead of each paying for the timing.
      const int wide = 2 * cv_grid_smem(g, h, nh) > ctx->smem_optin ? 1 : 0;
      const std::vector<int> key = {g->m[0], g->m[1], F, COMP ? 1 : 0, nh, wide};
      auto it = ctx->cv_choice.find(key);
      if (it == ctx->cv_choice.end()) {
        if (fpca_no_capture(ctx, "timing the CV schedules") != FPCA_OK) return FPCA_E_UNSUPPORTED;
        st = run_items();
        cudaEvent_t ev[3];
        for (auto& x : ev) cudaEventCreate(&x);
        cudaEventRecord(ev[0], ctx->stream);
        if (st == FPCA_OK) st = run_batched();
        cudaEventRecord(ev[1], ctx->stream);
        if (st == FPCA_OK) st = run_items();
        cudaEventRecord(ev[2], ctx->stream);
        if (st == FPCA_OK && cudaEventSynchronize(ev[2]) != cudaSuccess)
          st = fpca_check_launch(ctx, "CV schedule autotune");
        float tb = 0.f, ti = 0.f;
        cudaEventElapsedTime(&tb, ev[0], ev[1]);
        cudaEventElapsedTime(&ti, ev[1], ev[2]);
        for (auto& x : ev) cudaEventDestroy(x);
        if (st != FPCA_OK) return st;
        ctx->cv_choice.emplace(key, tb < ti ? 1 : 0);
      } else {
        st = it->second == 1 ? run_batched() : run_items();
      }
    }
    if (st != FPCA_OK) return st;
  }
  if (cv) {
    k_cv_finish<<<(nh + 63) / 64, 64, 0, ctx->stream>>>(nh, F, cvacc, cv);
    FPCA_LAUNCHED(ctx, "cv_finish");
  }
  return FPCA_OK;
}

}  // namespace

size_t smooth_mean_scratch_bytes(int P) {
  const size_t tb = (sizeof(double) * 3 * TROWS * TW + 255) & ~size_t(255);
  const size_t stack = (sizeof(double) * (size_t)MJ_MAX * P + 255) & ~size_t(255);
  return tb + 2 * stack;
}

fpca_status launch_smooth_mean(fpca_ctx* ctx, const fpca_grid* g, const int32_t* cnt,
                               const double* w, const double* v, const double* h, double* mu,
                               uint8_t* status, void* scratch) {
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
  const int T0 = host_taps(tp.h[0], tp.m[0]);
  const int T1 = g->d > 1 ? host_taps(tp.h[1], tp.m[1]) : 0;
  const int T2 = g->d > 2 ? host_taps(tp.h[2], tp.m[2]) : 0;
  const int taps[3] = {T0, T1, T2};
  // pass plan: arrays carry (kind, exponents of the processed axes); kind 0 = W
  // (total degree <= 2), 1 = V (<= 1), 2 = the non-empty indicator (box sums)
  struct Arr {
    int kind, deg, e[3];
  };
  std::vector<Arr> cur = {{0, 0, {0, 0, 0}}, {1, 0, {0, 0, 0}}, {2, 0, {0, 0, 0}}};
  std::vector<MeanPass> passes;
  for (int ax = g->d - 1; ax >= 0; --ax) {
    MeanPass mp{};
    mp.axis = ax;
    int st = 1;
    for (int k = ax + 1; k < g->d; ++k) st *= g->m[k];
    mp.stride = st;
    mp.T = taps[ax];
    std::vector<Arr> next;
    for (int i = 0; i < (int)cur.size(); ++i) {
      const Arr& a = cur[i];
      if (a.kind == 2) {
        mp.src[mp.njobs] = i;
        mp.row[mp.njobs++] = 3;
        next.push_back(a);
        continue;
      }
      const int maxd = (a.kind == 0 ? 2 : 1) - a.deg;
      for (int e = 0; e <= maxd; ++e) {
        mp.src[mp.njobs] = i;
        mp.row[mp.njobs++] = e;
        Arr b = a;
        b.deg += e;
        b.e[ax] = e;
        next.push_back(b);
      }
    }
    passes.push_back(mp);
    cur = next;
  }
  // final array index of each normal-matrix entry
  const int D = g->d + 1;
  auto find = [&](int kind, const int e[3]) {
    for (int i = 0; i < (int)cur.size(); ++i)
      if (cur[i].kind == kind && cur[i].e[0] == e[0] && cur[i].e[1] == e[1] && cur[i].e[2] == e[2])
        return i;
    return -1;
  };
  MeanIdx ix{};
  for (int i = 0; i < D; ++i) {
    for (int j = 0; j < D; ++j) {
      int e[3] = {0, 0, 0};
      if (i > 0) e[i - 1] += 1;
      if (j > 0) e[j - 1] += 1;
      ix.a[i * D + j] = find(0, e);
    }
    int e[3] = {0, 0, 0};
    if (i > 0) e[i - 1] = 1;
    ix.r[i] = find(1, e);
  }
  {
    const int e[3] = {0, 0, 0};
    ix.n = find(2, e);
  }
  // workspace (or the caller's scratch): taps table and two ping-pong stacks of
  // MJ_MAX arrays
  const size_t tb = (sizeof(double) * 3 * TROWS * TW + 255) & ~size_t(255);
  const size_t stack = (sizeof(double) * (size_t)MJ_MAX * P + 255) & ~size_t(255);
  char* base = scratch ? static_cast<char*>(scratch)
                       : static_cast<char*>(fpca_workspace(ctx, tb + 2 * stack));
  if (!base) return fpca_fail(ctx, FPCA_E_OOM, "workspace");
  double* tabw = reinterpret_cast<double*>(base);
  double* bufA = reinterpret_cast<double*>(base + tb);
  double* bufB = reinterpret_cast<double*>(base + tb + stack);
  k_taps<<<g->d, 128, 0, ctx->stream>>>(tp, tabw);
  FPCA_LAUNCHED(ctx, "taps");
  const int nb = (P + 255) / 256;
  k_mean_prep<<<nb, 256, 0, ctx->stream>>>(P, cnt, w, v, bufA);
  FPCA_LAUNCHED(ctx, "mean_prep");
  double* in = bufA;
  double* out = bufB;
  for (const MeanPass& mp : passes) {
    k_mean_pass<<<(int)(((long long)P * mp.njobs + 255) / 256), 256, 0, ctx->stream>>>(
        P, g->m[mp.axis], mp, tabw, in, out);
    FPCA_LAUNCHED(ctx, "mean_pass");
    std::swap(in, out);
  }
  if (g->d == 1)
    k_mean_solve<1><<<nb, 256, 0, ctx->stream>>>(P, in, ix, mu, status);
  else if (g->d == 2)
    k_mean_solve<2><<<nb, 256, 0, ctx->stream>>>(P, in, ix, mu, status);
  else
    k_mean_solve<3><<<nb, 256, 0, ctx->stream>>>(P, in, ix, mu, status);
  FPCA_LAUNCHED(ctx, "smooth_mean");
  return FPCA_OK;
}

fpca_status launch_sigma2(fpca_ctx* ctx, const fpca_grid* g, const int32_t* cnt, const double* w,
                          const double* v2, const double* h, const double* mu, const void* gdiag,
                          int gprec, long long gstride, const int32_t* domain, double* sig_t,
                          uint8_t* status, double* sigma2) {
  // b0 of Eq. (2.5): the mean smoother on the bins of Y^2, written into sig_t
  fpca_status s = launch_smooth_mean(ctx, g, cnt, w, v2, h, sig_t, status);
  if (s != FPCA_OK) return s;
  const int P = grid_P(g);
  const int nb = (P + 255) / 256;
  if (gprec == FPCA_F64)
    k_sigma2_curve<double><<<nb, 256, 0, ctx->stream>>>(P, mu, static_cast<const double*>(gdiag),
                                                       gstride, status, sig_t);
  else
    k_sigma2_curve<float><<<nb, 256, 0, ctx->stream>>>(P, mu, static_cast<const float*>(gdiag),
                                                      gstride, status, sig_t);
  FPCA_LAUNCHED(ctx, "sigma2_curve");
  if (sigma2) {
    k_sigma2_mean<<<1, 1024, 0, ctx->stream>>>(P, sig_t, domain, sigma2);
    FPCA_LAUNCHED(ctx, "sigma2_mean");
  }
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

// ---------------------------------------------------------------------------
// cross-validation of the mean smoother (Eq. 2.3), scattered data
// ---------------------------------------------------------------------------
// Subject-level K-fold: for fold f the mean is fitted (the smoother above) on
// the mean bins of the other folds and scored on fold f's observations at their
// bin centres, weights 1/N_i: sum over bins of V2_f - 2 mu V_f + mu^2 W_f where
// the fit is not EMPTY, normalised by the held-out weight scored; +inf when
// EMPTY bins hold more than 1% of the held-out weight.
namespace {

__device__ __forceinline__ int mcv_bin(const double* t, int d, const int* m) {
  int flat = 0;
  for (int k = 0; k < d; ++k) {
    const double x = floor(__dmul_rn(t[k], (double)m[k]));
    const int ik = (int)fmin(fmax(x, 0.0), (double)(m[k] - 1));
    flat = flat * m[k] + ik;
  }
  return flat;
}

// Mean bins of every fold: subject i adds to slice fold[i] (cnt, w, v, v2 are F x P).
__global__ void k_bin_mean_folds(int n, long long N, int d, int m0, int m1, int m2, int P,
                                 const int64_t* __restrict__ offs, const double* __restrict__ t,
                                 const double* __restrict__ y, const int32_t* __restrict__ fold,
                                 int nfold, int32_t* cnt, double* w, double* v, double* v2,
                                 int* __restrict__ err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int m[3] = {m0, m1, m2};
  const int64_t lo = offs[i], hi = offs[i + 1];
  const int f = fold[i];
  if (lo < 0 || hi < lo || hi > N || f < 0 || f >= nfold) {
    atomicExch(err, DERR_BOUNDS);
    return;
  }
  if (hi == lo) return;
  const double wi = 1.0 / (double)(hi - lo);
  const size_t base = (size_t)f * P;
  for (int64_t j = lo; j < hi; ++j) {
    const size_t b = base + mcv_bin(t + j * d, d, m);
    const double yy = y[j];
    atomicAdd(cnt + b, 1);
    atomicAdd(w + b, wi);
    atomicAdd(v + b, __dmul_rn(wi, yy));
    atomicAdd(v2 + b, __dmul_rn(wi, __dmul_rn(yy, yy)));
  }
}

// Training bins of fold f: the sums over all folds minus fold f's.
__global__ void k_mean_train(int P, int F, int f, const int32_t* __restrict__ cnt,
                             const double* __restrict__ w, const double* __restrict__ v,
                             int32_t* __restrict__ ct, double* __restrict__ wt,
                             double* __restrict__ vt) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  int c = 0;
  double sw = 0.0, sv = 0.0;
  for (int q = 0; q < F; ++q) {  // pooled sums in fold order (the same order every fold)
    c += cnt[(size_t)q * P + p];
    sw += w[(size_t)q * P + p];
    sv += v[(size_t)q * P + p];
  }
  ct[p] = c - cnt[(size_t)f * P + p];
  wt[p] = sw - w[(size_t)f * P + p];
  vt[p] = sv - v[(size_t)f * P + p];
}

// Held-out terms of fold f against the fit mu (status st): acc[0] += error,
// acc[1] += scored weight, acc[2] += weight on EMPTY fits.
__global__ void k_mean_cv_terms(int P, const double* __restrict__ mu, const uint8_t* __restrict__ st,
                                const double* __restrict__ wf, const double* __restrict__ vf,
                                const double* __restrict__ v2f, double* __restrict__ acc) {
  __shared__ double red[256 / 32];
  double e = 0.0, win = 0.0, wout = 0.0;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < P; p += gridDim.x * blockDim.x) {
    if (st[p] == FPCA_PT_EMPTY) {
      wout += wf[p];
    } else {
      const double g = mu[p];
      e += v2f[p] - 2.0 * g * vf[p] + g * g * wf[p];
      win += wf[p];
    }
  }
  const double s0 = block_sum<256>(e, red);
  const double s1 = block_sum<256>(win, red);
  const double s2 = block_sum<256>(wout, red);
  if (threadIdx.x == 0) {
    atomicAdd(acc + 0, s0);
    atomicAdd(acc + 1, s1);
    atomicAdd(acc + 2, s2);
  }
}

}  // namespace

fpca_status mean_cv_run(fpca_ctx* ctx, const fpca_grid* g, int n, const int64_t* offs,
                        const double* t, const double* y, const int32_t* fold, int nfold,
                        const double* h, int nh, double* cv) {
  const int P = grid_P(g), F = nfold, d = g->d;
  for (int k = 0; k < d; ++k)
    if (g->m[k] > TMAX + 1)
      return fpca_fail(ctx, FPCA_E_UNSUPPORTED, "mean smoothing is built for m <= %d", TMAX + 1);
  long long Nobs = 0;
  if (fpca_no_capture(ctx, "reading offs[n] of scattered data") != FPCA_OK) return FPCA_E_UNSUPPORTED;
  if (cudaMemcpyAsync(&Nobs, offs + n, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(ctx->stream) != cudaSuccess)
    return fpca_check_launch(ctx, "mean_cv: offsets");
  const size_t need = WsCarve::round(smooth_mean_scratch_bytes(P)) +
                      WsCarve::round(sizeof(int32_t) * (size_t)F * P) +
                      3 * WsCarve::round(sizeof(double) * (size_t)F * P) +
                      WsCarve::round(sizeof(int32_t) * P) + 3 * WsCarve::round(sizeof(double) * P) +
                      WsCarve::round(P) + WsCarve::round(sizeof(double) * 3 * (size_t)nh * F) + 4096;
  void* ws = fpca_workspace(ctx, need);
  if (!ws) return fpca_fail(ctx, FPCA_E_OOM, "workspace (%zu bytes)", need);
  WsCarve c(ws);
  char* scratch = c.take<char>(smooth_mean_scratch_bytes(P));
  int32_t* fc = c.take<int32_t>((size_t)F * P);
  double* fw = c.take<double>((size_t)F * P);
  double* fv = c.take<double>((size_t)F * P);
  double* fv2 = c.take<double>((size_t)F * P);
  int32_t* ct = c.take<int32_t>(P);
  double* wt = c.take<double>(P);
  double* vt = c.take<double>(P);
  double* mu = c.take<double>(P);
  uint8_t* st = c.take<uint8_t>(P);
  double* acc = c.take<double>((size_t)3 * nh * F);
  cudaMemsetAsync(fc, 0, sizeof(int32_t) * (size_t)F * P, ctx->stream);
  cudaMemsetAsync(fw, 0, sizeof(double) * (size_t)F * P, ctx->stream);
  cudaMemsetAsync(fv, 0, sizeof(double) * (size_t)F * P, ctx->stream);
  cudaMemsetAsync(fv2, 0, sizeof(double) * (size_t)F * P, ctx->stream);
  cudaMemsetAsync(acc, 0, sizeof(double) * 3 * (size_t)nh * F, ctx->stream);
  k_bin_mean_folds<<<(n + 127) / 128, 128, 0, ctx->stream>>>(
      n, Nobs, d, g->m[0], d > 1 ? g->m[1] : 1, d > 2 ? g->m[2] : 1, P, offs, t, y, fold, F, fc,
      fw, fv, fv2, ctx->d_err);
  FPCA_LAUNCHED(ctx, "bin_mean_folds");
  const int nb = (P + 255) / 256;
  for (int f = 0; f < F; ++f) {
    k_mean_train<<<nb, 256, 0, ctx->stream>>>(P, F, f, fc, fw, fv, ct, wt, vt);
    FPCA_LAUNCHED(ctx, "mean_train");
    for (int ih = 0; ih < nh; ++ih) {
      fpca_status s = launch_smooth_mean(ctx, g, ct, wt, vt, h + (size_t)ih * d, mu, st, scratch);
      if (s != FPCA_OK) return s;
      k_mean_cv_terms<<<std::min(nb, 64), 256, 0, ctx->stream>>>(
          P, mu, st, fw + (size_t)f * P, fv + (size_t)f * P, fv2 + (size_t)f * P,
          acc + 3 * ((size_t)ih * F + f));
      FPCA_LAUNCHED(ctx, "mean_cv_terms");
    }
  }
  k_cv_finish<<<(nh + 63) / 64, 64, 0, ctx->stream>>>(nh, F, acc, cv);
  FPCA_LAUNCHED(ctx, "cv_finish");
  return FPCA_OK;
}
