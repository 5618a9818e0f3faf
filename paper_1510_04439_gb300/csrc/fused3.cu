// d = 3 covariance smoothing of fully observed gridded data, fused into its
// product with a block of vectors, Y = Gamma_hat X (Eq. 2.4 with the
// Section 3.2 binning; Section 3.4 projection).  Neither the P x P bins nor
// the P x P surface is formed.
//
// Factorisation.  With every node observed in every subject the covariance
// bins are W[p,q] = c for p != q and V = R~'R~ with its diagonal zeroed
// (R~ = R / sqrt(n); the constant subject weights cancel, c = 1).  At an
// output pair (s,t) whose kernel windows share no node, no zeroed diagonal
// bin enters the sums, the weights K_s(p) K_t(q) form a product measure, and
// the local linear fit on z = [1, u_s, u_t] splits into one-sided fits:
//     Gamma_hat(s,t) = [L V E' + E V L' - E V E'](s,t),     V = R~'R~,
// with E and L the 3-dimensional local constant and local linear smoothing
// matrices (their equivalent kernels are products of 1-D kernels).  Hence
//     Gamma_prod X = L V (E'X) + E V ((L - E)'X)
// costs two skinny products with R~ and separable convolutions of X.
// Where every |s_k - t_k| <= 2 T_k (T_k the taps of axis k) the windows share
// nodes and the exact fit differs from the product-form one by
//     corr = e0' (A_p - A_d)^{-1} (A_d beta_prod - r_d),
// A_p / A_d the normal matrices of all bin pairs / of the diagonal pairs only,
// r_d the diagonal pairs' part of the right-hand side.  beta_prod follows in
// closed form from seven kernel-weighted products P_ab(s,t) =
// sum_i B_a(i,s) B_b(i,t), B_a = R~ conv (K u_a), computed on tcgen05 tensor
// cores tile pair by tile pair; corr is multiplied into Y on the tensor cores
// too.  Far pairs need no correction, so their smoothing is exactly the
// product form already applied.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "ptx.cuh"

namespace {

constexpr int F3_TMAX = 8;                 // largest taps per axis
constexpr int F3_MMAX = 64;                // largest nodes per axis
constexpr int F3_NTAP = 2 * F3_TMAX + 1;
constexpr int F3_NOFF = 4 * F3_TMAX + 1;   // pair offsets -2T .. 2T
constexpr int SB = 128, TB = 64, BK = 64;  // S-tile rows, T-tile columns, K chunk
constexpr int CORR_BYTES = SB * TB * 2;    // BF16 corrections of one tile pair
constexpr int XT_BYTES = 64 * 128;         // up to 64 vectors x 64 nodes, BF16
constexpr int NEAR_THREADS = 320;          // warp 0 TMA, warp 1 MMA, warps 2..9 epilogue
constexpr int F3_CHUNKS = 8;               // CTAs sharing one S-tile's T-list

struct Geo3 {
  int m[3];
  int T[3];
  int nb[3];        // S-tiles per axis: ceil(m0/4), ceil(m1/4), ceil(m2/8)
  int P, p_pad, n, n_pad;
};

// Per-axis tables in FP32 (computed in FP64 on the device).
struct Tab3 {
  float tapK[3][F3_NTAP];     // K(r / hM), r = -T..T (index r + F3_TMAX)
  float tapKu[3][F3_NTAP];    // K(r / hM) r / hM
  float k0[3][F3_MMAX];       // sum_p K(u), u = (p - x)/hM over the window of node x
  float mu1[3][F3_MMAX];      // sum K u / k0
  float var[3][F3_MMAX];      // sum K u^2 / k0 - mu1^2
  float inv_hM[3];
  // diagonal-pair moments between nodes x and y = x + dx (|dx| <= 2T):
  // sum_p K(u_x)K(u_y) u_x^a u_y^b / (k0(x) k0(y)), (a,b) = 00,10,01,20,11,02
  float rho[3][F3_MMAX][F3_NOFF][6];
};

__host__ __device__ inline int f3_perm(const Geo3& g, int a0, int a1, int a2) {
  const int S = ((a0 >> 2) * g.nb[1] + (a1 >> 2)) * g.nb[2] + (a2 >> 3);
  return S * SB + ((a2 & 7) >> 2) * 64 + (a0 & 3) * 16 + (a1 & 3) * 4 + (a2 & 3);
}

__global__ void k_f3_tables(Geo3 g, double h0, double h1, double h2, Tab3* tab) {
  const int k = blockIdx.x;
  const double hM = (k == 0 ? h0 : k == 1 ? h1 : h2) * g.m[k];
  const int M = g.m[k], T = g.T[k];
  auto K = [](double u) { return 0.75 * (1.0 - u * u); };
  if (threadIdx.x == 0) tab->inv_hM[k] = (float)(1.0 / hM);
  for (int i = threadIdx.x; i < F3_NTAP; i += blockDim.x) {
    const int r = i - F3_TMAX;
    const double u = r / hM;
    const bool in = r >= -T && r <= T;
    tab->tapK[k][i] = in ? (float)K(u) : 0.f;
    tab->tapKu[k][i] = in ? (float)(K(u) * u) : 0.f;
  }
  __shared__ double kap0[F3_MMAX];
  for (int x = threadIdx.x; x < F3_MMAX; x += blockDim.x) {
    double s0 = 0, s1 = 0, s2 = 0;
    if (x < M) {
      for (int p = max(0, x - T); p <= min(M - 1, x + T); ++p) {
        const double u = (p - x) / hM, w = K(u);
        s0 += w;
        s1 += w * u;
        s2 += w * u * u;
      }
    }
    kap0[x] = s0;
    const double m1 = s0 > 0 ? s1 / s0 : 0.0;
    tab->k0[k][x] = (float)s0;
    tab->mu1[k][x] = (float)m1;
    tab->var[k][x] = s0 > 0 ? (float)(s2 / s0 - m1 * m1) : 0.f;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < F3_MMAX * F3_NOFF; e += blockDim.x) {
    const int x = e / F3_NOFF, dx = e % F3_NOFF - 2 * F3_TMAX;
    const int y = x + dx;
    double d[6] = {0, 0, 0, 0, 0, 0};
    if (x < M && y >= 0 && y < M && dx >= -2 * T && dx <= 2 * T) {
      for (int p = max(max(x, y) - T, 0); p <= min(min(x, y) + T, M - 1); ++p) {
        const double ux = (p - x) / hM, uy = (p - y) / hM, w = K(ux) * K(uy);
        d[0] += w;
        d[1] += w * ux;
        d[2] += w * uy;
        d[3] += w * ux * ux;
        d[4] += w * ux * uy;
        d[5] += w * uy * uy;
      }
      const double nrm = 1.0 / (kap0[x] * kap0[y]);
      for (int j = 0; j < 6; ++j) d[j] *= nrm;
    }
    for (int j = 0; j < 6; ++j) tab->rho[k][x][e % F3_NOFF][j] = (float)d[j];
  }
}

// ---------------------------------------------------------------------------
// residual factor: Rt32 (P x n_pad, FP32, natural node order), Rbt
// (p_pad x n_pad, BF16, tile order), Rb (n_pad x p_pad, BF16, tile order)
// ---------------------------------------------------------------------------
template <typename TY>
__global__ void k_f3_residuals(Geo3 g, const TY* __restrict__ y, const double* __restrict__ mu,
                               float scale, float* __restrict__ Rt32, __nv_bfloat16* __restrict__ Rbt,
                               __nv_bfloat16* __restrict__ Rb) {
  __shared__ float tile[32][33];
  __shared__ float muf[32];
  __shared__ int qs[32];
  const int p0 = blockIdx.x * 32, i0 = blockIdx.y * 32;
  // the mean and the tile-order index of the block's 32 nodes, once per block
  if (threadIdx.y == 0) {
    const int p = p0 + threadIdx.x;
    muf[threadIdx.x] = p < g.P ? (float)mu[p] : 0.f;
    int q = -1;
    if (p < g.P) {
      const int a2 = p % g.m[2], a1 = (p / g.m[2]) % g.m[1], a0 = p / (g.m[2] * g.m[1]);
      q = (int)f3_perm(g, a0, a1, a2);
    }
    qs[threadIdx.x] = q;
  }
  __syncthreads();
  // residuals in FP32 (the factor is FP32 and BF16; FP64 is slow on this GPU)
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int i = i0 + r, p = p0 + threadIdx.x;
    float v = 0.f;
    if (i < g.n && p < g.P) v = ((float)y[(size_t)i * g.P + p] - muf[threadIdx.x]) * scale;
    tile[r][threadIdx.x] = v;
    // R~ (n_pad x p_pad, tile order): consecutive nodes are runs of consecutive q
    if (i < g.n_pad && p < g.P) Rb[(size_t)i * g.p_pad + qs[threadIdx.x]] = __float2bfloat16_rn(v);
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int p = p0 + r, i = i0 + threadIdx.x;
    if (p >= g.P || i >= g.n_pad) continue;
    const float v = tile[threadIdx.x][r];
    Rt32[(size_t)p * g.n_pad + i] = v;
    Rbt[(size_t)qs[r] * g.n_pad + i] = __float2bfloat16_rn(v);
  }
}

// D'_p = sum_i R~_ip^2 (one warp per node)
__global__ void k_f3_diag(Geo3 g, const float* __restrict__ Rt32, float* __restrict__ Dp) {
  const int p = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (p >= g.P) return;
  float s = 0.f;
  for (int i = lane; i < g.n; i += 32) {
    const float v = Rt32[(size_t)p * g.n_pad + i];
    s = fmaf(v, v, s);
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) Dp[p] = s;
}

// ---------------------------------------------------------------------------
// separable convolution along one axis of column blocks stored row-per-node:
//   out[x, c] = sum_{r=-T..T} tap_c[r] in[x + r e_axis, c]   (nodes off the grid skipped)
// tap_c = tapKu for columns in [ku_lo, ku_hi), tapK otherwise; DUAL writes
// both the tapK (out0) and the tapKu (out1) result.  Rows are in natural node
// order unless IN_PERM (input rows in tile order) / OUT_BF16 (output rows in
// tile order, BF16).
// ---------------------------------------------------------------------------
constexpr int CONV_NB = 8;  // output nodes per thread along the convolution axis

struct ConvArgs {
  Geo3 g;
  const Tab3* tab;
  int axis, ncols;
  const float* in;
  long long ld_in;
  int in_perm;
  void* out0;
  void* out1;
  long long ld_out;
  int ku_lo, ku_hi;
};

template <bool DUAL, bool OUT_BF16>
__global__ void __launch_bounds__(256) k_f3_conv(ConvArgs a) {
  // one thread: CONV_NB consecutive nodes of one line along the axis, 4 columns;
  // every input row of the line segment (plus halo) is loaded once
  constexpr int NB = CONV_NB;
  const int nc4 = a.ncols >> 2;
  const int ax = a.axis;
  const int M = ax == 0 ? a.g.m[0] : ax == 1 ? a.g.m[1] : a.g.m[2];
  const int T = ax == 0 ? a.g.T[0] : ax == 1 ? a.g.T[1] : a.g.T[2];
  const long long stride = ax == 0 ? (long long)a.g.m[1] * a.g.m[2] : ax == 1 ? a.g.m[2] : 1;
  const int nseg = (M + NB - 1) / NB;
  const long long lines = (long long)a.g.P / M;
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= lines * nseg * nc4) return;
  const int c = (int)(idx % nc4) * 4;
  const long long rest = idx / nc4;
  const int seg = (int)(rest % nseg);
  const long long line = rest / nseg;
  // node of the line at axis coordinate 0
  const long long base = (line / stride) * stride * M + (line % stride);
  const int x0 = seg * NB;
  const bool ku = c >= a.ku_lo && c < a.ku_hi;
  const float* tk = ku ? a.tab->tapKu[ax] : a.tab->tapK[ax];
  const float* tu = a.tab->tapKu[ax];
  float4 s0[NB], s1[NB];
#pragma unroll
  for (int o = 0; o < NB; ++o) {
    s0[o] = make_float4(0.f, 0.f, 0.f, 0.f);
    s1[o] = s0[o];
  }
  const int jlo = max(0, x0 - T), jhi = min(M - 1, x0 + NB - 1 + T);
  for (int jn = jlo; jn <= jhi; ++jn) {
    const long long node = base + jn * stride;
    long long row = node;
    if (a.in_perm) {
      const int c2 = (int)(node % a.g.m[2]), c1 = (int)((node / a.g.m[2]) % a.g.m[1]);
      const int c0 = (int)(node / ((long long)a.g.m[2] * a.g.m[1]));
      row = f3_perm(a.g, c0, c1, c2);
    }
    const float4 v = *reinterpret_cast<const float4*>(a.in + row * a.ld_in + c);
#pragma unroll
    for (int o = 0; o < NB; ++o) {
      const int r = jn - (x0 + o);   // input minus output offset
      if (r < -T || r > T) continue;
      const float w = tk[r + F3_TMAX];
      s0[o].x = fmaf(w, v.x, s0[o].x);
      s0[o].y = fmaf(w, v.y, s0[o].y);
      s0[o].z = fmaf(w, v.z, s0[o].z);
      s0[o].w = fmaf(w, v.w, s0[o].w);
      if (DUAL) {
        const float u = tu[r + F3_TMAX];
        s1[o].x = fmaf(u, v.x, s1[o].x);
        s1[o].y = fmaf(u, v.y, s1[o].y);
        s1[o].z = fmaf(u, v.z, s1[o].z);
        s1[o].w = fmaf(u, v.w, s1[o].w);
      }
    }
  }
#pragma unroll
  for (int o = 0; o < NB; ++o) {
    if (x0 + o >= M) break;
    const long long x = base + (long long)(x0 + o) * stride;
    if (OUT_BF16) {
      const int c2 = (int)(x % a.g.m[2]), c1 = (int)((x / a.g.m[2]) % a.g.m[1]);
      const int c0 = (int)(x / ((long long)a.g.m[2] * a.g.m[1]));
      const long long row = f3_perm(a.g, c0, c1, c2);
      __nv_bfloat162* o0 = reinterpret_cast<__nv_bfloat162*>(
          static_cast<__nv_bfloat16*>(a.out0) + row * a.ld_out + c);
      o0[0] = __floats2bfloat162_rn(s0[o].x, s0[o].y);
      o0[1] = __floats2bfloat162_rn(s0[o].z, s0[o].w);
      if (DUAL) {
        __nv_bfloat162* o1 = reinterpret_cast<__nv_bfloat162*>(
            static_cast<__nv_bfloat16*>(a.out1) + row * a.ld_out + c);
        o1[0] = __floats2bfloat162_rn(s1[o].x, s1[o].y);
        o1[1] = __floats2bfloat162_rn(s1[o].z, s1[o].w);
      }
    } else {
      *reinterpret_cast<float4*>(static_cast<float*>(a.out0) + x * a.ld_out + c) = s0[o];
      if (DUAL) *reinterpret_cast<float4*>(static_cast<float*>(a.out1) + x * a.ld_out + c) = s1[o];
    }
  }
}

// ---------------------------------------------------------------------------
// point geometry: k0, mu1, var of the product kernel at node (c0, c1, c2)
// ---------------------------------------------------------------------------
struct PtGeo {
  float k0, ik0, mu1[3], var[3], ivar[3];
};

__device__ __forceinline__ PtGeo f3_geo(const Tab3* __restrict__ tab, int c0, int c1, int c2) {
  PtGeo p;
  const int c[3] = {c0, c1, c2};
  p.k0 = tab->k0[0][c0] * tab->k0[1][c1] * tab->k0[2][c2];
  p.ik0 = 1.f / p.k0;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    p.mu1[j] = tab->mu1[j][c[j]];
    p.var[j] = tab->var[j][c[j]];
    p.ivar[j] = 1.f / p.var[j];
  }
  return p;
}

// X-side scaling for the product form (columns padded to lp, zero beyond l):
// F = [X/k0 | alpha X/k0 | gamma_0 X/k0 | gamma_1 X/k0 | gamma_2 X/k0] (P x 5lp),
// alpha = sum_j mu1_j^2/var_j, gamma_j = mu1_j/var_j.
__global__ void k_f3_xscale(Geo3 g, const Tab3* __restrict__ tab, int l, int lp,
                            const float* __restrict__ X, float* __restrict__ F) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)g.P * lp) return;
  const int x = (int)(e / lp), c = (int)(e - (long long)x * lp);
  const int c2 = x % g.m[2], c1 = (x / g.m[2]) % g.m[1], c0 = x / (g.m[2] * g.m[1]);
  const PtGeo p = f3_geo(tab, c0, c1, c2);
  const float v = c < l ? X[(long long)x * l + c] / p.k0 : 0.f;
  float al = 0.f;
#pragma unroll
  for (int j = 0; j < 3; ++j) al += p.mu1[j] * p.mu1[j] / p.var[j];
  float* row = F + (long long)x * 5 * lp;
  row[c] = v;
  row[lp + c] = al * v;
#pragma unroll
  for (int j = 0; j < 3; ++j) row[(2 + j) * lp + c] = p.mu1[j] / p.var[j] * v;
}

// Ut (128 x p_pad, BF16, tile-order columns): rows [0, lp) = E'X,
// rows [lp, 2lp) = (L - E)'X, from the convolved F (P x 5lp):
//   E'X = KKK(X/k0),  (L - E)'X = KKK(alpha X/k0) + sum_j K..Ku_j..K(gamma_j X/k0)
// (the slope factor of L' is (p_j - t_j)/hM = -(t_j - p_j)/hM, hence the +).
// XT (lp x p_pad, BF16) gets X itself for the correction MMA.
__global__ void k_f3_ut(Geo3 g, int l, int lp, const float* __restrict__ Fc,
                        const float* __restrict__ X, __nv_bfloat16* __restrict__ Ut,
                        __nv_bfloat16* __restrict__ XT) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)g.P * lp) return;
  const int x = (int)(e / lp), c = (int)(e - (long long)x * lp);
  const int c2 = x % g.m[2], c1 = (x / g.m[2]) % g.m[1], c0 = x / (g.m[2] * g.m[1]);
  const long long q = f3_perm(g, c0, c1, c2);
  const float* row = Fc + (long long)x * 5 * lp;
  Ut[(long long)c * g.p_pad + q] = __float2bfloat16_rn(row[c]);
  Ut[(long long)(lp + c) * g.p_pad + q] =
      __float2bfloat16_rn(row[lp + c] + row[2 * lp + c] + row[3 * lp + c] + row[4 * lp + c]);
  XT[(long long)c * g.p_pad + q] = __float2bfloat16_rn(c < l ? X[(long long)x * l + c] : 0.f);
}

// Zb (128 x n_pad, BF16) = sum over the K splits of the partial products.
__global__ void k_f3_zsum(int n_pad, int nsplit, const float* __restrict__ Zp,
                          __nv_bfloat16* __restrict__ Zb) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long N = 128LL * n_pad;
  if (e >= N) return;
  float s = 0.f;
  for (int z = 0; z < nsplit; ++z) s += Zp[z * N + e];
  Zb[e] = __float2bfloat16_rn(s);
}

// Y-side input from W (p_pad x 128, tile-order rows): V = [We We We We Wd] (P x 5lp)
__global__ void k_f3_wgather(Geo3 g, int lp, const float* __restrict__ W, float* __restrict__ Vw) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)g.P * lp) return;
  const int x = (int)(e / lp), c = (int)(e - (long long)x * lp);
  const int c2 = x % g.m[2], c1 = (x / g.m[2]) % g.m[1], c0 = x / (g.m[2] * g.m[1]);
  const long long q = f3_perm(g, c0, c1, c2);
  const float we = W[q * 128 + c], wd = W[q * 128 + lp + c];
  float* row = Vw + (long long)x * 5 * lp;
  row[c] = we;
  row[lp + c] = we;
  row[2 * lp + c] = we;
  row[3 * lp + c] = we;
  row[4 * lp + c] = wd;
}

// Y = Gamma_prod X = L We + E Wd:
//   Y(s) = [(1 + alpha(s)) KKK(We) - sum_j gamma_j(s) K..Ku_j..K(We) + KKK(Wd)](s) / k0(s)
__global__ void k_f3_ycombine(Geo3 g, const Tab3* __restrict__ tab, int l, int lp,
                              const float* __restrict__ Vc, float* __restrict__ Y) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)g.P * l) return;
  const int x = (int)(e / l), c = (int)(e - (long long)x * l);
  const int c2 = x % g.m[2], c1 = (x / g.m[2]) % g.m[1], c0 = x / (g.m[2] * g.m[1]);
  const PtGeo p = f3_geo(tab, c0, c1, c2);
  const float* row = Vc + (long long)x * 5 * lp;
  float al = 0.f, v = 0.f;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const float gj = p.mu1[j] / p.var[j];
    al += p.mu1[j] * gj;
    v -= gj * row[(1 + j) * lp + c];
  }
  v += (1.f + al) * row[c] + row[4 * lp + c];
  Y[e] = v / p.k0;
}

// ---------------------------------------------------------------------------
// per output pair: product-form fit and the near-diagonal correction
// ---------------------------------------------------------------------------
// beta of the product-form fit from the seven products (Pv: P00, P10, P20, P30,
// P01, P02, P03); returns the normalisation 1/(k0(s) k0(t)).
__device__ __forceinline__ float f3_beta(const PtGeo& s, const PtGeo& t, const float Pv[7],
                                         float beta[7]) {
  const float inv = s.ik0 * t.ik0;
  const float z0 = Pv[0] * inv;
  float b0 = z0;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    beta[1 + j] = (Pv[1 + j] * inv - s.mu1[j] * z0) * s.ivar[j];
    beta[4 + j] = (Pv[4 + j] * inv - t.mu1[j] * z0) * t.ivar[j];
    b0 -= s.mu1[j] * beta[1 + j] + t.mu1[j] * beta[4 + j];
  }
  beta[0] = b0;
  return inv;
}

// corr = e0' (A_p - A_d)^{-1} (A_d beta - z_d) for a near pair (all moments
// normalised by k0(s) k0(t)).
//
// On the diagonal pairs p = q the design row is x = [1, u, u - delta] with
// u = u_s(p) and delta = (t - s)/hM, i.e. x = T [1, u] for a fixed 7 x 4 matrix T,
// so A_d = T Md T' and z_d = T qd with the 4 x 4 moment matrix Md of the
// diagonal pairs (a product measure over the axes: per-axis ratios r00, r10,
// r20 of sum_p K_s K_t u^a) and qd = sum_p K_s K_t [1, u] D'_p.  With A_p's
// closed-form inverse (the product-form fit) the Woodbury identity gives
//     corr = g' (I - Md H)^{-1} c,   g = T' A_p^{-1} e0,   H = T' A_p^{-1} T,
//     c = Md T' beta - qd,
// a 4 x 4 solve; g and H have closed forms in the per-axis moments.
__device__ __forceinline__ float f3_corr(const PtGeo& s, const PtGeo& t, const float r00[3],
                                         const float r10[3], const float r20[3], float Q0,
                                         const float Qs[3], const int dx[3], const float ihM[3],
                                         const float beta[7], float inv, int& bad) {
  float dl[3], as[3], et[3], ft[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    dl[j] = dx[j] * ihM[j];
    as[j] = s.mu1[j] * s.ivar[j];
    et[j] = (t.mu1[j] + dl[j]) * t.ivar[j];
    ft[j] = t.mu1[j] * t.ivar[j];
  }
  // H (arrow-shaped: H00, H0k = Hk0, diagonal Hkk) and g
  float H00 = 1.f, g0 = 1.f, H0[3], Hd[3], gk[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    H00 = fmaf(s.mu1[j], as[j], fmaf(t.mu1[j] + dl[j], et[j], H00));
    g0 = fmaf(s.mu1[j], as[j], fmaf(t.mu1[j], et[j], g0));
    H0[j] = -(as[j] + et[j]);
    Hd[j] = s.ivar[j] + t.ivar[j];
    gk[j] = -(as[j] + ft[j]);
  }
  // Md: w0 = prod r00; Md0j = r10_j prod_{k!=j} r00; Mdjj = r20_j prod_{k!=j} r00;
  // Mdjk = r10_j r10_k r00_o
  const float q[3] = {r00[1] * r00[2], r00[0] * r00[2], r00[0] * r00[1]};
  float Md[4][4];
  Md[0][0] = r00[0] * q[0];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    Md[0][1 + j] = Md[1 + j][0] = r10[j] * q[j];
    Md[1 + j][1 + j] = r20[j] * q[j];
  }
  Md[1][2] = Md[2][1] = r10[0] * r10[1] * r00[2];
  Md[1][3] = Md[3][1] = r10[0] * r10[2] * r00[1];
  Md[2][3] = Md[3][2] = r10[1] * r10[2] * r00[0];
  // c = Md T' beta - qd, T' beta = [b0 - sum delta_j bt_j, bs_j + bt_j]
  float tb[4];
  tb[0] = beta[0];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    tb[0] = fmaf(-dl[j], beta[4 + j], tb[0]);
    tb[1 + j] = beta[1 + j] + beta[4 + j];
  }
  const float qd[4] = {Q0 * inv, Qs[0] * inv, Qs[1] * inv, Qs[2] * inv};
  float c[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    float v = -qd[a];
#pragma unroll
    for (int b = 0; b < 4; ++b) v = fmaf(Md[a][b], tb[b], v);
    c[a] = v;
  }
  // M4 = I - Md H
  float M4[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    float v = Md[a][0] * H00;
#pragma unroll
    for (int k = 0; k < 3; ++k) v = fmaf(Md[a][1 + k], H0[k], v);
    M4[a][0] = (a == 0 ? 1.f : 0.f) - v;
#pragma unroll
    for (int b = 1; b < 4; ++b)
      M4[a][b] = (a == b ? 1.f : 0.f) - fmaf(Md[a][0], H0[b - 1], Md[a][b] * Hd[b - 1]);
  }
  // Gaussian elimination (M4 is the identity minus a small term: no pivoting)
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (!(fabsf(M4[k][k]) > 1e-4f)) {
      bad = 1;
      return 0.f;
    }
    const float ip = 1.f / M4[k][k];
#pragma unroll
    for (int i = k + 1; i < 4; ++i) {
      const float f = M4[i][k] * ip;
#pragma unroll
      for (int j = k + 1; j < 4; ++j) M4[i][j] = fmaf(-f, M4[k][j], M4[i][j]);
      c[i] = fmaf(-f, c[k], c[i]);
    }
    M4[k][k] = ip;
  }
  float y[4];
#pragma unroll
  for (int i = 3; i >= 0; --i) {
    float v = c[i];
#pragma unroll
    for (int j = i + 1; j < 4; ++j) v = fmaf(-M4[i][j], y[j], v);
    y[i] = v * M4[i][i];
  }
  return fmaf(g0, y[0], fmaf(gk[0], y[1], fmaf(gk[1], y[2], gk[2] * y[3])));
}

// Diagonal moments by direct sums over the shared window (used for the trace).
__device__ void f3_tdiag_direct(const Geo3& g, const Tab3* __restrict__ tab,
                                const float* __restrict__ Dp, const int sc[3], const int tc[3],
                                float& Q0, float Qs[3]) {
  Q0 = 0.f;
  Qs[0] = Qs[1] = Qs[2] = 0.f;
  int lo[3], hi[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    lo[j] = max(max(sc[j], tc[j]) - g.T[j], 0);
    hi[j] = min(min(sc[j], tc[j]) + g.T[j], g.m[j] - 1);
  }
  for (int p0 = lo[0]; p0 <= hi[0]; ++p0) {
    const float a0 = tab->tapK[0][p0 - sc[0] + F3_TMAX] * tab->tapK[0][p0 - tc[0] + F3_TMAX];
    const float u0 = (p0 - sc[0]) * tab->inv_hM[0];
    float f0 = 0.f, f1 = 0.f, f2 = 0.f;
    for (int p1 = lo[1]; p1 <= hi[1]; ++p1) {
      const float a1 = tab->tapK[1][p1 - sc[1] + F3_TMAX] * tab->tapK[1][p1 - tc[1] + F3_TMAX];
      const float u1 = (p1 - sc[1]) * tab->inv_hM[1];
      const float* drow = Dp + ((long long)p0 * g.m[1] + p1) * g.m[2];
      float e0 = 0.f, e2 = 0.f;
      for (int p2 = lo[2]; p2 <= hi[2]; ++p2) {
        const float w2 = tab->tapK[2][p2 - sc[2] + F3_TMAX] * tab->tapK[2][p2 - tc[2] + F3_TMAX];
        const float dv = w2 * __ldg(drow + p2);
        e0 += dv;
        e2 = fmaf((p2 - sc[2]) * tab->inv_hM[2], dv, e2);
      }
      f0 = fmaf(a1, e0, f0);
      f1 = fmaf(a1 * u1, e0, f1);
      f2 = fmaf(a1, e2, f2);
    }
    Q0 = fmaf(a0, f0, Q0);
    Qs[0] = fmaf(a0 * u0, f0, Qs[0]);
    Qs[1] = fmaf(a0, f1, Qs[1]);
    Qs[2] = fmaf(a0, f2, Qs[2]);
  }
}

// f3_tdiag_direct with the (p0, p1) rows of the window dealt over the 32 lanes of
// a warp and the four sums joined by shuffles (every lane returns them).
__device__ void f3_tdiag_warp(const Geo3& g, const Tab3* __restrict__ tab,
                              const float* __restrict__ Dp, const int sc[3], const int tc[3],
                              int lane, float& Q0, float Qs[3]) {
  int lo[3], hi[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    lo[j] = max(max(sc[j], tc[j]) - g.T[j], 0);
    hi[j] = min(min(sc[j], tc[j]) + g.T[j], g.m[j] - 1);
  }
  const int n1 = hi[1] - lo[1] + 1;
  const int nrow = (hi[0] - lo[0] + 1) * n1;
  float q0 = 0.f, qs0 = 0.f, qs1 = 0.f, qs2 = 0.f;
  for (int r = lane; r < nrow; r += 32) {
    const int p0 = lo[0] + r / n1, p1 = lo[1] + r % n1;
    const float a = tab->tapK[0][p0 - sc[0] + F3_TMAX] * tab->tapK[0][p0 - tc[0] + F3_TMAX] *
                    tab->tapK[1][p1 - sc[1] + F3_TMAX] * tab->tapK[1][p1 - tc[1] + F3_TMAX];
    const float u0 = (p0 - sc[0]) * tab->inv_hM[0];
    const float u1 = (p1 - sc[1]) * tab->inv_hM[1];
    const float* drow = Dp + ((long long)p0 * g.m[1] + p1) * g.m[2];
    float e0 = 0.f, e2 = 0.f;
    for (int p2 = lo[2]; p2 <= hi[2]; ++p2) {
      const float w2 = tab->tapK[2][p2 - sc[2] + F3_TMAX] * tab->tapK[2][p2 - tc[2] + F3_TMAX];
      const float dv = w2 * __ldg(drow + p2);
      e0 += dv;
      e2 = fmaf((p2 - sc[2]) * tab->inv_hM[2], dv, e2);
    }
    q0 = fmaf(a, e0, q0);
    qs0 = fmaf(a * u0, e0, qs0);
    qs1 = fmaf(a * u1, e0, qs1);
    qs2 = fmaf(a, e2, qs2);
  }
  for (int o = 16; o > 0; o >>= 1) {
    q0 += __shfl_xor_sync(0xffffffffu, q0, o);
    qs0 += __shfl_xor_sync(0xffffffffu, qs0, o);
    qs1 += __shfl_xor_sync(0xffffffffu, qs1, o);
    qs2 += __shfl_xor_sync(0xffffffffu, qs2, o);
  }
  Q0 = q0;
  Qs[0] = qs0;
  Qs[1] = qs1;
  Qs[2] = qs2;
}

__device__ __forceinline__ void f3_tile_origin_S(const Geo3& g, int S, int o[3]) {
  const int b2 = S % g.nb[2], b1 = (S / g.nb[2]) % g.nb[1], b0 = S / (g.nb[2] * g.nb[1]);
  o[0] = 4 * b0;
  o[1] = 4 * b1;
  o[2] = 8 * b2;
}

// local row r of an S-tile -> node offsets (the tile order of f3_perm)
__device__ __forceinline__ void f3_srow(int r, int d[3]) {
  d[0] = (r >> 4) & 3;
  d[1] = (r >> 2) & 3;
  d[2] = ((r >> 6) << 2) + (r & 3);
}

// ---------------------------------------------------------------------------
// near-diagonal tile pairs on tcgen05
//
// One CTA walks its S-tiles (128 nodes, a 4 x 4 x 8 box) and, for each, the
// T-tiles (64 nodes, 4 x 4 x 4) that hold near pairs.  Per tile pair:
//   warp 0   TMA loads of the four B_a planes, K = 32 subjects per stage
//            (64-byte rows, 64-byte swizzle), 3 stages;
//   warp 1   tcgen05.mma: the seven products P00, P10..P30, P01..P03 into
//            7 x 64 TMEM columns, then (apply mode) Y_corr += corr X_T into
//            TMEM columns 448.. (BF16 corrections and X, FP32 accumulate);
//   warps 2-9 the epilogue: while the products run they stage the diagonal
//            moments of the pair in shared memory (separable sums over axes
//            0 and 1), then per output pair form beta_prod, and where the
//            windows share nodes the correction; corrections go to shared
//            memory as the A operand of the Y_corr product (apply mode) or
//            Gamma_hat = b0 + corr to global memory (tile mode).
// ---------------------------------------------------------------------------
constexpr int NBK = 32;                    // subjects per K chunk
constexpr int NA_BYTES = SB * NBK * 2;     // 8 KB
constexpr int NB_BYTES = TB * NBK * 2;     // 4 KB
constexpr int NSTAGE_BYTES = 4 * NA_BYTES + 4 * NB_BYTES;
constexpr int NNSTAGE = 3;
constexpr int WMAX = 12;                   // window-union extent per axis (taps <= 4)
constexpr int F3_TSTAGE = 4;               // largest taps the staged kernel takes
constexpr int G0_FLOATS = WMAX * WMAX * 16 * 2;
constexpr int G1_S0 = 16 * 3 + 1;           // padded strides of G1 (bank spread)
constexpr int G1_P2 = 16 * G1_S0 + 5;
constexpr int G1_FLOATS = WMAX * G1_P2;
constexpr int PT_FLOATS = 576;             // pair tables: rho slices, t geometry, taps
constexpr int OFF_CORR = NNSTAGE * NSTAGE_BYTES;
constexpr int OFF_XT = OFF_CORR + CORR_BYTES;
constexpr int OFF_G0 = OFF_XT + XT_BYTES;
constexpr int OFF_G1 = OFF_G0 + G0_FLOATS * 4;
constexpr int OFF_PT = OFF_G1 + G1_FLOATS * 4;
constexpr int OFF_BAR = OFF_PT + PT_FLOATS * 4;
constexpr size_t NEAR_SMEM2 = OFF_BAR + 256 + 1024;
static_assert(NEAR_SMEM2 <= 232448, "near kernel exceeds the 227 KB opt-in shared memory");

struct NearArgs {
  Geo3 g;
  const Tab3* tab;
  const float* Dp;
  int mode;                 // 0: Y += corr X over the work lists; 1: Gamma_hat on tile pairs
  int lp;                   // vectors (columns of X/Y) padded to 16/32/64
  int l;
  float* Y;                 // P x l (mode 0)
  const int* cta_off;       // mode 0: per-CTA ranges of items
  const int* items;         // items x 4: S-tile, first and end index into tlist, output slot
  const int* tlist;         // T-tile indices, grouped per S-tile
  float* Ypart;             // mode 0: per-slot partial sums of corr X (128 x lp each)
  const int* pairs;         // mode 1: npairs x 2 (S, T)
  int npairs;
  float* tiles_out;         // mode 1: npairs x 128 x 64
  int* err;
};

__global__ void __launch_bounds__(NEAR_THREADS, 1)
    k_f3_near(const __grid_constant__ CUtensorMap mapB, const __grid_constant__ CUtensorMap mapX,
              NearArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~uintptr_t(1023));
  uint8_t* corr_s = smem + OFF_CORR;
  uint8_t* xt_s = smem + OFF_XT;
  float* G0 = reinterpret_cast<float*>(smem + OFF_G0);
  float* G1 = reinterpret_cast<float*>(smem + OFF_G1);
  float* PT = reinterpret_cast<float*>(smem + OFF_PT);
  float* rho0 = PT;              // [16][3]  (s0, t0): r00, r10, r20
  float* rho1 = PT + 48;         // [16][3]  (s1, t1)
  float* rho2 = PT + 96;         // [32][3]  (s2, t2)
  float* tgeo = PT + 192;        // [3][4][3] 1/k0, mu1, var of the T-box nodes per axis
  float* tk = PT + 240;          // [3][17]  K(r/hM)
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + OFF_BAR);
  uint64_t* full = bars;
  uint64_t* empty = bars + NNSTAGE;
  uint64_t* tmem_full = bars + 2 * NNSTAGE;
  uint64_t* tmem_empty = tmem_full + 1;
  uint64_t* corr_full = tmem_full + 2;
  uint64_t* ymma_done = tmem_full + 3;
  uint64_t* xt_full = tmem_full + 4;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(tmem_full + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const Geo3& g = a.g;
  const bool apply = a.mode == 0;
  int it_lo = 0, it_hi = 0;
  if (apply) {
    it_lo = a.cta_off[blockIdx.x];
    it_hi = a.cta_off[blockIdx.x + 1];
  }

  if (threadIdx.x == 0) {
    for (int st = 0; st < NNSTAGE; ++st) {
      ptx::mbar_init(ptx::smem_u32(&full[st]), 1);
      ptx::mbar_init(ptx::smem_u32(&empty[st]), 1);
    }
    ptx::mbar_init(ptx::smem_u32(tmem_full), 1);
    ptx::mbar_init(ptx::smem_u32(tmem_empty), 256);
    ptx::mbar_init(ptx::smem_u32(corr_full), 256);
    ptx::mbar_init(ptx::smem_u32(ymma_done), 1);
    ptx::mbar_init(ptx::smem_u32(xt_full), 1);
    *abort_flag = 0;
    ptx::fence_mbar_init();
  }
  if (warp == 2) {
    ptx::tmem_alloc(ptx::smem_u32(tslot), 512);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tslot;
  const int nk = g.n_pad / NBK;

  // Walks this CTA's tile pairs in order: f(S, T, first_of_S, last_of_S, slot).
  auto for_pairs = [&](auto&& f) {
    if (apply) {
      for (int it = it_lo; it < it_hi; ++it) {
        const int S = a.items[4 * it], t0 = a.items[4 * it + 1], t1 = a.items[4 * it + 2];
        const int slot = a.items[4 * it + 3];
        for (int j = t0; j < t1; ++j)
          if (!f(S, a.tlist[j], j == t0, j == t1 - 1, slot)) return;
      }
    } else {
      for (int pi = blockIdx.x; pi < a.npairs; pi += gridDim.x)
        if (!f(a.pairs[2 * pi], a.pairs[2 * pi + 1], true, true, pi)) return;
    }
  };

  if (warp == 0) {
    if (lane == 0) {
      // TMA producer
      uint32_t q = 0, gi = 0, xt_issued = 0;
      for_pairs([&](int S, int T, bool, bool, int) -> bool {
        if (*abort_flag) return false;
        for (int kb = 0; kb < nk; ++kb, ++q) {
          const int st = q % NNSTAGE;
          if (!ptx::mbar_wait(ptx::smem_u32(&empty[st]), ((q / NNSTAGE) & 1) ^ 1u, a.err)) {
            *abort_flag = 1;
            return false;
          }
          const uint32_t fb = ptx::smem_u32(&full[st]);
          ptx::mbar_arrive_expect_tx(fb, NSTAGE_BYTES);
          const uint32_t dst = ptx::smem_u32(smem + st * NSTAGE_BYTES);
#pragma unroll
          for (int p = 0; p < 4; ++p) {
            ptx::tma_load_2d(dst + p * NA_BYTES, &mapB, fb, kb * NBK, p * g.p_pad + S * SB);
            ptx::tma_load_2d(dst + p * NA_BYTES + NA_BYTES / 2, &mapB, fb, kb * NBK,
                             p * g.p_pad + S * SB + 64);
            ptx::tma_load_2d(dst + 4 * NA_BYTES + p * NB_BYTES, &mapB, fb, kb * NBK,
                             p * g.p_pad + T * TB);
          }
        }
        if (apply) {
          // the X tile of this pair, once the previous correction product is done with it
          if (gi > 0 && !ptx::mbar_wait(ptx::smem_u32(ymma_done), (gi - 1) & 1, a.err)) {
            *abort_flag = 1;
            return false;
          }
          const uint32_t xb = ptx::smem_u32(xt_full);
          ptx::mbar_arrive_expect_tx(xb, a.lp * 128);
          ptx::tma_load_2d(ptx::smem_u32(xt_s), &mapX, xb, T * TB, 0);
          xt_issued = gi + 1;
        }
        ++gi;
        return true;
      });
      // let every copy already issued land before the CTA exits
      for (uint32_t k = (q > NNSTAGE ? q - NNSTAGE : 0); k < q; ++k)
        ptx::mbar_wait(ptx::smem_u32(&full[k % NNSTAGE]), (k / NNSTAGE) & 1, a.err);
      if (xt_issued > 0) ptx::mbar_wait(ptx::smem_u32(xt_full), (xt_issued - 1) & 1, a.err);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer
      constexpr uint32_t IDESC_P = ptx::idesc_f32acc(1u, SB, TB);
      const uint32_t idesc_y = ptx::idesc_f32acc(1u, SB, (uint32_t)a.lp);
      uint32_t q = 0, gi = 0;
      for_pairs([&](int, int, bool first, bool, int) -> bool {
        if (*abort_flag) return false;
        if (gi > 0 && !ptx::mbar_wait(ptx::smem_u32(tmem_empty), (gi - 1) & 1, a.err)) {
          *abort_flag = 1;
          return false;
        }
        ptx::tc_fence_after();
        for (int kb = 0; kb < nk; ++kb, ++q) {
          const int st = q % NNSTAGE;
          if (!ptx::mbar_wait(ptx::smem_u32(&full[st]), (q / NNSTAGE) & 1, a.err)) {
            *abort_flag = 1;
            return false;
          }
          ptx::tc_fence_after();
          const uint32_t base = ptx::smem_u32(smem + st * NSTAGE_BYTES);
          const uint32_t bb = base + 4 * NA_BYTES;
#pragma unroll
          for (int kk = 0; kk < NBK / 16; ++kk) {
            const uint32_t acc = (kb | kk) != 0;
            const uint32_t ko = kk * 32;
            const uint64_t b0d = ptx::sdesc_kmajor_sw64(bb + ko);
            const uint64_t a0d = ptx::sdesc_kmajor_sw64(base + ko);
            ptx::tc_mma_f16(tmem + 0, a0d, b0d, IDESC_P, acc);
#pragma unroll
            for (int j = 1; j < 4; ++j) {
              ptx::tc_mma_f16(tmem + 64 * j, ptx::sdesc_kmajor_sw64(base + j * NA_BYTES + ko), b0d,
                              IDESC_P, acc);
              ptx::tc_mma_f16(tmem + 64 * (3 + j), a0d,
                              ptx::sdesc_kmajor_sw64(bb + j * NB_BYTES + ko), IDESC_P, acc);
            }
          }
          ptx::tc_commit(ptx::smem_u32(&empty[st]));
        }
        ptx::tc_commit(ptx::smem_u32(tmem_full));
        if (apply) {
          if (!ptx::mbar_wait(ptx::smem_u32(corr_full), gi & 1, a.err) ||
              !ptx::mbar_wait(ptx::smem_u32(xt_full), gi & 1, a.err)) {
            *abort_flag = 1;
            return false;
          }
          ptx::tc_fence_after();
          const uint32_t cb = ptx::smem_u32(corr_s), xb = ptx::smem_u32(xt_s);
#pragma unroll
          for (int kk = 0; kk < TB / 16; ++kk)
            ptx::tc_mma_f16(tmem + 448, ptx::sdesc_kmajor_sw128(cb + kk * 32),
                            ptx::sdesc_kmajor_sw128(xb + kk * 32), idesc_y,
                            (!first || kk != 0) ? 1u : 0u);
          ptx::tc_commit(ptx::smem_u32(ymma_done));
        }
        ++gi;
        return true;
      });
    }
  } else {
    // epilogue: 8 warps; TMEM lanes 32*(warp % 4).., t columns [32 h, 32 h + 32)
    const int et = threadIdx.x - 64;
    const int quad = warp & 3, half = (warp - 2) >> 2;
    const int r = quad * 32 + lane;
    const uint32_t lane_base = static_cast<uint32_t>(quad * 32) << 16;
    int dr[3];
    f3_srow(r, dr);
    const float ihM[3] = {a.tab->inv_hM[0], a.tab->inv_hM[1], a.tab->inv_hM[2]};
    for (int i = et; i < 3 * 17; i += 256) tk[i] = a.tab->tapK[i / 17][i % 17];
    uint32_t gi = 0;
    int bad = 0;
    for_pairs([&](int S, int T, bool, bool last, int slot) -> bool {
      // uniform start: the previous pair is done with the shared tables
      if (!ptx::named_sync_and(1, 256, *abort_flag == 0)) return false;
      int so[3], to[3], wlo[3], wlen[3];
      f3_tile_origin_S(g, S, so);
      f3_tile_origin_S(g, T >> 1, to);
      to[2] += 4 * (T & 1);
      const int sx[3] = {4, 4, 8};
      bool staged = true;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const int shi = min(so[k] + sx[k] - 1, g.m[k] - 1), thi = min(to[k] + 3, g.m[k] - 1);
        wlo[k] = max(0, max(so[k], to[k]) - g.T[k]);
        wlen[k] = min(g.m[k] - 1, min(shi, thi) + g.T[k]) - wlo[k] + 1;
        staged = staged && wlen[k] > 0;
      }
      // pair tables
      for (int i = et; i < 64 * 3 + 36; i += 256) {
        if (i < 64 * 3) {
          const int e = i / 3, qk = i % 3;
          int ax, sl, tl;
          if (e < 16) { ax = 0; sl = e >> 2; tl = e & 3; }
          else if (e < 32) { ax = 1; sl = (e - 16) >> 2; tl = (e - 16) & 3; }
          else { ax = 2; sl = (e - 32) >> 2; tl = (e - 32) & 3; }
          const int sv = so[ax] + sl, tv = to[ax] + tl, dd = tv - sv;
          float v = 0.f;
          if (sv < g.m[ax] && tv < g.m[ax] && dd <= 2 * g.T[ax] && -dd <= 2 * g.T[ax])
            v = a.tab->rho[ax][sv][dd + 2 * F3_TMAX][qk == 2 ? 3 : qk];
          PT[i] = v;
        } else {
          const int e = i - 64 * 3, ax = e / 12, tl = (e % 12) / 3, qk = e % 3;
          const int tv = to[ax] + tl;
          float v = qk == 1 ? 0.f : 1.f;
          if (tv < g.m[ax])
            v = qk == 0 ? 1.f / a.tab->k0[ax][tv]
                        : qk == 1 ? a.tab->mu1[ax][tv] : a.tab->var[ax][tv];
          tgeo[e] = v;
        }
      }
      if (staged) {
        // stage 1, axis 0: G0[p1][p2][s0 t0][a0] = sum_p0 K_s0 K_t0 u0^a0 D'
        const int n1 = wlen[1] * wlen[2] * 16;
        for (int e = et; e < n1; e += 256) {
          const int p1i = e / (wlen[2] * 16), rem = e - p1i * wlen[2] * 16;
          const int p2i = rem >> 4, st0 = rem & 15;
          const int s0 = so[0] + (st0 >> 2), t0 = to[0] + (st0 & 3);
          float c0 = 0.f, c1 = 0.f;
          if (s0 < g.m[0] && t0 < g.m[0]) {
            const int lo = max(max(s0, t0) - g.T[0], 0), hi = min(min(s0, t0) + g.T[0], g.m[0] - 1);
            const float* dcol = a.Dp + (long long)(wlo[1] + p1i) * g.m[2] + (wlo[2] + p2i);
            const long long stp = (long long)g.m[1] * g.m[2];
            for (int p0 = lo; p0 <= hi; ++p0) {
              const float w = tk[p0 - s0 + F3_TMAX] * tk[p0 - t0 + F3_TMAX];
              const float dv = w * __ldg(dcol + p0 * stp);
              c0 += dv;
              c1 = fmaf((p0 - s0) * ihM[0], dv, c1);
            }
          }
          float* o = G0 + ((p1i * WMAX + p2i) * 16 + st0) * 2;
          o[0] = c0;
          o[1] = c1;
        }
        ptx::named_sync(1, 256);
        // stage 2, axis 1: G1[p2][s0 t0][s1 t1][c], c = (a0,a1) = 00, 10, 01
        const int n2 = wlen[2] * 256;
        for (int e = et; e < n2; e += 256) {
          const int p2i = e >> 8, st0 = (e >> 4) & 15, st1 = e & 15;
          const int s1 = so[1] + (st1 >> 2), t1 = to[1] + (st1 & 3);
          float c0 = 0.f, c1 = 0.f, c2 = 0.f;
          if (s1 < g.m[1] && t1 < g.m[1]) {
            const int lo = max(max(s1, t1) - g.T[1], 0), hi = min(min(s1, t1) + g.T[1], g.m[1] - 1);
            for (int p1 = lo; p1 <= hi; ++p1) {
              const float w = tk[17 + p1 - s1 + F3_TMAX] * tk[17 + p1 - t1 + F3_TMAX];
              const float* src = G0 + (((p1 - wlo[1]) * WMAX + p2i) * 16 + st0) * 2;
              c0 = fmaf(w, src[0], c0);
              c1 = fmaf(w, src[1], c1);
              c2 = fmaf(w * (p1 - s1) * ihM[1], src[0], c2);
            }
          }
          float* o = G1 + p2i * G1_P2 + st0 * G1_S0 + st1 * 3;
          o[0] = c0;
          o[1] = c1;
          o[2] = c2;
        }
      }
      ptx::named_sync(1, 256);
      // the seven products of this pair
      bool ok = ptx::mbar_wait(ptx::smem_u32(tmem_full), gi & 1, a.err);
      if (apply && gi > 0) ok = ok && ptx::mbar_wait(ptx::smem_u32(ymma_done), (gi - 1) & 1, a.err);
      if (!ptx::named_sync_and(1, 256, ok)) {
        *abort_flag = 1;
        return false;
      }
      ptx::tc_fence_after();
      const int sc[3] = {so[0] + dr[0], so[1] + dr[1], so[2] + dr[2]};
      const bool s_ok = sc[0] < g.m[0] && sc[1] < g.m[1] && sc[2] < g.m[2];
      PtGeo sg = {};
      if (s_ok) sg = f3_geo(a.tab, sc[0], sc[1], sc[2]);
      float cv[8];
#pragma unroll 1
      for (int ch = 0; ch < 8; ++ch) {
        const int col0 = half * 32 + ch * 4;
        uint32_t v[7][4];
#pragma unroll
        for (int p = 0; p < 7; ++p)
          asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                       : "=r"(v[p][0]), "=r"(v[p][1]), "=r"(v[p][2]), "=r"(v[p][3])
                       : "r"(tmem + lane_base + p * 64 + col0));
        ptx::tmem_ld_wait();
#pragma unroll 1
        for (int j = 0; j < 4; ++j) {
          const int tj = col0 + j;
          const int tl[3] = {tj >> 4, (tj >> 2) & 3, tj & 3};
          const int tc[3] = {to[0] + tl[0], to[1] + tl[1], to[2] + tl[2]};
          const bool t_ok = tc[0] < g.m[0] && tc[1] < g.m[1] && tc[2] < g.m[2];
          float b0 = 0.f, corr = 0.f;
          if (s_ok && t_ok) {
            float Pv[7];
#pragma unroll
            for (int p = 0; p < 7; ++p) {
              uint32_t x = v[p][0];
#pragma unroll
              for (int qq = 1; qq < 4; ++qq) x = (qq == j) ? v[p][qq] : x;   // register select
              Pv[p] = __uint_as_float(x);
            }
            PtGeo tg;
            tg.ik0 = tgeo[0 * 12 + tl[0] * 3] * tgeo[1 * 12 + tl[1] * 3] * tgeo[2 * 12 + tl[2] * 3];
            tg.k0 = 1.f / tg.ik0;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
              tg.mu1[k] = tgeo[k * 12 + tl[k] * 3 + 1];
              tg.var[k] = tgeo[k * 12 + tl[k] * 3 + 2];
              tg.ivar[k] = 1.f / tg.var[k];
            }
            float beta[7];
            const float inv = f3_beta(sg, tg, Pv, beta);
            b0 = beta[0];
            const int dx[3] = {tc[0] - sc[0], tc[1] - sc[1], tc[2] - sc[2]};
            bool near = true;
#pragma unroll
            for (int k = 0; k < 3; ++k) near = near && dx[k] <= 2 * g.T[k] && -dx[k] <= 2 * g.T[k];
            if (near) {
              const float* r0 = rho0 + (dr[0] * 4 + tl[0]) * 3;
              const float* r1 = rho1 + (dr[1] * 4 + tl[1]) * 3;
              const float* r2 = rho2 + (dr[2] * 4 + tl[2]) * 3;
              const float r00[3] = {r0[0], r1[0], r2[0]};
              const float r10[3] = {r0[1], r1[1], r2[1]};
              const float r20[3] = {r0[2], r1[2], r2[2]};
              // stage 3, axis 2, from G1
              const int st0 = dr[0] * 4 + tl[0], st1 = dr[1] * 4 + tl[1];
              const int lo = max(max(sc[2], tc[2]) - g.T[2], 0);
              const int hi = min(min(sc[2], tc[2]) + g.T[2], g.m[2] - 1);
              float Q0 = 0.f, Qs[3] = {0.f, 0.f, 0.f};
              for (int p2 = lo; p2 <= hi; ++p2) {
                const float w = tk[34 + p2 - sc[2] + F3_TMAX] * tk[34 + p2 - tc[2] + F3_TMAX];
                const float* src = G1 + (p2 - wlo[2]) * G1_P2 + st0 * G1_S0 + st1 * 3;
                Q0 = fmaf(w, src[0], Q0);
                Qs[0] = fmaf(w, src[1], Qs[0]);
                Qs[1] = fmaf(w, src[2], Qs[1]);
                Qs[2] = fmaf(w * (p2 - sc[2]) * ihM[2], src[0], Qs[2]);
              }
              corr = f3_corr(sg, tg, r00, r10, r20, Q0, Qs, dx, ihM, beta, inv, bad);
            }
          }
          const int cj = (ch & 1) * 4 + j;
#pragma unroll
          for (int qq = 0; qq < 8; ++qq) cv[qq] = (qq == cj) ? corr : cv[qq];
          if (!apply) {
            const int sl = (dr[0] * 4 + dr[1]) * 8 + dr[2];
            const int tlc = (tl[0] * 4 + tl[1]) * 4 + tl[2];
            a.tiles_out[((long long)slot * SB + sl) * TB + tlc] =
                (s_ok && t_ok) ? b0 + corr : __int_as_float(0x7fc00000);
          }
        }
        if (apply && (ch & 1)) {
          // row r, 16-byte chunk (half*4 + ch/2) of the 128-byte swizzled row
          const int chunk = (half * 4 + (ch >> 1)) ^ (r & 7);
          uint4 pk;
          __nv_bfloat162 h0 = __floats2bfloat162_rn(cv[0], cv[1]);
          __nv_bfloat162 h1 = __floats2bfloat162_rn(cv[2], cv[3]);
          __nv_bfloat162 h2 = __floats2bfloat162_rn(cv[4], cv[5]);
          __nv_bfloat162 h3 = __floats2bfloat162_rn(cv[6], cv[7]);
          pk.x = *reinterpret_cast<uint32_t*>(&h0);
          pk.y = *reinterpret_cast<uint32_t*>(&h1);
          pk.z = *reinterpret_cast<uint32_t*>(&h2);
          pk.w = *reinterpret_cast<uint32_t*>(&h3);
          *reinterpret_cast<uint4*>(corr_s + (r >> 3) * 1024 + (r & 7) * 128 + chunk * 16) = pk;
        }
      }
      ptx::tc_fence_before();
      if (apply) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(ptx::smem_u32(tmem_empty))
                   : "memory");
      if (apply) {
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(ptx::smem_u32(corr_full))
                     : "memory");
        if (last) {
          // the S-tile's correction sum: Y rows += TMEM columns 448..
          const bool okw = ptx::mbar_wait(ptx::smem_u32(ymma_done), gi & 1, a.err);
          if (!ptx::named_sync_and(1, 256, okw)) {
            *abort_flag = 1;
            return false;
          }
          ptx::tc_fence_after();
          const int cpw = a.lp / 2;
          float* yp = a.Ypart + ((long long)slot * SB + r) * a.lp;
          for (int c0 = half * cpw; c0 < (half + 1) * cpw; c0 += 8) {
            uint32_t y[8];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                : "=r"(y[0]), "=r"(y[1]), "=r"(y[2]), "=r"(y[3]), "=r"(y[4]), "=r"(y[5]),
                  "=r"(y[6]), "=r"(y[7])
                : "r"(tmem + lane_base + 448 + c0));
            ptx::tmem_ld_wait();
            float4* d4 = reinterpret_cast<float4*>(yp + c0);
            d4[0] = make_float4(__uint_as_float(y[0]), __uint_as_float(y[1]), __uint_as_float(y[2]),
                                __uint_as_float(y[3]));
            d4[1] = make_float4(__uint_as_float(y[4]), __uint_as_float(y[5]), __uint_as_float(y[6]),
                                __uint_as_float(y[7]));
          }
          ptx::tc_fence_before();
        }
      }
      ++gi;
      return true;
    });
    if (bad) atomicExch(a.err, DERR_NUMERIC);
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 2) ptx::tmem_dealloc(tmem, 512);
}

// Y += the partial correction sums of the NCHUNK slots of each S-tile, in slot order.
__global__ void k_f3_yreduce(Geo3 g, int nchunk, int l, int lp, const float* __restrict__ Ypart,
                             float* __restrict__ Y) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int nS = g.nb[0] * g.nb[1] * g.nb[2];
  if (e >= (long long)nS * SB * l) return;
  const int c = (int)(e % l);
  const int r = (int)((e / l) % SB);
  const int S = (int)(e / ((long long)l * SB));
  int o[3], d[3];
  f3_tile_origin_S(g, S, o);
  f3_srow(r, d);
  const int c0 = o[0] + d[0], c1 = o[1] + d[1], c2 = o[2] + d[2];
  if (c0 >= g.m[0] || c1 >= g.m[1] || c2 >= g.m[2]) return;
  float acc = 0.f;
  for (int k = 0; k < nchunk; ++k) acc += Ypart[(((long long)S * nchunk + k) * SB + r) * lp + c];
  Y[(((long long)c0 * g.m[1] + c1) * g.m[2] + c2) * l + c] += acc;
}

// ---------------------------------------------------------------------------
// generic C[M x N] (+)= A[M x K] B[N x K]' on tcgen05, BF16 K-major operands,
// FP32 output; blockIdx = (m tile, n tile, k split)
// ---------------------------------------------------------------------------
constexpr int GM_STAGES = 4;
constexpr int GM_TILE = 128 * BK * 2;
constexpr size_t GM_SMEM = GM_STAGES * 2 * GM_TILE + 1024 + 256;

__global__ void __launch_bounds__(128, 1)
    k_f3_gemm(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
              int kchunks, int kper, float* out, long long ld, long long split_stride, int* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + GM_STAGES * 2 * GM_TILE);
  uint64_t* empty = full + GM_STAGES;
  uint64_t* done = empty + GM_STAGES;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int k0 = blockIdx.z * kper, k1 = min(kchunks, k0 + kper);
  const int nk = max(0, k1 - k0);
  if (threadIdx.x == 0) {
    for (int s = 0; s < GM_STAGES; ++s) {
      ptx::mbar_init(ptx::smem_u32(&full[s]), 1);
      ptx::mbar_init(ptx::smem_u32(&empty[s]), 1);
    }
    ptx::mbar_init(ptx::smem_u32(done), 1);
    ptx::fence_mbar_init();
  }
  if (warp == 2) {
    ptx::tmem_alloc(ptx::smem_u32(tslot), 128);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tslot;
  if (warp == 0 && lane == 0) {
    int issued = 0;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % GM_STAGES;
      if (!ptx::mbar_wait(ptx::smem_u32(&empty[s]), ((kb / GM_STAGES) & 1) ^ 1u, err)) break;
      const uint32_t fb = ptx::smem_u32(&full[s]);
      ptx::mbar_arrive_expect_tx(fb, 2 * GM_TILE);
      const uint32_t dst = ptx::smem_u32(smem + s * 2 * GM_TILE);
      ptx::tma_load_2d(dst, &mapA, fb, (k0 + kb) * BK, blockIdx.x * 128);
      ptx::tma_load_2d(dst + GM_TILE, &mapB, fb, (k0 + kb) * BK, blockIdx.y * 128);
      issued = kb + 1;
    }
    if (issued < nk)
      for (int kb = (issued > GM_STAGES ? issued - GM_STAGES : 0); kb < issued; ++kb)
        ptx::mbar_wait(ptx::smem_u32(&full[kb % GM_STAGES]), (kb / GM_STAGES) & 1, err);
  } else if (warp == 1 && lane == 0 && nk > 0) {
    constexpr uint32_t IDESC = ptx::idesc_f32acc(1u, 128, 128);
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % GM_STAGES;
      if (!ptx::mbar_wait(ptx::smem_u32(&full[s]), (kb / GM_STAGES) & 1, err)) break;
      ptx::tc_fence_after();
      const uint32_t ab = ptx::smem_u32(smem + s * 2 * GM_TILE);
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk)
        ptx::tc_mma_f16(tmem, ptx::sdesc_kmajor_sw128(ab + kk * 32),
                        ptx::sdesc_kmajor_sw128(ab + GM_TILE + kk * 32), IDESC, (kb | kk) != 0);
      ptx::tc_commit(ptx::smem_u32(&empty[s]));
    }
    ptx::tc_commit(ptx::smem_u32(done));
  }
  __syncwarp();
  const bool have = nk > 0 && ptx::mbar_wait(ptx::smem_u32(done), 0, err);
  __syncwarp();
  ptx::tc_fence_after();
  const long long row = blockIdx.x * 128LL + warp * 32 + lane;
  float* o = out + blockIdx.z * split_stride + row * ld + blockIdx.y * 128LL;
#pragma unroll 1
  for (int c = 0; c < 4; ++c) {
    uint32_t r[32];
    if (have) {
      ptx::tmem_ld_32x32b_x32(tmem + (static_cast<uint32_t>(warp * 32) << 16) + c * 32, r);
      ptx::tmem_ld_wait();
    } else {
#pragma unroll
      for (int j = 0; j < 32; ++j) r[j] = 0u;
    }
    float4* dst = reinterpret_cast<float4*>(o + c * 32);
#pragma unroll
    for (int j = 0; j < 8; ++j)
      dst[j] = make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]),
                           __uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3]));
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 2) ptx::tmem_dealloc(tmem, 128);
}

// trace of Gamma_hat: sum_s Gamma_hat(s, s) from the seven products at (s, s)
__global__ void k_f3_trace(Geo3 g, const Tab3* __restrict__ tab, const float* __restrict__ Dp,
                           const __nv_bfloat16* __restrict__ Bpl, double* trace, double* diag,
                           int* err) {
  const int x = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  double contrib = 0.0;
  if (x < g.P) {
    const int c2 = x % g.m[2], c1 = (x / g.m[2]) % g.m[1], c0 = x / (g.m[2] * g.m[1]);
    const long long q = f3_perm(g, c0, c1, c2);
    const size_t plane = (size_t)g.p_pad * g.n_pad;
    const __nv_bfloat16* b[4];
    for (int p = 0; p < 4; ++p) b[p] = Bpl + p * plane + q * g.n_pad;
    float Pv[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int i = lane; i < g.n_pad; i += 32) {
      const float v0 = __bfloat162float(b[0][i]);
      Pv[0] = fmaf(v0, v0, Pv[0]);
      for (int j = 1; j < 4; ++j) {
        const float vj = __bfloat162float(b[j][i]);
        Pv[j] = fmaf(vj, v0, Pv[j]);
        Pv[3 + j] = fmaf(v0, vj, Pv[3 + j]);
      }
    }
    for (int p = 0; p < 7; ++p)
      for (int o = 16; o > 0; o >>= 1) Pv[p] += __shfl_xor_sync(0xffffffffu, Pv[p], o);
    const int sc[3] = {c0, c1, c2};
    float Q0, Qs[3];
    f3_tdiag_warp(g, tab, Dp, sc, sc, lane, Q0, Qs);
    if (lane == 0) {
      const PtGeo sg = f3_geo(tab, c0, c1, c2);
      float beta[7];
      const float inv = f3_beta(sg, sg, Pv, beta);
      float r00[3], r10[3], r20[3];
      for (int j = 0; j < 3; ++j) {
        r00[j] = tab->rho[j][sc[j]][2 * F3_TMAX][0];
        r10[j] = tab->rho[j][sc[j]][2 * F3_TMAX][1];
        r20[j] = tab->rho[j][sc[j]][2 * F3_TMAX][3];
      }
      const int dx[3] = {0, 0, 0};
      int bad = 0;
      const float corr = f3_corr(sg, sg, r00, r10, r20, Q0, Qs, dx, tab->inv_hM, beta, inv, bad);
      if (bad) atomicExch(err, DERR_NUMERIC);
      contrib = (double)(beta[0] + corr);
      if (diag) diag[x] = contrib;
    }
  }
  // the block's warps summed in shared memory, one atomic per block
  __shared__ double wsum[32];
  if (lane == 0) wsum[threadIdx.x >> 5] = contrib;
  __syncthreads();
  if (trace && threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wsum[w];
    atomicAdd(trace, t);
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 2-D BF16 tensor map: rows x cols (cols contiguous), box {box_cols, box_rows},
// 128-byte swizzle for 64-column boxes, 64-byte swizzle for 32-column boxes.
bool make_map(CUtensorMap* map, const void* base, long long rows, long long cols, int box_rows,
              int box_cols = 64) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUtensorMapSwizzle sw =
      box_cols == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
  return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box,
             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int taps_of(double h, int M) {
  int k = 0;
  while ((double)(k + 1) / (h * M) < 1.0) ++k;
  return k;
}

struct FactorLayout {
  size_t off_rt32, off_rb, off_rbt, off_dp, bytes;
};

FactorLayout factor_layout(const Geo3& g) {
  FactorLayout L;
  size_t o = 0;
  auto take = [&](size_t b) {
    const size_t at = o;
    o = (o + b + 255) & ~size_t(255);
    return at;
  };
  L.off_rt32 = take(sizeof(float) * (size_t)g.P * g.n_pad);
  L.off_rb = take(2 * (size_t)g.n_pad * g.p_pad);
  L.off_rbt = take(2 * (size_t)g.p_pad * g.n_pad);
  L.off_dp = take(sizeof(float) * (size_t)g.P);
  L.bytes = o;
  return L;
}

Geo3 make_geo(const fpca_grid* grid, int n, const double* h) {
  Geo3 g{};
  for (int k = 0; k < 3; ++k) {
    g.m[k] = grid->m[k];
    g.T[k] = h ? taps_of(h[k], grid->m[k]) : 0;
  }
  g.nb[0] = (g.m[0] + 3) / 4;
  g.nb[1] = (g.m[1] + 3) / 4;
  g.nb[2] = (g.m[2] + 7) / 8;
  g.P = g.m[0] * g.m[1] * g.m[2];
  g.p_pad = g.nb[0] * g.nb[1] * g.nb[2] * SB;
  g.n = n;
  g.n_pad = (n + 127) / 128 * 128;
  return g;
}

fpca_status check_grid(fpca_ctx* ctx, const fpca_grid* grid, int n) {
  if (!grid || grid->d != 3)
    return fpca_fail(ctx, FPCA_E_UNSUPPORTED, "the fused smoother is built for d = 3 grids");
  for (int k = 0; k < 3; ++k)
    if (grid->m[k] < 2 || grid->m[k] > F3_MMAX)
      return fpca_fail(ctx, FPCA_E_UNSUPPORTED, "fused smoother: grid.m[%d] must be 2..%d", k,
                       F3_MMAX);
  if (n < 2) return fpca_fail(ctx, FPCA_E_INVALID_ARG, "the covariance needs n >= 2 subjects");
  return FPCA_OK;
}

fpca_status check_h(fpca_ctx* ctx, const Geo3& g, const double* h) {
  if (!h) return fpca_fail(ctx, FPCA_E_INVALID_ARG, "h is required");
  for (int k = 0; k < 3; ++k) {
    if (!(h[k] > 0.0)) return fpca_fail(ctx, FPCA_E_INVALID_ARG, "h[%d] must be positive", k);
    if (g.T[k] < 1 || g.T[k] > F3_TSTAGE)
      return fpca_fail(ctx, FPCA_E_UNSUPPORTED,
                       "fused smoother: taps per axis must be 1..%d (axis %d has %d)", F3_TSTAGE, k,
                       g.T[k]);
  }
  return FPCA_OK;
}

// Near tile-pair work lists (cached per grid and taps in the context).
fpca_status ensure_lists(fpca_ctx* ctx, const Geo3& g) {
  const int key[8] = {g.m[0], g.m[1], g.m[2], g.T[0], g.T[1], g.T[2], 1, 0};
  if (ctx->f3_lists && std::memcmp(key, ctx->f3_key, sizeof(key)) == 0) return FPCA_OK;
  const int nS = g.nb[0] * g.nb[1] * g.nb[2];
  std::vector<int> t_off(nS + 1, 0), tlist;
  for (int S = 0; S < nS; ++S) {
    const int b2 = S % g.nb[2], b1 = (S / g.nb[2]) % g.nb[1], b0 = S / (g.nb[2] * g.nb[1]);
    const int slo[3] = {4 * b0, 4 * b1, 8 * b2};
    const int shi[3] = {std::min(4 * b0 + 3, g.m[0] - 1), std::min(4 * b1 + 3, g.m[1] - 1),
                        std::min(8 * b2 + 7, g.m[2] - 1)};
    t_off[S] = (int)tlist.size();
    for (int T = 0; T < 2 * nS; ++T) {
      const int Sb = T >> 1;
      const int c2 = Sb % g.nb[2], c1 = (Sb / g.nb[2]) % g.nb[1], c0 = Sb / (g.nb[2] * g.nb[1]);
      const int tlo[3] = {4 * c0, 4 * c1, 8 * c2 + 4 * (T & 1)};
      bool ok = true;
      for (int k = 0; k < 3 && ok; ++k) {
        const int thi = std::min(tlo[k] + 3, g.m[k] - 1);
        if (tlo[k] > g.m[k] - 1) {
          ok = false;
          break;
        }
        const int dist = std::max(0, std::max(tlo[k] - shi[k], slo[k] - thi));
        ok = dist <= 2 * g.T[k];
      }
      if (ok) tlist.push_back(T);
    }
  }
  t_off[nS] = (int)tlist.size();
  // Each S-tile's T-list is cut into F3_CHUNKS nearly equal items; items are dealt
  // round-robin to the CTAs in S-tile order, so that the chunks of one S-tile run
  // on different SMs at about the same time and share its operands through L2.
  std::vector<int> items;
  for (int S = 0; S < nS; ++S) {
    const int len = t_off[S + 1] - t_off[S];
    for (int k = 0; k < F3_CHUNKS; ++k) {
      const int tb = t_off[S] + (int)((long long)len * k / F3_CHUNKS);
      const int te = t_off[S] + (int)((long long)len * (k + 1) / F3_CHUNKS);
      if (te > tb) {
        items.push_back(S);
        items.push_back(tb);
        items.push_back(te);
        items.push_back(S * F3_CHUNKS + k);
      }
    }
  }
  const int nitems = (int)items.size() / 4;
  const int ncta = std::max(1, std::min(nitems, ctx->num_sms > 0 ? ctx->num_sms : 148));
  std::vector<int> cta_off(ncta + 1, 0), order;
  for (int c = 0; c < ncta; ++c) {
    cta_off[c] = (int)order.size() / 4;
    for (int it = c; it < nitems; it += ncta)
      order.insert(order.end(), items.begin() + 4 * it, items.begin() + 4 * it + 4);
  }
  cta_off[ncta] = (int)order.size() / 4;
  std::vector<int> all;
  all.insert(all.end(), cta_off.begin(), cta_off.end());
  all.insert(all.end(), order.begin(), order.end());
  all.insert(all.end(), tlist.begin(), tlist.end());
  const size_t bytes = all.size() * sizeof(int);
  // building the lists uploads from the host and waits: the first call for a grid and
  // taps runs outside a capture; later calls find the lists cached
  if (fpca_no_capture(ctx, "building the near-pair work lists") != FPCA_OK)
    return FPCA_E_UNSUPPORTED;
  if (bytes > ctx->f3_lists_bytes) {
    if (ctx->f3_lists) cudaFree(ctx->f3_lists);
    ctx->f3_lists = nullptr;
    ctx->f3_lists_bytes = 0;
    if (cudaMalloc(&ctx->f3_lists, bytes) != cudaSuccess) {
      cudaGetLastError();
      return fpca_fail(ctx, FPCA_E_OOM, "work lists");
    }
    ctx->f3_lists_bytes = bytes;
  }
  if (cudaMemcpyAsync(ctx->f3_lists, all.data(), bytes, cudaMemcpyHostToDevice, ctx->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(ctx->stream) != cudaSuccess)
    return fpca_fail(ctx, FPCA_E_CUDA, "work list upload");
  std::memcpy(ctx->f3_key, key, sizeof(key));
  ctx->f3_ncta = ncta;
  ctx->f3_nitems = nitems;
  ctx->f3_npairs = (int)tlist.size();
  return FPCA_OK;
}

// Everything one fused apply needs, carved from the workspace.
struct F3Work {
  Geo3 g;
  int l, lp, nsplit;
  const float* Rt32;
  const __nv_bfloat16* Rb;
  const __nv_bfloat16* Rbt;
  const float* Dp;
  Tab3* tab;
  __nv_bfloat16* Bpl;   // 4 planes p_pad x n_pad
  float* H[5];          // P x n_pad scratch for the B planes
  float *F, *F1, *F2;   // P x 5l
  __nv_bfloat16* Ut;    // 128 x p_pad
  __nv_bfloat16* XT;    // lp x p_pad
  float* Zp;            // nsplit x 128 x n_pad
  __nv_bfloat16* Zb;    // 128 x n_pad
  float* Wf;            // p_pad x 128
  float* Ypart;         // S-tiles x F3_CHUNKS x 128 x lp
  CUtensorMap mapB, mapX, mapUt, mapRb, mapRbt, mapZb;
  fpca_ctx* ctx;
};

size_t f3_work_bytes(const Geo3& g, int l, int lp, int nsplit) {
  size_t b = WsCarve::round(sizeof(Tab3));
  b += WsCarve::round(2 * 4 * (size_t)g.p_pad * g.n_pad);
  b += 5 * WsCarve::round(sizeof(float) * (size_t)g.P * g.n_pad);
  b += 3 * WsCarve::round(sizeof(float) * (size_t)g.P * 5 * lp);
  b += WsCarve::round(2 * 128 * (size_t)g.p_pad) + WsCarve::round(2 * (size_t)lp * g.p_pad);
  b += WsCarve::round(sizeof(float) * (size_t)nsplit * 128 * g.n_pad);
  b += WsCarve::round(2 * 128 * (size_t)g.n_pad) + WsCarve::round(sizeof(float) * (size_t)g.p_pad * 128);
  b += WsCarve::round(sizeof(float) * (size_t)(g.p_pad / SB) * F3_CHUNKS * SB * lp);
  return b + 4096;
}

void f3_work_carve(WsCarve& c, F3Work& w) {
  const Geo3& g = w.g;
  w.tab = c.take<Tab3>(1);
  w.Bpl = c.take<__nv_bfloat16>(4 * (size_t)g.p_pad * g.n_pad);
  for (int i = 0; i < 5; ++i) w.H[i] = c.take<float>((size_t)g.P * g.n_pad);
  w.F = c.take<float>((size_t)g.P * 5 * w.lp);
  w.F1 = c.take<float>((size_t)g.P * 5 * w.lp);
  w.F2 = c.take<float>((size_t)g.P * 5 * w.lp);
  w.Ut = c.take<__nv_bfloat16>(128 * (size_t)g.p_pad);
  w.XT = c.take<__nv_bfloat16>((size_t)w.lp * g.p_pad);
  w.Zp = c.take<float>((size_t)w.nsplit * 128 * g.n_pad);
  w.Zb = c.take<__nv_bfloat16>(128 * (size_t)g.n_pad);
  w.Wf = c.take<float>((size_t)g.p_pad * 128);
  w.Ypart = c.take<float>((size_t)(g.p_pad / SB) * F3_CHUNKS * SB * w.lp);
}

fpca_status conv_launch(fpca_ctx* ctx, const F3Work& w, int axis, int ncols, const float* in,
                        long long ld_in, int in_perm, void* out0, void* out1, long long ld_out,
                        int ku_lo, int ku_hi, bool dual, bool bf16) {
  ConvArgs a;
  a.g = w.g;
  a.tab = w.tab;
  a.axis = axis;
  a.ncols = ncols;
  a.in = in;
  a.ld_in = ld_in;
  a.in_perm = in_perm;
  a.out0 = out0;
  a.out1 = out1;
  a.ld_out = ld_out;
  a.ku_lo = ku_lo;
  a.ku_hi = ku_hi;
  const int M = w.g.m[axis];
  const long long total = (long long)(w.g.P / M) * ((M + CONV_NB - 1) / CONV_NB) * (ncols / 4);
  const int nb = (int)((total + 255) / 256);
  if (dual && bf16)
    k_f3_conv<true, true><<<nb, 256, 0, ctx->stream>>>(a);
  else if (dual)
    k_f3_conv<true, false><<<nb, 256, 0, ctx->stream>>>(a);
  else if (bf16)
    k_f3_conv<false, true><<<nb, 256, 0, ctx->stream>>>(a);
  else
    k_f3_conv<false, false><<<nb, 256, 0, ctx->stream>>>(a);
  FPCA_LAUNCHED(ctx, "f3_conv");
  return FPCA_OK;
}

// B_a = R~ conv (K u_a), a = 0 (K K K), 1 (Ku K K), 2 (K Ku K), 3 (K K Ku): BF16 planes.
fpca_status f3_planes(fpca_ctx* ctx, const F3Work& w) {
  const Geo3& g = w.g;
  const long long ldn = g.n_pad;
  const size_t plane = (size_t)g.p_pad * g.n_pad;
  cudaMemsetAsync(w.Bpl, 0, 2 * 4 * plane, ctx->stream);
  fpca_status s;
  // axis 0: R -> H0 (K), H1 (Ku)
  s = conv_launch(ctx, w, 0, g.n_pad, w.Rt32, ldn, 0, w.H[0], w.H[1], ldn, 0, 0, true, false);
  if (s != FPCA_OK) return s;
  // axis 1: H0 -> H2 (KK), H3 (K Ku); H1 -> H4 (Ku K)
  s = conv_launch(ctx, w, 1, g.n_pad, w.H[0], ldn, 0, w.H[2], w.H[3], ldn, 0, 0, true, false);
  if (s != FPCA_OK) return s;
  s = conv_launch(ctx, w, 1, g.n_pad, w.H[1], ldn, 0, w.H[4], nullptr, ldn, 0, 0, false, false);
  if (s != FPCA_OK) return s;
  // axis 2: H2 -> B0 (KKK), B3 (KKKu); H3 -> B2 (KKuK); H4 -> B1 (KuKK)
  s = conv_launch(ctx, w, 2, g.n_pad, w.H[2], ldn, 0, w.Bpl, w.Bpl + 3 * plane, ldn, 0, 0, true, true);
  if (s != FPCA_OK) return s;
  s = conv_launch(ctx, w, 2, g.n_pad, w.H[3], ldn, 0, w.Bpl + 2 * plane, nullptr, ldn, 0, 0, false,
                  true);
  if (s != FPCA_OK) return s;
  return conv_launch(ctx, w, 2, g.n_pad, w.H[4], ldn, 0, w.Bpl + 1 * plane, nullptr, ldn, 0, 0,
                     false, true);
}

fpca_status f3_prepare(fpca_ctx* ctx, F3Work& w, const void* factor, const double* h) {
  const Geo3& g = w.g;
  const FactorLayout L = factor_layout(g);
  const char* base = static_cast<const char*>(factor);
  w.Rt32 = reinterpret_cast<const float*>(base + L.off_rt32);
  w.Rb = reinterpret_cast<const __nv_bfloat16*>(base + L.off_rb);
  w.Rbt = reinterpret_cast<const __nv_bfloat16*>(base + L.off_rbt);
  w.Dp = reinterpret_cast<const float*>(base + L.off_dp);
  w.ctx = ctx;
  k_f3_tables<<<3, 256, 0, ctx->stream>>>(g, h[0], h[1], h[2], w.tab);
  FPCA_LAUNCHED(ctx, "f3_tables");
  if (!make_map(&w.mapB, w.Bpl, 4LL * g.p_pad, g.n_pad, 64, NBK) ||
      !make_map(&w.mapX, w.XT, w.lp, g.p_pad, w.lp) ||
      !make_map(&w.mapUt, w.Ut, 128, g.p_pad, 128) ||
      !make_map(&w.mapRb, w.Rb, g.n_pad, g.p_pad, 128) ||
      !make_map(&w.mapRbt, w.Rbt, g.p_pad, g.n_pad, 128) ||
      !make_map(&w.mapZb, w.Zb, 128, g.n_pad, 128))
    return fpca_fail(ctx, FPCA_E_CUDA, "tensor map encode failed");
  return f3_planes(ctx, w);
}

fpca_status f3_gemm(fpca_ctx* ctx, const CUtensorMap& A, const CUtensorMap& B, int mt, int nt,
                    int kchunks, int nsplit, float* out, long long ld, long long split_stride) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_f3_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GM_SMEM);
    attr = true;
  }
  const int kper = (kchunks + nsplit - 1) / nsplit;
  k_f3_gemm<<<dim3(mt, nt, nsplit), 128, GM_SMEM, ctx->stream>>>(A, B, kchunks, kper, out, ld,
                                                                 split_stride, ctx->d_err);
  FPCA_LAUNCHED(ctx, "f3_gemm");
  return FPCA_OK;
}

fpca_status f3_near_launch(fpca_ctx* ctx, const F3Work& w, int mode, float* Y, const int* pairs,
                           int npairs, float* tiles_out) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_f3_near, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)NEAR_SMEM2);
    attr = true;
  }
  NearArgs a{};
  a.g = w.g;
  a.tab = w.tab;
  a.Dp = w.Dp;
  a.mode = mode;
  a.lp = w.lp;
  a.l = w.l;
  a.Y = Y;
  a.err = ctx->d_err;
  int grid;
  if (mode == 0) {
    const int* L = static_cast<const int*>(ctx->f3_lists);
    const int ncta = ctx->f3_ncta;
    a.cta_off = L;
    a.items = L + ncta + 1;
    a.tlist = a.items + 4 * ctx->f3_nitems;
    a.Ypart = w.Ypart;
    grid = ncta;
    const size_t nS = (size_t)w.g.nb[0] * w.g.nb[1] * w.g.nb[2];
    cudaMemsetAsync(w.Ypart, 0, sizeof(float) * nS * F3_CHUNKS * SB * w.lp, ctx->stream);
  } else {
    a.pairs = pairs;
    a.npairs = npairs;
    a.tiles_out = tiles_out;
    grid = std::max(1, std::min(npairs, ctx->num_sms > 0 ? ctx->num_sms : 148));
  }
  k_f3_near<<<grid, NEAR_THREADS, NEAR_SMEM2, ctx->stream>>>(w.mapB, w.mapX, a);
  FPCA_LAUNCHED(ctx, "f3_near");
  if (mode == 0) {
    const long long nS = (long long)w.g.nb[0] * w.g.nb[1] * w.g.nb[2];
    const long long tot = nS * SB * w.l;
    k_f3_yreduce<<<(int)((tot + 255) / 256), 256, 0, ctx->stream>>>(w.g, F3_CHUNKS, w.l, w.lp,
                                                                   w.Ypart, Y);
    FPCA_LAUNCHED(ctx, "f3_yreduce");
  }
  return FPCA_OK;
}

// Y = Gamma_hat X (P x l, natural node order).
fpca_status f3_apply(fpca_ctx* ctx, F3Work& w, const float* X, float* Y) {
  const Geo3& g = w.g;
  const int l = w.l, lp = w.lp, c5 = 5 * lp;
  const int nbp = (int)(((long long)g.P * lp + 255) / 256);
  const int nbl = (int)(((long long)g.P * l + 255) / 256);
  fpca_status s;
  // X side: F = scaled copies, three axis passes, then Ut and XT
  k_f3_xscale<<<nbp, 256, 0, ctx->stream>>>(g, w.tab, l, lp, X, w.F);
  FPCA_LAUNCHED(ctx, "f3_xscale");
  s = conv_launch(ctx, w, 0, c5, w.F, c5, 0, w.F1, nullptr, c5, 2 * lp, 3 * lp, false, false);
  if (s != FPCA_OK) return s;
  s = conv_launch(ctx, w, 1, c5, w.F1, c5, 0, w.F2, nullptr, c5, 3 * lp, 4 * lp, false, false);
  if (s != FPCA_OK) return s;
  s = conv_launch(ctx, w, 2, c5, w.F2, c5, 0, w.F1, nullptr, c5, 4 * lp, 5 * lp, false, false);
  if (s != FPCA_OK) return s;
  cudaMemsetAsync(w.Ut, 0, 2 * 128 * (size_t)g.p_pad, ctx->stream);
  cudaMemsetAsync(w.XT, 0, 2 * (size_t)lp * g.p_pad, ctx->stream);
  k_f3_ut<<<nbp, 256, 0, ctx->stream>>>(g, l, lp, w.F1, X, w.Ut, w.XT);
  FPCA_LAUNCHED(ctx, "f3_ut");
  // Z' = R~ [E'X, (L-E)'X] (as its transpose, split over the node range), then W = R~' Z'
  s = f3_gemm(ctx, w.mapUt, w.mapRb, 1, g.n_pad / 128, g.p_pad / BK, w.nsplit, w.Zp, g.n_pad,
              128LL * g.n_pad);
  if (s != FPCA_OK) return s;
  k_f3_zsum<<<(int)((128LL * g.n_pad + 255) / 256), 256, 0, ctx->stream>>>(g.n_pad, w.nsplit, w.Zp,
                                                                           w.Zb);
  FPCA_LAUNCHED(ctx, "f3_zsum");
  s = f3_gemm(ctx, w.mapRbt, w.mapZb, g.p_pad / 128, 1, g.n_pad / BK, 1, w.Wf, 128, 0);
  if (s != FPCA_OK) return s;
  // Y side: V = [We We We We Wd], axis passes (Ku on one We copy per axis), combine
  k_f3_wgather<<<nbp, 256, 0, ctx->stream>>>(g, lp, w.Wf, w.F);
  FPCA_LAUNCHED(ctx, "f3_wgather");
  s = conv_launch(ctx, w, 0, c5, w.F, c5, 0, w.F1, nullptr, c5, lp, 2 * lp, false, false);
  if (s != FPCA_OK) return s;
  s = conv_launch(ctx, w, 1, c5, w.F1, c5, 0, w.F2, nullptr, c5, 2 * lp, 3 * lp, false, false);
  if (s != FPCA_OK) return s;
  s = conv_launch(ctx, w, 2, c5, w.F2, c5, 0, w.F1, nullptr, c5, 3 * lp, 4 * lp, false, false);
  if (s != FPCA_OK) return s;
  k_f3_ycombine<<<nbl, 256, 0, ctx->stream>>>(g, w.tab, l, lp, w.F1, Y);
  FPCA_LAUNCHED(ctx, "f3_ycombine");
  // near-diagonal corrections
  return f3_near_launch(ctx, w, 0, Y, nullptr, 0, nullptr);
}

fpca_status f3_apply_cb(void* self, const float* X, float* Y) {
  F3Work* w = static_cast<F3Work*>(self);
  return f3_apply(w->ctx, *w, X, Y);
}

int pad_l(int l) { return l <= 16 ? 16 : l <= 32 ? 32 : 64; }

}  // namespace

extern "C" {

size_t fpca_cov_factor_bytes(const fpca_grid* grid, int n) {
  if (!grid || grid->d != 3 || n < 1) return 0;
  return factor_layout(make_geo(grid, n, nullptr)).bytes;
}

fpca_status fpca_bin_cov_factor(fpca_ctx* ctx, const fpca_data* data, const fpca_grid* grid,
                                const double* mu, void* factor, size_t factor_bytes) {
  if (!ctx) return FPCA_E_INVALID_ARG;
  fpca_prof_mark(ctx);
  if (!data || !mu || !factor)
    return fpca_fail(ctx, FPCA_E_INVALID_ARG, "data, mu and factor are required");
  fpca_status s = check_grid(ctx, grid, data->n);
  if (s != FPCA_OK) return s;
  if (data->layout != FPCA_DENSE || data->mask != nullptr)
    return fpca_fail(ctx, FPCA_E_UNSUPPORTED,
                     "the factored covariance needs fully observed gridded data (dense, mask NULL)");
  if (!data->y || (data->y_prec != FPCA_F64 && data->y_prec != FPCA_F32))
    return fpca_fail(ctx, FPCA_E_INVALID_ARG, "dense y must be FPCA_F64 or FPCA_F32");
  const Geo3 g = make_geo(grid, data->n, nullptr);
  const FactorLayout L = factor_layout(g);
  if (factor_bytes < L.bytes)
    return fpca_fail(ctx, FPCA_E_INVALID_ARG, "factor buffer holds %zu bytes, needs %zu",
                     factor_bytes, L.bytes);
  char* base = static_cast<char*>(factor);
  cudaMemsetAsync(factor, 0, L.bytes, ctx->stream);
  float* Rt32 = reinterpret_cast<float*>(base + L.off_rt32);
  __nv_bfloat16* Rb = reinterpret_cast<__nv_bfloat16*>(base + L.off_rb);
  __nv_bfloat16* Rbt = reinterpret_cast<__nv_bfloat16*>(base + L.off_rbt);
  float* Dp = reinterpret_cast<float*>(base + L.off_dp);
  const float scale = (float)(1.0 / std::sqrt((double)g.n));
  dim3 grd((g.P + 31) / 32, (g.n_pad + 31) / 32), blk(32, 8);
  if (data->y_prec == FPCA_F64)
    k_f3_residuals<double><<<grd, blk, 0, ctx->stream>>>(g, static_cast<const double*>(data->y), mu,
                                                         scale, Rt32, Rbt, Rb);
  else
    k_f3_residuals<float><<<grd, blk, 0, ctx->stream>>>(g, static_cast<const float*>(data->y), mu,
                                                        scale, Rt32, Rbt, Rb);
  FPCA_LAUNCHED(ctx, "f3_residuals");
  k_f3_diag<<<(g.P + 7) / 8, 256, 0, ctx->stream>>>(g, Rt32, Dp);
  FPCA_LAUNCHED(ctx, "f3_diag");
  return FPCA_OK;
}

static fpca_status f3_setup(fpca_ctx* ctx, const fpca_grid* grid, const void* factor, int n,
                            const double* h, int l, size_t extra, F3Work& w, void** ws_out) {
  fpca_status s = check_grid(ctx, grid, n);
  if (s != FPCA_OK) return s;
  if (!factor) return fpca_fail(ctx, FPCA_E_INVALID_ARG, "factor is required");
  w.g = make_geo(grid, n, h);
  s = check_h(ctx, w.g, h);
  if (s != FPCA_OK) return s;
  if (l < 1 || l > 64) return fpca_fail(ctx, FPCA_E_INVALID_ARG, "l must be 1..64");
  w.l = l;
  w.lp = pad_l(l);
  const int ntile = w.g.n_pad / 128;
  const int sms = ctx->num_sms > 0 ? ctx->num_sms : 148;
  w.nsplit = std::max(1, std::min(w.g.p_pad / BK, sms / std::max(1, ntile)));
  s = ensure_lists(ctx, w.g);
  if (s != FPCA_OK) return s;
  const size_t need = f3_work_bytes(w.g, l, w.lp, w.nsplit) + extra;
  void* ws = fpca_workspace(ctx, need);
  if (!ws) return fpca_fail(ctx, FPCA_E_OOM, "workspace (%zu bytes)", need);
  *ws_out = ws;
  return FPCA_OK;
}

fpca_status fpca_smooth_cov_apply(fpca_ctx* ctx, const fpca_grid* grid, const void* factor, int n,
                                  const double* h, const float* x, int l, float* y) {
  if (!ctx) return FPCA_E_INVALID_ARG;
  fpca_prof_mark(ctx);
  if (!x || !y) return fpca_fail(ctx, FPCA_E_INVALID_ARG, "x and y are required");
  F3Work w{};
  void* ws = nullptr;
  fpca_status s = f3_setup(ctx, grid, factor, n, h, l, 0, w, &ws);
  if (s != FPCA_OK) return s;
  WsCarve c(ws);
  f3_work_carve(c, w);
  s = f3_prepare(ctx, w, factor, h);
  if (s != FPCA_OK) return s;
  return f3_apply(ctx, w, x, y);
}

fpca_status fpca_smooth_cov_tiles(fpca_ctx* ctx, const fpca_grid* grid, const void* factor, int n,
                                  const double* h, int ntiles, const int32_t* tiles, float* out) {
  if (!ctx) return FPCA_E_INVALID_ARG;
  fpca_prof_mark(ctx);
  if (ntiles < 1 || !tiles || !out)
    return fpca_fail(ctx, FPCA_E_INVALID_ARG, "ntiles >= 1, tiles and out are required");
  F3Work w{};
  void* ws = nullptr;
  const size_t extra = WsCarve::round(sizeof(int) * 2 * (size_t)ntiles);
  fpca_status s = f3_setup(ctx, grid, factor, n, h, 16, extra, w, &ws);
  if (s != FPCA_OK) return s;
  const Geo3& g = w.g;
  std::vector<int> pairs(2 * (size_t)ntiles);
  for (int i = 0; i < ntiles; ++i) {
    const int32_t* t = tiles + 6 * (size_t)i;
    if (t[0] % 4 || t[1] % 4 || t[2] % 8 || t[3] % 4 || t[4] % 4 || t[5] % 4)
      return fpca_fail(ctx, FPCA_E_INVALID_ARG,
                       "tile %d: s corner must be a multiple of (4,4,8), t corner of (4,4,4)", i);
    for (int k = 0; k < 3; ++k)
      if (t[k] < 0 || t[k] >= g.m[k] || t[3 + k] < 0 || t[3 + k] >= g.m[k])
        return fpca_fail(ctx, FPCA_E_INVALID_ARG, "tile %d: corner outside the grid", i);
    const int S = ((t[0] / 4) * g.nb[1] + t[1] / 4) * g.nb[2] + t[2] / 8;
    const int Sb = ((t[3] / 4) * g.nb[1] + t[4] / 4) * g.nb[2] + t[5] / 8;
    pairs[2 * i] = S;
    pairs[2 * i + 1] = 2 * Sb + ((t[5] % 8) / 4);
  }
  WsCarve c(ws);
  f3_work_carve(c, w);
  int* dpairs = c.take<int>(2 * (size_t)ntiles);
  if (fpca_no_capture(ctx, "fpca_smooth_cov_tiles") != FPCA_OK) return FPCA_E_UNSUPPORTED;
  if (cudaMemcpyAsync(dpairs, pairs.data(), sizeof(int) * pairs.size(), cudaMemcpyHostToDevice,
                      ctx->stream) != cudaSuccess)
    return fpca_fail(ctx, FPCA_E_CUDA, "tile list upload");
  s = f3_prepare(ctx, w, factor, h);
  if (s != FPCA_OK) return s;
  s = f3_near_launch(ctx, w, 1, nullptr, dpairs, ntiles, out);
  if (s != FPCA_OK) return s;
  // the host tile list must outlive the upload
  if (cudaStreamSynchronize(ctx->stream) != cudaSuccess)
    return fpca_fail(ctx, FPCA_E_CUDA, "stream");
  return FPCA_OK;
}

fpca_status fpca_rproj_eig_factor(fpca_ctx* ctx, const fpca_grid* grid, const void* factor, int n,
                                  const double* h, const float* omega, int l, int k,
                                  int power_iters, double* evals, double* evecs, double* fve) {
  if (!ctx) return FPCA_E_INVALID_ARG;
  fpca_prof_mark(ctx);
  if (!omega || !evals || !evecs)
    return fpca_fail(ctx, FPCA_E_INVALID_ARG, "omega, evals and evecs are required");
  if (k < 1 || l <= k || l > 64)
    return fpca_fail(ctx, FPCA_E_INVALID_ARG, "random projection needs 1 <= k < l <= 64");
  if (power_iters < 0 || power_iters > 16)
    return fpca_fail(ctx, FPCA_E_INVALID_ARG, "power_iters must be 0..16");
  F3Work w{};
  void* ws = nullptr;
  const int P = grid ? grid->m[0] * grid->m[1] * grid->m[2] : 0;
  fpca_status s = f3_setup(ctx, grid, factor, n, h, l, rproj_ws_bytes(ctx, P, l), w, &ws);
  if (s != FPCA_OK) return s;
  WsCarve c(ws);
  f3_work_carve(c, w);
  RprojWs rw;
  rproj_ws_carve(ctx, c, P, l, rw);
  s = f3_prepare(ctx, w, factor, h);
  if (s != FPCA_OK) return s;
  cudaMemsetAsync(rw.trace, 0, sizeof(double), ctx->stream);
  k_f3_trace<<<(P + 7) / 8, 256, 0, ctx->stream>>>(w.g, w.tab, w.Dp, w.Bpl, rw.trace, nullptr,
                                                    ctx->d_err);
  FPCA_LAUNCHED(ctx, "f3_trace");
  RprojOp op{f3_apply_cb, &w};
  return rproj_operator(ctx, P, l, k, power_iters, 1.0 / (double)P, omega, op, rw, evals, evecs,
                        fve);
}

fpca_status fpca_smooth_cov_diag(fpca_ctx* ctx, const fpca_grid* grid, const void* factor, int n,
                                 const double* h, double* diag) {
  if (!ctx) return FPCA_E_INVALID_ARG;
  fpca_prof_mark(ctx);
  if (!diag) return fpca_fail(ctx, FPCA_E_INVALID_ARG, "diag is required");
  F3Work w{};
  void* ws = nullptr;
  fpca_status s = f3_setup(ctx, grid, factor, n, h, 16, 0, w, &ws);
  if (s != FPCA_OK) return s;
  WsCarve c(ws);
  f3_work_carve(c, w);
  s = f3_prepare(ctx, w, factor, h);
  if (s != FPCA_OK) return s;
  const int P = w.g.P;
  k_f3_trace<<<(P + 7) / 8, 256, 0, ctx->stream>>>(w.g, w.tab, w.Dp, w.Bpl, nullptr, diag,
                                                    ctx->d_err);
  FPCA_LAUNCHED(ctx, "f3_diag_values");
  return FPCA_OK;
}

}  // extern "C"
