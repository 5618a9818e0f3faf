// Eigen step: matrixisation (Section 3.1, Eq. 3.1) and the random projection
// of Section 3.4 (range finder with power iterations and Rayleigh-Ritz).
//
//  Sigma    = (G + G')/2, NaN -> 0, rows/columns outside the domain -> 0
//  Y        = Sigma Omega;  repeat q times { Q = orth(Y); Y = Sigma Q }
//  Q        = orth(Y) by CholeskyQR2 (compensated FP32 Gram, float-float Cholesky)
//  B        = Q' Sigma Q (compensated FP32 sums, FP64 result); eigenpairs of B
//             by FP32 Jacobi and two Ogita-Aishima refinement steps
//  Psi      = Q U;  lambda = theta dV;  phi = psi / sqrt(dV);  dV = 1/P
// The dense path (full = 1) diagonalises Sigma itself (n <= 1024): block Jacobi in
// FP32 spread over the GPU, then FP64 Ogita-Aishima refinement (launch_dense_eig).
#include <cmath>

#include "fpca_internal.cuh"
#include "ff.cuh"
#include "ptx.cuh"

namespace {

template <typename TG>
__device__ __forceinline__ double gval(const TG* G, long long idx) {
  const double x = (double)G[idx];
  return isnan(x) ? 0.0 : x;
}

// Sigma = sym(G) with NaN and out-of-domain entries zeroed; trace accumulated.
// The arithmetic is done in the type of Sigma (FP32 for the projected path).
// A block takes the pair of 32 x 32 tiles (I, J) and (J, I), I <= J (blocks
// below the diagonal return at once), so G is read once and Sigma written once:
// s = (g_pq + g_qp) / 2 is formed for (p, q) in (I, J) and written there and,
// through the shared tile, to (q, p).  Since the sum is commutative, Sigma is
// exactly symmetric.
template <typename TG, typename TS>
__global__ void k_matrixize(int P, const TG* __restrict__ G, const int32_t* __restrict__ dom,
                            TS* __restrict__ S, double* __restrict__ trace) {
  __shared__ TS tile[32][33];
  __shared__ double dsum;  // this block's part of the trace (diagonal blocks only)
  if (blockIdx.y > blockIdx.x) return;
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  if (threadIdx.x == 0 && threadIdx.y == 0) dsum = 0.0;
  // tile[r][c] = g(j0 + r, i0 + c)
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int q = j0 + r, p = i0 + threadIdx.x;
    TS v = TS(0);
    if (q < P && p < P) {
      v = (TS)G[(long long)q * P + p];
      if (isnan(v)) v = TS(0);
    }
    tile[r][threadIdx.x] = v;
  }
  __syncthreads();
  // (p, q) = (i0 + r, j0 + c): s = (g_pq + tile[c][r]) / 2, kept in tile[c][r]
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int p = i0 + r, q = j0 + threadIdx.x;
    TS sv = TS(0);
    if (p < P && q < P) {
      TS g = (TS)G[(long long)p * P + q];
      if (isnan(g)) g = TS(0);
      sv = TS(0.5) * (g + tile[threadIdx.x][r]);
      if (dom && (dom[p] <= 0 || dom[q] <= 0)) sv = TS(0);
      S[(long long)p * P + q] = sv;
      if (p == q) atomicAdd(&dsum, (double)sv);
    }
    tile[threadIdx.x][r] = sv;
  }
  __syncthreads();
  if (i0 == j0) {
    // one global atomic per diagonal block instead of one per diagonal entry
    if (threadIdx.x == 0 && threadIdx.y == 0) atomicAdd(trace, dsum);
    return;
  }
  // (q, p) = (j0 + r, i0 + c) takes s(p, q) = tile[r][c]
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int q = j0 + r, p = i0 + threadIdx.x;
    if (q < P && p < P) S[(long long)q * P + p] = tile[r][threadIdx.x];
  }
}

// Y (P x l) = S X for the symmetric S that k_matrixize writes (P x P, FP32).
// Since S[k][p] == S[p][k] exactly, S is read by its rows k: the lanes of a warp
// hold 32 consecutive output rows p (coalesced loads of S), and X[k][.] is the
// same for the whole warp (shared-memory broadcasts).  A thread owns RPT rows
// 32 apart, a block PJ_WARPS warps side by side (a tile of PJ_WARPS * 32 * RPT
// rows) over one range of kb values of k, X staged in shared memory in chunks of
// kc rows (a multiple of 2 PJ_U; the last chunk's missing rows are zero).
// Every k range writes its partial product to part[range][c][p]; k_proj_sum adds
// the ranges in order (no atomics: the result does not depend on scheduling).
constexpr int PJ_WARPS = 8;
constexpr int PJ_U = 8;    // k values per batch of loads of S

// Accumulators of k_proj: RPT rows x LM columns per thread.  PAIRED keeps them in
// column pairs, so that one paired FMA (fma.rn.f32x2) updates two columns of a row
// and a k step issues LM / 2 FMA instructions per row (used where the pairs fit the
// registers without spilling: LM <= 20 with RPT = 2, LM = 8 with RPT = 4).
template <int LM, int RPT, bool PAIRED>
struct ProjAcc;
template <int LM, int RPT>
struct ProjAcc<LM, RPT, true> {
  float2 a[RPT][LM / 2];
  __device__ __forceinline__ ProjAcc() {
#pragma unroll
    for (int r = 0; r < RPT; ++r)
#pragma unroll
      for (int c = 0; c < LM / 2; ++c) a[r][c] = make_float2(0.f, 0.f);
  }
  __device__ __forceinline__ void fma4(int r, int c4, float sv, float4 x) {
    const float2 s2 = make_float2(sv, sv);
    a[r][2 * c4] = __ffma2_rn(s2, make_float2(x.x, x.y), a[r][2 * c4]);
    a[r][2 * c4 + 1] = __ffma2_rn(s2, make_float2(x.z, x.w), a[r][2 * c4 + 1]);
  }
  __device__ __forceinline__ float get(int r, int c) const {
    return (c & 1) ? a[r][c >> 1].y : a[r][c >> 1].x;
  }
};
template <int LM, int RPT>
struct ProjAcc<LM, RPT, false> {
  float a[RPT][LM];
  __device__ __forceinline__ ProjAcc() {
#pragma unroll
    for (int r = 0; r < RPT; ++r)
#pragma unroll
      for (int c = 0; c < LM; ++c) a[r][c] = 0.f;
  }
  __device__ __forceinline__ void fma4(int r, int c4, float sv, float4 x) {
    a[r][4 * c4] = fmaf(sv, x.x, a[r][4 * c4]);
    a[r][4 * c4 + 1] = fmaf(sv, x.y, a[r][4 * c4 + 1]);
    a[r][4 * c4 + 2] = fmaf(sv, x.z, a[r][4 * c4 + 2]);
    a[r][4 * c4 + 3] = fmaf(sv, x.w, a[r][4 * c4 + 3]);
  }
  __device__ __forceinline__ float get(int r, int c) const { return a[r][c]; }
};

template <int LM, int RPT>
__global__ void __launch_bounds__(PJ_WARPS * 32, 2)
    k_proj(int P, int l, int kb, int kc, const float* __restrict__ S,
           const float* __restrict__ X, float* __restrict__ part) {
  extern __shared__ float4 xs4[];   // [kc][LM / 4]: one chunk of X, rows past the range zero
  constexpr int L4 = LM / 4;
  float* xs = reinterpret_cast<float*>(xs4);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int pbase = (blockIdx.x * PJ_WARPS + warp) * 32 * RPT + lane;
  const int kend = min(P, (blockIdx.y + 1) * kb);
  ProjAcc<LM, RPT, (LM <= 20)> acc;
  for (int k0 = blockIdx.y * kb; k0 < kend; k0 += kc) {
    const int nk = min(kend - k0, kc);
    __syncthreads();
    for (int e = threadIdx.x; e < kc * LM; e += blockDim.x) {
      const int kk = e / LM, c = e - kk * LM;
      xs[e] = (kk < nk && c < l) ? X[(long long)(k0 + kk) * l + c] : 0.f;
    }
    __syncthreads();
    // two batches of S in registers: the loads of one are in flight while the
    // other is multiplied (X holds zero rows up to a multiple of 2 PJ_U)
    float sa[PJ_U][RPT], sb[PJ_U][RPT];
    auto load = [&](float (&sv)[PJ_U][RPT], int k) {
#pragma unroll
      for (int u = 0; u < PJ_U; ++u)
#pragma unroll
        for (int r = 0; r < RPT; ++r) {
          const int p = pbase + 32 * r;
          sv[u][r] = (k + u < nk && p < P) ? __ldg(S + (long long)(k0 + k + u) * P + p) : 0.f;
        }
    };
    auto fmas = [&](const float (&sv)[PJ_U][RPT], int k) {
#pragma unroll
      for (int u = 0; u < PJ_U; ++u)
#pragma unroll
        for (int c4 = 0; c4 < L4; ++c4) {
          const float4 x = xs4[(k + u) * L4 + c4];
#pragma unroll
          for (int r = 0; r < RPT; ++r) acc.fma4(r, c4, sv[u][r], x);
        }
    };
    load(sa, 0);
    for (int k = 0; k < nk; k += 2 * PJ_U) {
      load(sb, k + PJ_U);
      fmas(sa, k);
      load(sa, k + 2 * PJ_U);
      fmas(sb, k + PJ_U);
    }
  }
  float* out = part + (long long)blockIdx.y * l * P;
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    const int p = pbase + 32 * r;
    if (p < P) {
#pragma unroll
      for (int c = 0; c < LM; ++c)
        if (c < l) out[(long long)c * P + p] = acc.get(r, c);
    }
  }
}

// Y[p][c] = sum over the k ranges, in range order, of part[range][c][p].
__global__ void k_proj_sum(int P, int l, int ranges, const float* __restrict__ part,
                           float* __restrict__ Y) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;   // c * P + p
  const long long n = (long long)P * l;
  if (i >= n) return;
  // loads in groups of eight (independent of the sum), added in range order
  float s = 0.f;
  int j = 0;
  for (; j + 8 <= ranges; j += 8) {
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = part[(j + u) * n + i];
#pragma unroll
    for (int u = 0; u < 8; ++u) s += v[u];
  }
  for (; j < ranges; ++j) s += part[j * n + i];
  const int c = (int)(i / P), p = (int)(i - (long long)c * P);
  Y[(long long)p * l + c] = s;
}

// Y = S X as above, for 8 < l <= 20 and P a multiple of 8, with the rows of S
// brought into shared memory by the TMA engine: a stage holds PJT_KS values of k,
// each one bulk copy of the tile's (up to) 512 entries of row k, and PJT_ST stages
// are in flight on mbarriers (issued by thread 0, a slot released by the block
// barrier that ends its stage), so no register holds a load in flight.  Thread
// (rg, cg) = (t / 4, t % 4) owns rows 4 rg .. 4 rg + 3 and 256 + 4 rg .. 256 + 4 rg + 3
// of the tile and columns 5 cg .. 5 cg + 4 (X staged as [k][cg][8], three zero pads):
// per k, two 128-bit reads of S (a warp's eight row groups are 128 contiguous
// bytes), a 128-bit and a 32-bit read of X, and 20 paired FMAs over row pairs.
// Each (p, c) adds its products over k in the order of k_proj: the same bits.
constexpr int PJT_KS = 8;
constexpr int PJT_ST = 4;
constexpr int PJT_ROWS = 512;
constexpr int PJT_KC = 128;   // k values of X per staged chunk (16 KB)

inline size_t proj_tma_smem(int kc) {
  return sizeof(float) * ((size_t)PJT_ST * PJT_KS * PJT_ROWS + (size_t)kc * 32);
}

__global__ void __launch_bounds__(256, 2)
    k_proj_tma(int P, int l, int kb, int kc, const float* __restrict__ S,
               const float* __restrict__ X, float* __restrict__ part, int* __restrict__ err) {
  extern __shared__ __align__(128) float pts[];
  __shared__ __align__(8) uint64_t bars[PJT_ST];
  float* ss = pts;                                             // [PJT_ST][PJT_KS][512]
  float* xs = pts + (size_t)PJT_ST * PJT_KS * PJT_ROWS;        // [kc][4][8]
  const int t = threadIdx.x, rg = t >> 2, cg = t & 3;
  const int p_tile = blockIdx.x * PJT_ROWS;
  const int nrows = min(PJT_ROWS, P - p_tile);                 // a multiple of 8
  const uint32_t rbytes = (uint32_t)nrows * 4u;
  const int kbeg = blockIdx.y * kb, kend = min(P, kbeg + kb);
  if (t == 0) {
    for (int i = 0; i < PJT_ST; ++i) ptx::mbar_init(ptx::smem_u32(&bars[i]), 1);
    ptx::fence_mbar_init();
  }
  float2 acc[4][5];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 5; ++c) acc[r][c] = make_float2(0.f, 0.f);
  int g = 0;   // stages consumed before this chunk (slot and phase of the next one)
  for (int k0 = kbeg; k0 < kend; k0 += kc) {
    const int ns = min(kend - k0, kc) / PJT_KS;   // kb, kc and P are multiples of PJT_KS
    __syncthreads();   // the barriers' init (first chunk) / last chunk's reads of X
    for (int e = t; e < ns * PJT_KS * 32; e += 256) {
      const int j = e & 7, c = ((e >> 3) & 3) * 5 + j;
      xs[e] = (j < 5 && c < l) ? X[(long long)(k0 + (e >> 5)) * l + c] : 0.f;
    }
    // stage st of this chunk into slot (g + st) % PJT_ST (thread 0)
    auto issue = [&](int st) {
      const int slot = (g + st) % PJT_ST;
      const uint32_t bar = ptx::smem_u32(&bars[slot]);
      ptx::mbar_arrive_expect_tx(bar, rbytes * PJT_KS);
      for (int u = 0; u < PJT_KS; ++u)
        ptx::bulk_load(ptx::smem_u32(ss + ((size_t)slot * PJT_KS + u) * PJT_ROWS),
                       S + (long long)(k0 + st * PJT_KS + u) * P + p_tile, rbytes, bar);
    };
    if (t == 0)
      for (int st = 0; st < min(ns, PJT_ST); ++st) issue(st);
    __syncthreads();   // X staged
    for (int st = 0; st < ns; ++st) {
      const int gi = g + st, slot = gi % PJT_ST;
      const bool landed = ptx::mbar_wait(ptx::smem_u32(&bars[slot]), (gi / PJT_ST) & 1, err);
      if (landed) {
        const float* sb = ss + (size_t)slot * PJT_KS * PJT_ROWS;
        const float* xb = xs + (size_t)st * PJT_KS * 32 + cg * 8;
#pragma unroll
        for (int u = 0; u < PJT_KS; ++u) {
          const float4 a = *reinterpret_cast<const float4*>(sb + u * PJT_ROWS + 4 * rg);
          const float4 b = *reinterpret_cast<const float4*>(sb + u * PJT_ROWS + 256 + 4 * rg);
          const float4 x4 = *reinterpret_cast<const float4*>(xb + u * 32);
          const float xv[5] = {x4.x, x4.y, x4.z, x4.w, xb[u * 32 + 4]};
          const float2 sp[4] = {make_float2(a.x, a.y), make_float2(a.z, a.w),
                                make_float2(b.x, b.y), make_float2(b.z, b.w)};
#pragma unroll
          for (int c = 0; c < 5; ++c) {
            const float2 xx = make_float2(xv[c], xv[c]);
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[r][c] = __ffma2_rn(sp[r], xx, acc[r][c]);
          }
        }
      }
      // every thread is done with the slot; a copy that never landed ends the block
      if (__syncthreads_or(!landed)) return;
      if (t == 0 && st + PJT_ST < ns) issue(st + PJT_ST);
    }
    g += ns;
  }
  float* out = part + (long long)blockIdx.y * l * P + p_tile;
#pragma unroll
  for (int c = 0; c < 5; ++c) {
    const int col = cg * 5 + c;
    if (col >= l) break;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int row = h * 256 + 4 * rg;
      if (row < nrows)
        *reinterpret_cast<float4*>(out + (long long)col * P + row) =
            make_float4(acc[2 * h][c].x, acc[2 * h][c].y, acc[2 * h + 1][c].x, acc[2 * h + 1][c].y);
    }
  }
}

// Launch shape of k_proj / k_proj_tma: rows per thread and the k ranges, chosen so
// that the grid is about two blocks per SM (the kernels' residency).
struct ProjShape {
  int rpt, lm, tiles, kb, kc, ranges;
  bool tma;   // k_proj_tma (8 < l <= 20, P a multiple of 8)
};

inline ProjShape proj_shape(int P, int l, int num_sms) {
  ProjShape s;
  s.lm = l <= 8 ? 8 : l <= 20 ? 20 : l <= 24 ? 24 : 64;
  s.tma = l > 8 && l <= 20 && P % PJT_KS == 0;
  s.rpt = l <= 8 ? 4 : l <= 24 ? 2 : 1;
  const int rows = PJ_WARPS * 32 * s.rpt;
  s.tiles = (P + rows - 1) / rows;
  const int want = max(1, (2 * max(num_sms, 1) + s.tiles / 2) / s.tiles);
  constexpr int q = 2 * PJ_U;
  s.kb = ((P + want - 1) / want + q - 1) / q * q;
  s.ranges = (P + s.kb - 1) / s.kb;
  s.kc = s.tma ? min(s.kb, PJT_KC) : min(s.kb, (32768 / (int)sizeof(float) / s.lm) / q * q);
  return s;
}

inline size_t proj_part_floats(int P, int l, int num_sms) {
  if (l > 64) return 0;
  const ProjShape sh = proj_shape(P, l, num_sms);
  return (size_t)sh.ranges * l * P;
}

// Partial Gram products A'B (l x l) over blocks of gram_rows() rows (A, B: P x l),
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
constexpr int GR_SUB = 32;

// Rows per block of the partial Gram products: about two blocks per SM (short
// per-entry chains, a wide grid), at least 16 rows.
inline int gram_rows(int P, int num_sms) {
  const int want = 2 * max(num_sms, 1);
  return max(16, ((P + want - 1) / want + 15) / 16 * 16);
}
inline size_t gram_part_doubles(int P, int l, int num_sms) {
  const int rows = gram_rows(P, num_sms);
  return (size_t)((P + rows - 1) / rows) * l * l;
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float z = s - a;
  e = (a - (s - z)) + (b - z);
}

template <typename TX>
__global__ void __launch_bounds__(256)
    k_cross_gram(int P, int l, int rows, const TX* __restrict__ A, const TX* __restrict__ B,
                 double* __restrict__ part) {
  __shared__ TX As[GR_SUB * 64], Bs[GR_SUB * 64];
  const int r0 = blockIdx.x * rows, r1 = min(P, r0 + rows);
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
  const int rows = gram_rows(P, ctx->num_sms);
  const int nb = (P + rows - 1) / rows;
  k_cross_gram<TX><<<nb, 256, 0, ctx->stream>>>(P, l, rows, A, B, part);
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

// Upper Cholesky G = R'R and R^-1 in float-float (l <= 64), one block,
// everything in shared memory.  Float-float rather than
// FP64: FP64 operations have long latency on this GPU and both factorisations
// are serial chains of l steps (the Gram matrix factored here is itself
// accurate to about 1e-14, from the compensated Gram kernel).  Every thread
// owns fixed entries of the l x l arrays and each step costs one barrier:
//   Cholesky, right-looking: at step j the owner of (i, k), j < i <= k,
//   subtracts R_ji R_jk = (G_ji y)(G_jk y), y = 1/sqrt(G_jj), each thread forming
//   y from the pivot itself.  Row j is final after step j - 1 and read unscaled;
//   the rows are scaled into R after the last step.
//   Inverse, by rows from the bottom: at step i the owner of (k, c), k < i <= c,
//   adds R_ki x_ic, x_ic = (delta_ic - a_ic) / R_ii formed from row i of the sums
//   (final after step i + 1); row i of R^-1 is x_i. (a starts at 0.)
// Output: R^-1 (l x l row-major, upper triangular) as hi parts Ih and lo parts
// Il.  Rank-deficient directions (pivot <= 1e-13 of the largest diagonal) get a
// zero row and column.
// OWN entries per thread: 1 (l <= 32, l^2 threads rounded up to a warp) or 4
// (l <= 64, 1024 threads); a fixed count keeps the owned entries in registers
// without predicated copies of the update for entries that do not exist.
inline size_t chol_ff_smem(int l) { return sizeof(float) * (4 * (size_t)l * (l + 1) + 2 * l + 1); }
inline int chol_ff_threads(int l) { return l <= 32 ? (l * l + 31) / 32 * 32 : 1024; }

template <int OWN>
__global__ void __launch_bounds__(1024) k_chol_ff(int l, const double* __restrict__ G,
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
  const int t = threadIdx.x, nt = blockDim.x;
  int oi[OWN], ok[OWN];   // owned entries (row, column); -1: none
#pragma unroll
  for (int r = 0; r < OWN; ++r) {
    const int e = t + r * nt;
    oi[r] = -1;
    ok[r] = 0;
    if (e < l * l) {
      oi[r] = e / l;
      ok[r] = e - oi[r] * l;
      const ff::F2 g = ff_of(G[e]);
      Gh[oi[r] * ld + ok[r]] = g.hi;
      Gl[oi[r] * ld + ok[r]] = g.lo;
      Ah[oi[r] * ld + ok[r]] = 0.f;
      Al[oi[r] * ld + ok[r]] = 0.f;
    }
  }
  __syncthreads();
  if (t < 32) {
    float dm = 0.f;
    for (int i = t; i < l; i += 32) dm = fmaxf(dm, Gh[i * ld + i]);
    for (int o = 16; o > 0; o >>= 1) dm = fmaxf(dm, __shfl_xor_sync(0xffffffffu, dm, o));
    if (t == 0) *dmax_s = dm;
  }
  __syncthreads();
  const float thr = 1e-13f * *dmax_s;
#pragma unroll 1
  for (int j = 0; j < l; ++j) {
    const ff::F2 piv = {Gh[j * ld + j], Gl[j * ld + j]};
    const ff::F2 y = piv.hi > thr ? rsqrt_ff(piv) : ff::make(0.f);
#pragma unroll
    for (int r = 0; r < OWN; ++r) {
      const int i = oi[r], k = ok[r];
      if (i > j && k >= i) {
        const ff::F2 rji = ff::mul(ff::F2{Gh[j * ld + i], Gl[j * ld + i]}, y);
        const ff::F2 rjk = ff::mul(ff::F2{Gh[j * ld + k], Gl[j * ld + k]}, y);
        const ff::F2 g = ff::sub_mul(ff::F2{Gh[i * ld + k], Gl[i * ld + k]}, rji, rjk);
        Gh[i * ld + k] = g.hi;
        Gl[i * ld + k] = g.lo;
      }
    }
    __syncthreads();
  }
  // 1 / R_jj from the final pivots, then the rows of R
  for (int jj = t; jj < l; jj += nt) {
    const ff::F2 piv = {Gh[jj * ld + jj], Gl[jj * ld + jj]};
    const ff::F2 y = piv.hi > thr ? rsqrt_ff(piv) : ff::make(0.f);
    yh[jj] = y.hi;
    yl[jj] = y.lo;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < OWN; ++r) {
    const int i = oi[r], k = ok[r];
    if (i >= 0 && k >= i) {
      const ff::F2 rr = ff::mul(ff::F2{Gh[i * ld + k], Gl[i * ld + k]}, ff::F2{yh[i], yl[i]});
      Gh[i * ld + k] = rr.hi;
      Gl[i * ld + k] = rr.lo;
    }
  }
  __syncthreads();
  // R^-1 by rows from the bottom
#pragma unroll 1
  for (int i = l - 1; i > 0; --i) {
    const ff::F2 d = {yh[i], yl[i]};
#pragma unroll
    for (int r = 0; r < OWN; ++r) {
      const int k = oi[r], c = ok[r];
      if (k >= 0 && k < i && c >= i) {
        const ff::F2 x = ff::mul(
            ff::add(ff::make(c == i ? 1.f : 0.f), ff::neg(ff::F2{Ah[i * ld + c], Al[i * ld + c]})), d);
        const ff::F2 a = ff::add(ff::F2{Ah[k * ld + c], Al[k * ld + c]},
                                 ff::mul(ff::F2{Gh[k * ld + i], Gl[k * ld + i]}, x));
        Ah[k * ld + c] = a.hi;
        Al[k * ld + c] = a.lo;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < OWN; ++r) {
    const int i = oi[r], c = ok[r];
    if (i >= 0) {
      ff::F2 x = ff::make(0.f);
      if (c >= i)
        x = ff::mul(ff::add(ff::make(c == i ? 1.f : 0.f), ff::neg(ff::F2{Ah[i * ld + c], Al[i * ld + c]})),
                    ff::F2{yh[i], yl[i]});
      Ih[i * l + c] = x.hi;
      Il[i * l + c] = x.lo;
    }
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

// Pair (p, q), p < q, of position i (0 <= i < ne / 2) at step `step` of a sweep of
// the round-robin (circle) schedule: ne / 2 disjoint pairs per step, ne - 1 steps
// (ne even; q == n marks the dummy of odd n).
__device__ __forceinline__ void rr_pair(int ne, int step, int i, int& p, int& q) {
  const int m = ne - 1;
  if (i == 0) {
    p = m;
    q = step;
  } else {
    p = step + i;
    if (p >= m) p -= m;
    q = step - i;
    if (q < 0) q += m;
  }
  if (p > q) {
    const int t = p;
    p = q;
    q = t;
  }
}

// The rotation (c, s) that annihilates a_pq: tau = (a_qq - a_pp) / (2 a_pq),
// t = sign(tau) / (|tau| + sqrt(1 + tau^2)), c = 1 / sqrt(1 + t^2), s = t c.
// The quotients and 1 / sqrt(1 + t^2) (argument in [1, 2]) use the fast
// approximate forms: c^2 + s^2 = 1 then holds to a few FP32 ulps, and the
// refinement that follows the FP32 Jacobi restores orthogonality anyway.  The
// square root of 1 + tau^2 stays exact so that tau^2 = inf still gives t = 0.
__device__ __forceinline__ void rr_rot(const float* A, int ld, int n, int p, int q, float& c,
                                       float& sn) {
  c = 1.f;
  sn = 0.f;
  if (q >= n) return;
  const float apq = A[p * ld + q], app = A[p * ld + p], aqq = A[q * ld + q];
  if (fabsf(apq) > 1e-30f && fabsf(apq) > 1e-18f * sqrtf(fabsf(app) * fabsf(aqq))) {
    const float tau = __fdividef(aqq - app, 2.f * apq);
    const float t = __fdividef(tau >= 0.f ? 1.f : -1.f, fabsf(tau) + sqrtf(1.f + tau * tau));
    c = rsqrtf(1.f + t * t);
    sn = t * c;
  }
}

// Cyclic parallel Jacobi in FP32 on the n x n matrix in Acur (ld = n + 1), V
// accumulating the rotations, until off(A)^2 <= tol diag(A)^2 or max_sweeps.
// Every step applies ne / 2 disjoint rotations as one two-sided update:
// each work item owns either a 2 x 2 block (rows of pair bi, columns of pair
// bj) of A, read from Acur and written to Anext after both rotations, or the
// two entries of one row k of V in the columns of pair bj (updated in place).
// With one item per thread each item forms the rotations it needs from Acur
// itself, so a step costs one barrier; with several items per thread the
// rotations are formed once into cs (np pairs) behind a second barrier.
// Returns the buffer that holds the final A.
// ITEMS work items per thread: (np^2 + n np) <= ITEMS * blockDim.x; 1 up to 1024
// items (n <= 36), else 3 (n <= 64).
template <int ITEMS>
__device__ float* rr_jacobi_f32(int n, float* Acur, float* Anext, float* V, int max_sweeps,
                                float tol, float* red, float* cs, int* done) {
  const int ld = n + 1;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int ne = (n + 1) & ~1, np = ne / 2;
  const int nblk = np * np, nitems = nblk + n * np;
  int ia[ITEMS], ib[ITEMS];   // block (bi, bj), or V row k (ia = -1 - k) and pair bj
#pragma unroll
  for (int r = 0; r < ITEMS; ++r) {
    const int w = tid + r * nt;
    ia[r] = -(1 << 30);
    ib[r] = 0;
    if (w < nblk) {
      ia[r] = w / np;
      ib[r] = w - ia[r] * np;
    } else if (w < nitems) {
      const int v = w - nblk;
      const int k = v / np;
      ia[r] = -1 - k;
      ib[r] = v - k * np;
    }
  }
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    float off = 0.f, dia = 0.f;
    for (int e = tid; e < n * n; e += nt) {
      const int r = e / n, c = e - r * n;
      const float a = Acur[r * ld + c];
      if (r == c) dia += a * a;
      else off += a * a;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      dia += __shfl_xor_sync(0xffffffffu, dia, o);
    }
    if ((tid & 31) == 0) {
      red[2 * (tid >> 5)] = off;
      red[2 * (tid >> 5) + 1] = dia;
    }
    __syncthreads();
    if (tid == 0) {
      float ot = 0.f, dt = 0.f;
      for (int w = 0; w < (nt + 31) / 32; ++w) {
        ot += red[2 * w];
        dt += red[2 * w + 1];
      }
      *done = (ot <= tol * dt) || ot == 0.f;
    }
    __syncthreads();
    if (*done) break;
    for (int step = 0; step < ne - 1; ++step) {
      if constexpr (ITEMS > 1) {
        // several items per thread: the np rotations once, then the updates
        for (int i = tid; i < np; i += nt) {
          int p, q;
          rr_pair(ne, step, i, p, q);
          rr_rot(Acur, ld, n, p, q, cs[2 * i], cs[2 * i + 1]);
        }
        __syncthreads();
      }
#pragma unroll
      for (int r = 0; r < ITEMS; ++r) {
        if (ia[r] == -(1 << 30)) continue;
        int pj, qj;
        float cj, sj;
        rr_pair(ne, step, ib[r], pj, qj);
        if constexpr (ITEMS > 1) {
          cj = cs[2 * ib[r]];
          sj = cs[2 * ib[r] + 1];
        } else {
          rr_rot(Acur, ld, n, pj, qj, cj, sj);
        }
        if (ia[r] >= 0) {
          int pi, qi;
          float ci, si;
          rr_pair(ne, step, ia[r], pi, qi);
          if constexpr (ITEMS > 1) {
            ci = cs[2 * ia[r]];
            si = cs[2 * ia[r] + 1];
          } else {
            rr_rot(Acur, ld, n, pi, qi, ci, si);
          }
          // columns (pj, qj) first, then rows (pi, qi); index n is the dummy
          const bool qiv = qi < n, qjv = qj < n;
          const float m00 = Acur[pi * ld + pj];
          const float m01 = qjv ? Acur[pi * ld + qj] : 0.f;
          const float m10 = qiv ? Acur[qi * ld + pj] : 0.f;
          const float m11 = (qiv && qjv) ? Acur[qi * ld + qj] : 0.f;
          const float c00 = cj * m00 - sj * m01, c01 = sj * m00 + cj * m01;
          const float c10 = cj * m10 - sj * m11, c11 = sj * m10 + cj * m11;
          Anext[pi * ld + pj] = ci * c00 - si * c10;
          if (qjv) Anext[pi * ld + qj] = ci * c01 - si * c11;
          if (qiv) Anext[qi * ld + pj] = si * c00 + ci * c10;
          if (qiv && qjv) Anext[qi * ld + qj] = si * c01 + ci * c11;
        } else {
          const int k = -1 - ia[r];
          if (qj < n) {
            const float vp = V[k * ld + pj], vq = V[k * ld + qj];
            V[k * ld + pj] = cj * vp - sj * vq;
            V[k * ld + qj] = sj * vp + cj * vq;
          }
        }
      }
      __syncthreads();
      float* t = Acur;
      Acur = Anext;
      Anext = t;
    }
  }
  return Acur;
}

// Symmetric eigendecomposition of the n x n (n <= 64) Rayleigh-Ritz matrix with an
// accurate result at a fraction of the FP64 work (FP64 is slow on this GPU):
//  1. cyclic Jacobi in FP32 on (A + A')/2 (off-diagonal to 3e-5 of the diagonal, at
//     most 10 sweeps: FP32 rounding stalls it near 1e-7), one block;
//  2. two steps of the iterative refinement of Ogita and Aishima ("Iterative
//     refinement for symmetric eigenvalue decomposition", 2018) on the FP32
//     eigenvectors X:  R = I - X'X,  S = X'AX,  lambda_i = s_ii / (1 - r_ii),
//     E_ij = (s_ij + lambda_j r_ij) / (lambda_j - lambda_i) for separated pairs and
//     r_ij / 2 inside clusters (gap <= delta = 2(|S - diag S| + |A| |R|), Frobenius
//     norms), X <- X + X E.  Each step squares the error.  For n <= 32 both steps
//     run in one block in float-float (k_rr_refine); beyond, in FP64 as separate
//     launches spread over n blocks.
// Outputs: A <- diag(lambda), V <- eigenvectors (columns, FP64).
inline size_t rr_jacobi32_smem(int n) { return sizeof(float) * 3 * (size_t)n * (n + 1); }

template <int ITEMS>
__global__ void __launch_bounds__(1024)
    k_rr_jacobi32(int n, double* __restrict__ Ag, double* __restrict__ Asym,
                  double* __restrict__ X) {
  extern __shared__ float rjs[];
  __shared__ float red[64];
  __shared__ float cs[64];   // (c, s) of each pair (ITEMS > 1)
  __shared__ int done;
  const int ld = n + 1;
  float* A0 = rjs;
  float* A1 = A0 + n * ld;
  float* V32 = A1 + n * ld;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < n * n; e += nt) {
    const int i = e / n, j = e - (e / n) * n;
    const double a = 0.5 * (Ag[e] + Ag[j * n + i]);
    Asym[e] = a;
    A0[i * ld + j] = (float)a;
    V32[i * ld + j] = (i == j) ? 1.f : 0.f;
  }
  __syncthreads();
  rr_jacobi_f32<ITEMS>(n, A0, A1, V32, 10, 1e-9f, red, cs, &done);
  for (int e = tid; e < n * n; e += nt) X[e] = (double)V32[(e / n) * ld + e % n];
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

// psi_j = Q u_{order[j]} (Q: P x l of type TX, U: l x l FP64), j < k: one
// thread per entry (j, r), its l-term FP64 sum in three interleaved chains
// (dependent FP64 operations have long latency on this GPU).
template <typename TX>
__global__ void k_ritz_vectors(int P, int l, int k, const TX* __restrict__ Q,
                               const double* __restrict__ U, const int* __restrict__ order,
                               double* __restrict__ psi) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;   // j * P + r
  if (e >= (long long)P * k) return;
  const int j = (int)(e / P), r = (int)(e - (long long)j * P);
  const int col = order[j];
  const TX* q = Q + (long long)r * l;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  int i = 0;
  for (; i + 3 <= l; i += 3) {
    s0 = fma((double)q[i], U[(long long)i * l + col], s0);
    s1 = fma((double)q[i + 1], U[(long long)(i + 1) * l + col], s1);
    s2 = fma((double)q[i + 2], U[(long long)(i + 2) * l + col], s2);
  }
  for (; i < l; ++i) s0 = fma((double)q[i], U[(long long)i * l + col], s0);
  psi[e] = (s0 + s1) + s2;
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
// phi = psi / sqrt(dV) (inv_sqrt_dv = 1 / sqrt(dV) from the host), lambda = theta
// dV, FVE = cumulative theta / trace.  One block per eigenvector.  The magnitudes
// are compared through their bit patterns (non-negative doubles order as their
// 64-bit integers), keyed with the index so that ties take the first entry.
__device__ __forceinline__ unsigned long long fin_better(unsigned long long a, int ia,
                                                         unsigned long long b, int ib) {
  return (b > a || (b == a && ib < ia)) ? 1ull : 0ull;
}

__global__ void __launch_bounds__(1024)
    k_finish(int P, int n, int k, double dv, double inv_sqrt_dv, const double* __restrict__ Aeig,
             const int* __restrict__ order, const double* __restrict__ trace,
             double* __restrict__ evals, double* __restrict__ evecs, double* __restrict__ fve) {
  const int j = blockIdx.x;
  double* v = evecs + (long long)j * P;
  __shared__ unsigned long long wb[32];
  __shared__ int wi[32];
  __shared__ double sgn;
  unsigned long long best = 0;
  int bidx = 0x7fffffff;
  for (int r = threadIdx.x; r < P; r += blockDim.x) {
    const unsigned long long a = (unsigned long long)__double_as_longlong(v[r]) & 0x7fffffffffffffffull;
    if (bidx == 0x7fffffff || fin_better(best, bidx, a, r)) {
      best = a;
      bidx = r;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
    if (oi != 0x7fffffff && (bidx == 0x7fffffff || fin_better(best, bidx, ob, oi))) {
      best = ob;
      bidx = oi;
    }
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  if (lane == 0) {
    wb[w] = best;
    wi[w] = bidx;
  }
  __syncthreads();
  if (w == 0) {
    best = lane < nw ? wb[lane] : 0ull;
    bidx = lane < nw ? wi[lane] : 0x7fffffff;
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
      if (oi != 0x7fffffff && (bidx == 0x7fffffff || fin_better(best, bidx, ob, oi))) {
        best = ob;
        bidx = oi;
      }
    }
    if (lane == 0) sgn = (bidx != 0x7fffffff && v[bidx] < 0.0) ? -inv_sqrt_dv : inv_sqrt_dv;
  }
  __syncthreads();
  const double scale = sgn;
  for (int r = threadIdx.x; r < P; r += blockDim.x) v[r] *= scale;
  if (threadIdx.x == 0) {
    const double th = Aeig[(long long)order[j] * n + order[j]];
    evals[j] = th * dv;
    if (fve) {
      double cum = 0.0;
      for (int i = 0; i <= j; ++i) cum += Aeig[(long long)order[i] * n + order[i]];
      fve[j] = cum / trace[0];
    }
  }
}

// Both Ogita-Aishima refinement steps of k_rr_jacobi32's eigenvectors in one block
// (n <= 32), in float-float with every n x n matrix in shared memory: per step
// R = I - X'X, U = A X, S = X'U, lambda_i = s_ii / (1 - r_ii),
// delta = 2 (|S - diag S| + |A| |R|), E_ij = (s_ij + lambda_j r_ij) / (lambda_j - lambda_i)
// or r_ij / 2 inside clusters, X <- X + X E; then A <- diag(lambda), V <- X.
// Float-float (about 2^-48) rather than FP64: the products are short serial
// chains, and dependent FP64 operations have long latency on this GPU; the
// result is accurate to about 1e-14, well below what the FP32 Sigma of the
// projection resolves.  The cluster threshold delta only needs FP32.
// Each product entry is split into two half-length dot products (neighbouring
// threads) joined by a shuffle.
constexpr int RF_THREADS = 1024;

struct FFMat {
  float* h;
  float* l;
  __device__ ff::F2 at(int e) const { return {h[e], l[e]}; }
  __device__ void put(int e, ff::F2 v) const {
    h[e] = v.hi;
    l[e] = v.lo;
  }
};

// C = diag I + sign op(L) M, op(L) = L' when tl
__device__ __forceinline__ void rf_product(int n, FFMat L, bool tl, FFMat M, FFMat C, float diag,
                                           float sign) {
  const int hn = (n + 1) / 2;
  const int ne2 = 2 * n * n;
  for (int base = 0; base < ne2; base += RF_THREADS) {
    const int e = base + threadIdx.x;
    const int o = e >> 1, part = e & 1;
    ff::F2 acc = ff::make(0.f);
    int i = 0, j = 0;
    if (e < ne2) {
      i = o / n;
      j = o - i * n;
      const int k0 = part * hn, k1 = min(n, k0 + hn);
#pragma unroll 4
      for (int k = k0; k < k1; ++k)
        acc = ff::add(acc, ff::mul(L.at(tl ? k * n + i : i * n + k), M.at(k * n + j)));
    }
    const float oh = __shfl_xor_sync(0xffffffffu, acc.hi, 1);
    const float ol = __shfl_xor_sync(0xffffffffu, acc.lo, 1);
    if (e < ne2 && part == 0) {
      ff::F2 v = ff::add(acc, ff::F2{oh, ol});
      if (sign < 0.f) v = ff::neg(v);
      if (i == j) v = ff::add(v, ff::make(diag));
      C.put(o, v);
    }
  }
  __syncthreads();
}

__device__ __forceinline__ float rf_block_sum(float v, float* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    float x = red[lane];  // RF_THREADS / 32 == 32 partials
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) red[32] = x;
  }
  __syncthreads();
  const float r = red[32];
  __syncthreads();
  return r;
}

inline size_t rr_refine_smem(int n) { return sizeof(float) * (10 * (size_t)n * n + 2 * n + 33); }

__global__ void __launch_bounds__(RF_THREADS)
    k_rr_refine(int n, const double* __restrict__ Asym, const double* __restrict__ X0,
                double* __restrict__ Ag, double* __restrict__ Vg) {
  extern __shared__ float rfs[];
  const int nn = n * n;
  const FFMat A{rfs, rfs + nn}, X{rfs + 2 * nn, rfs + 3 * nn}, R{rfs + 4 * nn, rfs + 5 * nn},
      U{rfs + 6 * nn, rfs + 7 * nn}, S{rfs + 8 * nn, rfs + 9 * nn};
  const FFMat lam{rfs + 10 * nn, rfs + 10 * nn + n};
  float* red = rfs + 10 * nn + 2 * n;  // [33]
  const int t = threadIdx.x;
  float an = 0.f;
  for (int e = t; e < nn; e += RF_THREADS) {
    const double a = Asym[e], x = X0[e];
    const float ah = (float)a, xh = (float)x;
    A.put(e, {ah, (float)(a - (double)ah)});
    X.put(e, {xh, (float)(x - (double)xh)});
    an += ah * ah;
  }
  an = rf_block_sum(an, red);  // (its barriers also publish A and X)
  for (int step = 0; step < 2; ++step) {
    rf_product(n, X, true, X, R, 1.f, -1.f);  // R = I - X'X
    rf_product(n, A, false, X, U, 0.f, 1.f);  // U = A X
    rf_product(n, X, true, U, S, 0.f, 1.f);   // S = X'AX
    for (int i = t; i < n; i += RF_THREADS)
      lam.put(i, ff::mul(S.at(i * n + i), ff::recip(ff::add(ff::make(1.f), ff::neg(R.at(i * n + i))))));
    float so = 0.f, rn = 0.f;
    for (int e = t; e < nn; e += RF_THREADS) {
      if (e / n != e % n) so += S.h[e] * S.h[e];
      rn += R.h[e] * R.h[e];
    }
    so = rf_block_sum(so, red);  // (the barriers inside also publish lam)
    rn = rf_block_sum(rn, red);
    const float delta = 2.f * (sqrtf(so) + sqrtf(an) * sqrtf(rn));
    for (int e = t; e < nn; e += RF_THREADS) {  // E into U (dead once S is formed)
      const int i = e / n, j = e - i * n;
      const ff::F2 gap = ff::add(lam.at(j), ff::neg(lam.at(i)));
      ff::F2 E;
      if (i == j || fabsf(gap.hi) <= delta) {
        E = R.at(e);
        E.hi *= 0.5f;
        E.lo *= 0.5f;
      } else {
        E = ff::mul(ff::add(S.at(e), ff::mul(lam.at(j), R.at(e))), ff::recip(gap));
      }
      U.put(e, E);
    }
    __syncthreads();
    rf_product(n, X, false, U, S, 0.f, 1.f);  // S = X E
    for (int e = t; e < nn; e += RF_THREADS) X.put(e, ff::add(X.at(e), S.at(e)));
    __syncthreads();
  }
  for (int e = t; e < nn; e += RF_THREADS) {
    const int i = e / n, j = e - i * n;
    Ag[e] = (i == j) ? ff::to_double(lam.at(i)) : 0.0;
    Vg[e] = ff::to_double(X.at(e));
  }
}

// Rayleigh-Ritz eigensolver (FP32 Jacobi + two refinement steps: float-float for
// l <= 32, FP64 beyond); scratch holds 5 l^2 + l doubles.
fpca_status launch_jacobi_rr(fpca_ctx* ctx, int l, double* A, double* V, double* scratch) {
  const size_t nn = (size_t)l * l;
  double* As = scratch;   // symmetrised input
  double* X = As + nn;    // FP32 Jacobi eigenvectors, refined in place
  double* R = X + nn;
  double* U = R + nn;
  double* S = U + nn;
  double* lam = S + nn;
  double* E = U;  // U is dead once S is formed
  // one thread per work item of a step (np^2 blocks of A, l np pairs of V entries)
  const int np = ((l + 1) & ~1) / 2;
  const int items = np * np + l * np;
  const int jt = min(1024, max(64, ((items + 31) / 32) * 32));
  const size_t jsm = rr_jacobi32_smem(l);
  if (items <= 1024) {
    k_rr_jacobi32<1><<<1, jt, jsm, ctx->stream>>>(l, A, As, X);
  } else {
    if (jsm > 48 * 1024)
      cudaFuncSetAttribute(k_rr_jacobi32<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)jsm);
    k_rr_jacobi32<3><<<1, jt, jsm, ctx->stream>>>(l, A, As, X);
  }
  FPCA_LAUNCHED(ctx, "jacobi");
  if (l <= 32) {
    k_rr_refine<<<1, RF_THREADS, rr_refine_smem(l), ctx->stream>>>(l, As, X, A, V);
    FPCA_LAUNCHED(ctx, "rr_refine");
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

// ---------------------------------------------------------------------------
// Dense symmetric eigensolver (n <= 1024): block Jacobi in FP32, then the
// Ogita-Aishima refinement in FP64.
// ---------------------------------------------------------------------------
// A one-block cyclic Jacobi keeps every rotation step of an n x n matrix on one
// SM, and one SM's FP64 rate and its round trips to memory make that take
// hundreds of milliseconds at n = 256.  The two-sided block Jacobi method spreads
// it: the indices are cut into blocks of BJ_S, and each round pairs the blocks
// (round-robin, nb - 1 rounds per sweep); per pair (I, J) one CTA diagonalises the
// 2 BJ_S x 2 BJ_S subproblem A[I u J, I u J] in shared memory (rr_jacobi_f32, a few
// sweeps) into an orthogonal J_IJ; then A <- J' A J (a J_a' A[P_a, P_b] J_b product
// per pair of pairs) and V <- V J spread over the whole GPU.  All of it in FP32;
// the eigenvectors X = V then go through the FP64 refinement steps of Ogita and
// Aishima (as launch_jacobi_rr), each of which squares the error, on the original
// FP64 matrix.  n is padded to a multiple of 2 BJ_S with zero rows and columns,
// which no rotation mixes with the real indices (their coupling is exactly zero).
constexpr int BJ_S = 16;
constexpr int BJ_W = 2 * BJ_S;  // subproblem width
constexpr int BJ_SWEEPS = 12;   // sweeps at most (each ends with the convergence test)
// The FP32 sweeps stop once the off-diagonal mass is at most this fraction of the
// diagonal mass (off-diagonal norm 1e-4 of the diagonal's; FP32 round-off alone
// leaves about (n eps)^2 ~ 4e-9 at n = 1024); the three FP64 refinement steps take
// the eigenvectors from there (each squares the error: 1e-4 -> 1e-8 -> 1e-16).
constexpr double BJ_TOL = 1e-8;

inline int bj_ne(int n) { return (n + BJ_W - 1) / BJ_W * BJ_W; }

// local index i of the subproblem of pair (I, J) -> global index
__device__ __forceinline__ int bj_index(int I, int J, int i) {
  return i < BJ_S ? I * BJ_S + i : J * BJ_S + (i - BJ_S);
}

__global__ void k_bj_init(int n, int ne, const double* __restrict__ A64, float* __restrict__ A,
                          float* __restrict__ V, int* __restrict__ done) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)ne * ne;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / ne), j = (int)(e - (long long)i * ne);
    A[e] = (i < n && j < n) ? (float)(0.5 * (A64[(long long)i * n + j] + A64[(long long)j * n + i])) : 0.f;
    V[e] = i == j ? 1.f : 0.f;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *done = 0;
}

// One CTA per block pair of the round: diagonalise the subproblem, write its
// rotation J (BJ_W x BJ_W, row-major) to Jg[pair].
__global__ void __launch_bounds__(1024)
    k_bj_sub(int ne, int round, const float* __restrict__ A, float* __restrict__ Jg,
             const int* __restrict__ done) {
  __shared__ float a0[BJ_W * (BJ_W + 1)], a1[BJ_W * (BJ_W + 1)], vs[BJ_W * (BJ_W + 1)];
  __shared__ float red[64], cs[64];
  __shared__ int sdone;
  if (*done) return;
  const int nb = ne / BJ_S;
  int I, J;
  rr_pair(nb, round, blockIdx.x, I, J);
  constexpr int ld = BJ_W + 1;
  for (int e = threadIdx.x; e < BJ_W * BJ_W; e += blockDim.x) {
    const int i = e / BJ_W, j = e - (e / BJ_W) * BJ_W;
    a0[i * ld + j] = A[(long long)bj_index(I, J, i) * ne + bj_index(I, J, j)];
    vs[i * ld + j] = i == j ? 1.f : 0.f;
  }
  __syncthreads();
  rr_jacobi_f32<1>(BJ_W, a0, a1, vs, 1, 1e-12f, red, cs, &sdone);
  __syncthreads();
  float* out = Jg + (size_t)blockIdx.x * BJ_W * BJ_W;
  for (int e = threadIdx.x; e < BJ_W * BJ_W; e += blockDim.x)
    out[e] = vs[(e / BJ_W) * ld + e % BJ_W];
}

// One launch per round applies the round's rotations:
//  blockIdx.y < npairs:  A[P_a, P_b] <- J_a' A[P_a, P_b] J_b (a = blockIdx.y, b = blockIdx.x);
//                        with mass != NULL the block adds the squared off-diagonal and
//                        diagonal entries of its new tile to mass[0], mass[1];
//  blockIdx.y >= npairs: V[rows, P_b] <- V[rows, P_b] J_b for BJ_W rows
//                        (row block blockIdx.y - npairs, pair b = blockIdx.x).
__global__ void __launch_bounds__(256)
    k_bj_apply(int ne, int round, float* __restrict__ A, float* __restrict__ V,
               const float* __restrict__ Jg, const int* __restrict__ done,
               double* __restrict__ mass) {
  __shared__ float ja[BJ_W][BJ_W + 1], jb[BJ_W][BJ_W + 1], m[BJ_W][BJ_W + 1], t[BJ_W][BJ_W + 1];
  __shared__ float red[8][2];
  if (*done) return;
  const int nb = ne / BJ_S, npairs = ne / BJ_W;
  int Ib, Jb;
  rr_pair(nb, round, blockIdx.x, Ib, Jb);
  const float* JB = Jg + (size_t)blockIdx.x * BJ_W * BJ_W;
  if ((int)blockIdx.y >= npairs) {
    const int r0 = (blockIdx.y - npairs) * BJ_W;
    for (int e = threadIdx.x; e < BJ_W * BJ_W; e += blockDim.x) {
      const int i = e / BJ_W, j = e - (e / BJ_W) * BJ_W;
      jb[i][j] = JB[e];
      m[i][j] = V[(long long)(r0 + i) * ne + bj_index(Ib, Jb, j)];
    }
    __syncthreads();
    for (int e = threadIdx.x; e < BJ_W * BJ_W; e += blockDim.x) {
      const int i = e / BJ_W, j = e - (e / BJ_W) * BJ_W;
      float s = 0.f;
#pragma unroll 8
      for (int k = 0; k < BJ_W; ++k) s = fmaf(m[i][k], jb[k][j], s);
      V[(long long)(r0 + i) * ne + bj_index(Ib, Jb, j)] = s;
    }
    return;
  }
  int Ia, Ja;
  rr_pair(nb, round, blockIdx.y, Ia, Ja);
  const float* JA = Jg + (size_t)blockIdx.y * BJ_W * BJ_W;
  for (int e = threadIdx.x; e < BJ_W * BJ_W; e += blockDim.x) {
    const int i = e / BJ_W, j = e - (e / BJ_W) * BJ_W;
    ja[i][j] = JA[e];
    jb[i][j] = JB[e];
    m[i][j] = A[(long long)bj_index(Ia, Ja, i) * ne + bj_index(Ib, Jb, j)];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < BJ_W * BJ_W; e += blockDim.x) {  // t = M J_b
    const int i = e / BJ_W, j = e - (e / BJ_W) * BJ_W;
    float s = 0.f;
#pragma unroll 8
    for (int k = 0; k < BJ_W; ++k) s = fmaf(m[i][k], jb[k][j], s);
    t[i][j] = s;
  }
  __syncthreads();
  float off = 0.f, dia = 0.f;
  for (int e = threadIdx.x; e < BJ_W * BJ_W; e += blockDim.x) {  // J_a' t
    const int i = e / BJ_W, j = e - (e / BJ_W) * BJ_W;
    float s = 0.f;
#pragma unroll 8
    for (int k = 0; k < BJ_W; ++k) s = fmaf(ja[k][i], t[k][j], s);
    const int gi = bj_index(Ia, Ja, i), gj = bj_index(Ib, Jb, j);
    A[(long long)gi * ne + gj] = s;
    if (gi == gj) dia += s * s;
    else off += s * s;
  }
  if (mass) {
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      dia += __shfl_xor_sync(0xffffffffu, dia, o);
    }
    if ((threadIdx.x & 31) == 0) {
      red[threadIdx.x >> 5][0] = off;
      red[threadIdx.x >> 5][1] = dia;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double so = 0.0, sd = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        so += red[w][0];
        sd += red[w][1];
      }
      atomicAdd(mass, so);
      atomicAdd(mass + 1, sd);
    }
  }
}

// V[rows, P_b] <- V[rows, P_b] J_b (the single-subproblem case): BJ_W rows
// (blockIdx.x) of pair b = blockIdx.y.
__global__ void __launch_bounds__(256)
    k_bj_apply_v(int ne, int round, float* __restrict__ V, const float* __restrict__ Jg,
                 const int* __restrict__ done) {
  __shared__ float jb[BJ_W][BJ_W + 1], m[BJ_W][BJ_W + 1];
  if (*done) return;
  const int nb = ne / BJ_S;
  int Ib, Jb;
  rr_pair(nb, round, blockIdx.y, Ib, Jb);
  const float* JB = Jg + (size_t)blockIdx.y * BJ_W * BJ_W;
  const int r0 = blockIdx.x * BJ_W;
  for (int e = threadIdx.x; e < BJ_W * BJ_W; e += blockDim.x) {
    const int i = e / BJ_W, j = e - (e / BJ_W) * BJ_W;
    jb[i][j] = JB[e];
    m[i][j] = V[(long long)(r0 + i) * ne + bj_index(Ib, Jb, j)];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < BJ_W * BJ_W; e += blockDim.x) {
    const int i = e / BJ_W, j = e - (e / BJ_W) * BJ_W;
    float s = 0.f;
#pragma unroll 8
    for (int k = 0; k < BJ_W; ++k) s = fmaf(m[i][k], jb[k][j], s);
    V[(long long)(r0 + i) * ne + bj_index(Ib, Jb, j)] = s;
  }
}

// done = 1 once the off-diagonal mass of the sweep's last round (mass[0], summed
// by k_bj_apply) is at most tol of the diagonal mass (mass[1]).
__global__ void k_bj_check(const double* __restrict__ mass, double tol, int* __restrict__ done) {
  if (threadIdx.x == 0 && (mass[0] <= tol * mass[1] || mass[0] == 0.0)) *done = 1;
}

// X (n x n, FP64) <- the leading n x n of V (ne x ne); As <- sym(A64).
__global__ void k_bj_extract(int n, int ne, const float* __restrict__ V, const double* __restrict__ A64,
                             double* __restrict__ X, double* __restrict__ As) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < (long long)n * n;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / n), j = (int)(e - (long long)i * n);
    X[e] = (double)V[(long long)i * ne + j];
    As[e] = 0.5 * (A64[e] + A64[(long long)j * n + i]);
  }
}

// Refinement pieces for n up to 1024 (one thread per column, lambda in global).
// Row i per block: lam[i] = S_ii / (1 - R_ii) and the squared norms of the
// off-diagonal of S, of A and of R added to acc[0..2] (zeroed by the caller).
__global__ void __launch_bounds__(256)
    k_oa_norms(int n, const double* __restrict__ A, const double* __restrict__ R,
               const double* __restrict__ S, double* __restrict__ lam, double* __restrict__ acc) {
  __shared__ double red[8][3];
  const int i = blockIdx.x;
  const long long o = (long long)i * n;
  double so = 0.0, an = 0.0, rn = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double sv = S[o + j], av = A[o + j], rv = R[o + j];
    if (j != i) so += sv * sv;
    an += av * av;
    rn += rv * rv;
  }
  for (int k = 16; k > 0; k >>= 1) {
    so += __shfl_xor_sync(0xffffffffu, so, k);
    an += __shfl_xor_sync(0xffffffffu, an, k);
    rn += __shfl_xor_sync(0xffffffffu, rn, k);
  }
  if ((threadIdx.x & 31) == 0) {
    red[threadIdx.x >> 5][0] = so;
    red[threadIdx.x >> 5][1] = an;
    red[threadIdx.x >> 5][2] = rn;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0, c = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a += red[w][0];
      b += red[w][1];
      c += red[w][2];
    }
    atomicAdd(acc, a);
    atomicAdd(acc + 1, b);
    atomicAdd(acc + 2, c);
    lam[i] = S[o + i] / (1.0 - R[o + i]);
  }
}

// Row i per block of the correction E: eigenvalues closer than
// delta = 2 (||offdiag S|| + ||A|| ||R||) are treated as one cluster.
__global__ void __launch_bounds__(256)
    k_oa_correction(int n, const double* __restrict__ R, const double* __restrict__ S,
                    const double* __restrict__ lam, const double* __restrict__ acc,
                    double* __restrict__ E) {
  const int i = blockIdx.x;
  const long long o = (long long)i * n;
  const double delta = 2.0 * (sqrt(acc[0]) + sqrt(acc[1]) * sqrt(acc[2]));
  const double li = lam[i];
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const double gap = lam[j] - li;
    E[o + j] = (j == i || fabs(gap) <= delta) ? 0.5 * R[o + j] : (S[o + j] + lam[j] * R[o + j]) / gap;
  }
}

// X <- X + X E (row i per block; the row is staged before it is written).
__global__ void k_oa_update(int n, double* __restrict__ X, const double* __restrict__ E) {
  extern __shared__ double xrow[];
  const int i = blockIdx.x;
  for (int j = threadIdx.x; j < n; j += blockDim.x) xrow[j] = X[(long long)i * n + j];
  __syncthreads();
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    double s0 = xrow[j], s1 = 0.0;
    int k = 0;
    for (; k + 1 < n; k += 2) {   // two chains: dependent FP64 adds are slow here
      s0 += xrow[k] * E[(long long)k * n + j];
      s1 += xrow[k + 1] * E[(long long)(k + 1) * n + j];
    }
    if (k < n) s0 += xrow[k] * E[(long long)k * n + j];
    X[(long long)i * n + j] = s0 + s1;
  }
}

// Row i (block) of C = op(L) M (+ diag I): n up to 1024, two interleaved chains.
__global__ void k_oa_rowmm(int n, const double* __restrict__ L, int tl, const double* __restrict__ M,
                           double* __restrict__ C, double diag, double sign) {
  const int i = blockIdx.x;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    double s0 = 0.0, s1 = 0.0;
    int k = 0;
    for (; k + 1 < n; k += 2) {
      s0 += (tl ? L[(long long)k * n + i] : L[(long long)i * n + k]) * M[(long long)k * n + j];
      s1 += (tl ? L[(long long)(k + 1) * n + i] : L[(long long)i * n + k + 1]) *
            M[(long long)(k + 1) * n + j];
    }
    if (k < n) s0 += (tl ? L[(long long)k * n + i] : L[(long long)i * n + k]) * M[(long long)k * n + j];
    C[(long long)i * n + j] = ((i == j) ? diag : 0.0) + sign * (s0 + s1);
  }
}

inline size_t dense_eig_bytes(int n) {
  const int ne = bj_ne(n);
  const int npairs = ne / BJ_W;
  return WsCarve::round(sizeof(float) * (size_t)ne * ne) * 2 +
         WsCarve::round(sizeof(float) * (size_t)npairs * BJ_W * BJ_W) + WsCarve::round(64) +
         WsCarve::round(sizeof(double) * (2 * BJ_SWEEPS + 4)) +
         5 * WsCarve::round(sizeof(double) * (size_t)n * n) + WsCarve::round(sizeof(double) * n);
}

// Eigenpairs of the symmetric n x n FP64 matrix A (n <= 1024): A <- diag(lambda),
// V <- eigenvectors (columns), like launch_jacobi_rr.
fpca_status launch_dense_eig(fpca_ctx* ctx, int n, double* A, double* V, void* scratch) {
  const int ne = bj_ne(n), nb = ne / BJ_S, npairs = ne / BJ_W;
  WsCarve c(scratch);
  float* Af = c.take<float>((size_t)ne * ne);
  float* Vf = c.take<float>((size_t)ne * ne);
  float* Jg = c.take<float>((size_t)npairs * BJ_W * BJ_W);
  int* done = c.take<int>(16);
  double* mass = c.take<double>(2 * BJ_SWEEPS + 4);  // per sweep; the last 3: refinement norms
  const size_t nn = (size_t)n * n;
  double* As = c.take<double>(nn);
  double* X = c.take<double>(nn);
  double* R = c.take<double>(nn);
  double* U = c.take<double>(nn);
  double* S = c.take<double>(nn);
  double* lam = c.take<double>(n);
  double* E = U;  // U is dead once S is formed
  const int eb = (int)std::min<long long>(((long long)ne * ne + 255) / 256, 4096);
  k_bj_init<<<eb, 256, 0, ctx->stream>>>(n, ne, A, Af, Vf, done);
  FPCA_LAUNCHED(ctx, "eig_bj_init");
  cudaMemsetAsync(mass, 0, sizeof(double) * (2 * BJ_SWEEPS + 4), ctx->stream);
  if (nb > 1) {
    for (int sweep = 0; sweep < BJ_SWEEPS; ++sweep) {
      for (int r = 0; r < nb - 1; ++r) {
        k_bj_sub<<<npairs, 768, 0, ctx->stream>>>(ne, r, Af, Jg, done);
        FPCA_LAUNCHED(ctx, "eig_bj_sub");
        k_bj_apply<<<dim3(npairs, npairs + ne / BJ_W), 256, 0, ctx->stream>>>(
            ne, r, Af, Vf, Jg, done, r == nb - 2 ? mass + 2 * sweep : nullptr);
        FPCA_LAUNCHED(ctx, "eig_bj_apply");
      }
      k_bj_check<<<1, 32, 0, ctx->stream>>>(mass + 2 * sweep, BJ_TOL, done);
      FPCA_LAUNCHED(ctx, "eig_bj_check");
    }
  } else {
    // a single subproblem holds the whole (padded) matrix
    k_bj_sub<<<1, 768, 0, ctx->stream>>>(ne, 0, Af, Jg, done);
    FPCA_LAUNCHED(ctx, "eig_bj_sub");
    k_bj_apply_v<<<dim3(ne / BJ_W, 1), 256, 0, ctx->stream>>>(ne, 0, Vf, Jg, done);
    FPCA_LAUNCHED(ctx, "eig_bj_apply_v");
  }
  const int xb = (int)std::min<long long>(((long long)nn + 255) / 256, 4096);
  k_bj_extract<<<xb, 256, 0, ctx->stream>>>(n, ne, Vf, A, X, As);
  FPCA_LAUNCHED(ctx, "eig_bj_extract");
  const int tpb = std::min(1024, ((n + 31) / 32) * 32);
  for (int step = 0; step < 3; ++step) {
    k_oa_rowmm<<<n, tpb, 0, ctx->stream>>>(n, X, 1, X, R, 1.0, -1.0);   // R = I - X'X
    FPCA_LAUNCHED(ctx, "eig_oa_rowmm");
    k_oa_rowmm<<<n, tpb, 0, ctx->stream>>>(n, As, 0, X, U, 0.0, 1.0);   // U = A X
    FPCA_LAUNCHED(ctx, "eig_oa_rowmm");
    k_oa_rowmm<<<n, tpb, 0, ctx->stream>>>(n, X, 1, U, S, 0.0, 1.0);    // S = X' A X
    FPCA_LAUNCHED(ctx, "eig_oa_rowmm");
    double* acc = mass + 2 * BJ_SWEEPS + 1;
    cudaMemsetAsync(acc, 0, sizeof(double) * 3, ctx->stream);
    k_oa_norms<<<n, 256, 0, ctx->stream>>>(n, As, R, S, lam, acc);
    FPCA_LAUNCHED(ctx, "eig_oa_norms");
    k_oa_correction<<<n, 256, 0, ctx->stream>>>(n, R, S, lam, acc, E);
    FPCA_LAUNCHED(ctx, "eig_oa_correction");
    k_oa_update<<<n, tpb, sizeof(double) * n, ctx->stream>>>(n, X, E);
    FPCA_LAUNCHED(ctx, "eig_oa_update");
  }
  k_rr_out<<<xb, 256, 0, ctx->stream>>>(n, lam, X, A, V);
  FPCA_LAUNCHED(ctx, "eig_out");
  return FPCA_OK;
}

template <int LM, int RPT>
void proj_launch(fpca_ctx* ctx, const ProjShape& sh, int P, int l, const float* S,
                 const float* X, float* part) {
  const size_t smem = sizeof(float) * (size_t)sh.kc * LM;
  k_proj<LM, RPT><<<dim3(sh.tiles, sh.ranges), PJ_WARPS * 32, smem, ctx->stream>>>(
      P, l, sh.kb, sh.kc, S, X, part);
}

template <typename TS>
fpca_status launch_proj(fpca_ctx* ctx, int P, int l, const TS* S, const TS* X, TS* Y,
                        float* part) {
  if constexpr (sizeof(TS) != 4) {
    return fpca_fail(ctx, FPCA_E_UNSUPPORTED, "projection runs on FP32 Sigma");
  } else {
    if (l > 64) return fpca_fail(ctx, FPCA_E_UNSUPPORTED, "projection built for l <= 64");
    const ProjShape sh = proj_shape(P, l, ctx->num_sms);
    if (sh.tma) {
      const size_t smem = proj_tma_smem(sh.kc);
      cudaFuncSetAttribute(k_proj_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      k_proj_tma<<<dim3(sh.tiles, sh.ranges), 256, smem, ctx->stream>>>(P, l, sh.kb, sh.kc, S, X,
                                                                       part, ctx->d_err);
    } else if (sh.lm == 8) proj_launch<8, 4>(ctx, sh, P, l, S, X, part);
    else if (sh.lm == 20) proj_launch<20, 2>(ctx, sh, P, l, S, X, part);
    else if (sh.lm == 24) proj_launch<24, 2>(ctx, sh, P, l, S, X, part);
    else proj_launch<64, 1>(ctx, sh, P, l, S, X, part);
    FPCA_LAUNCHED(ctx, "proj");
    const long long n = (long long)P * l;
    k_proj_sum<<<(int)((n + 255) / 256), 256, 0, ctx->stream>>>(P, l, sh.ranges, part, Y);
    FPCA_LAUNCHED(ctx, "proj_sum");
    return FPCA_OK;
  }
}

// Orthonormal basis Q of range(Y) by Cholesky QR: passes = 2 (CholeskyQR2) for the
// basis of the Rayleigh-Ritz step; one pass between power iterations, where only
// a well-conditioned basis of the range is needed.  The first of two passes writes
// tmp (P x l) and the second reads it, so that k_apply_ff never overwrites the rows
// it is reading.
template <typename TS>
fpca_status orth_cqr2(fpca_ctx* ctx, int P, int l, TS* Y, TS* Q, TS* tmp, double* G,
                      double* Rinv, double* part, int passes = 2) {
  for (int pass = 0; pass < passes; ++pass) {
    TS* src = pass == 0 ? Y : tmp;
    TS* dst = pass == passes - 1 ? Q : tmp;
    fpca_status gs = launch_cross_gram<TS>(ctx, P, l, src, src, part, G, "gram");
    if (gs != FPCA_OK) return gs;
    // Rinv holds R^-1 as hi and lo parts (l <= 64)
    float* Ih = reinterpret_cast<float*>(Rinv);
    float* Il = Ih + l * l;
    if (l <= 32)
      k_chol_ff<1><<<1, chol_ff_threads(l), chol_ff_smem(l), ctx->stream>>>(l, G, Ih, Il);
    else {
      cudaFuncSetAttribute(k_chol_ff<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)chol_ff_smem(l));
      k_chol_ff<4><<<1, chol_ff_threads(l), chol_ff_smem(l), ctx->stream>>>(l, G, Ih, Il);
    }
    FPCA_LAUNCHED(ctx, "chol_inv");
    const long long ne = (long long)P * l;
    k_apply_ff<TS><<<(int)((ne + 255) / 256), 256, 0, ctx->stream>>>(P, l, src, Ih, Il, dst);
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
                      2 * WsCarve::round(sizeof(double) * (size_t)l * l) +
                      2 * WsCarve::round(sizeof(double) * (size_t)n * n) +
                      WsCarve::round(sizeof(double) * 2 * n) + WsCarve::round(sizeof(int) * 3 * n) +
                      WsCarve::round(sizeof(double) * gram_part_doubles(P, l, ctx->num_sms)) +
                      WsCarve::round(sizeof(double) * (5 * (size_t)l * l + l)) +
                      WsCarve::round(sizeof(float) * proj_part_floats(P, l, ctx->num_sms)) +
                      (full ? WsCarve::round(dense_eig_bytes(n)) : 0) + 4096;
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
  double* A = carve.take<double>((size_t)n * n);
  double* V = carve.take<double>((size_t)n * n);
  int* order = carve.take<int>(n);
  double* part = carve.take<double>(gram_part_doubles(P, l, ctx->num_sms));
  double* rrs = carve.take<double>(5 * (size_t)l * l + l);
  float* ppart = carve.take<float>(proj_part_floats(P, l, ctx->num_sms));
  char* dense = full ? carve.take<char>(dense_eig_bytes(n)) : nullptr;

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
    fpca_status ds = launch_dense_eig(ctx, P, A, V, dense);
    if (ds != FPCA_OK) return ds;
    k_eig_order<<<1, 1024, 0, ctx->stream>>>(P, A, order);
    FPCA_LAUNCHED(ctx, "eig_order");
    k_dense_vectors<<<(int)(((long long)P * k + 255) / 256), 256, 0, ctx->stream>>>(P, k, V, order,
                                                                                    evecs);
    FPCA_LAUNCHED(ctx, "dense_vectors");
    k_finish<<<k, 1024, 0, ctx->stream>>>(P, P, k, dv, 1.0 / std::sqrt(dv), A, order, trace,
                                          evals, evecs, fve);
    FPCA_LAUNCHED(ctx, "eig_finish");
    return FPCA_OK;
  }
  // Omega in the working type
  if constexpr (sizeof(TS) == 4) {
    cudaMemcpyAsync(Om, omega, sizeof(float) * (size_t)P * l, cudaMemcpyDeviceToDevice, ctx->stream);
  } else {
    return fpca_fail(ctx, FPCA_E_UNSUPPORTED, "random projection runs on FP32 Sigma");
  }
  fpca_status s = launch_proj<TS>(ctx, P, l, S, Om, Y, ppart);
  if (s != FPCA_OK) return s;
  for (int it = 0; it < power_iters; ++it) {
    s = orth_cqr2<TS>(ctx, P, l, Y, Q, Z, G, Rinv, part, 1);
    if (s != FPCA_OK) return s;
    s = launch_proj<TS>(ctx, P, l, S, Q, Y, ppart);
    if (s != FPCA_OK) return s;
  }
  s = orth_cqr2<TS>(ctx, P, l, Y, Q, Z, G, Rinv, part);
  if (s != FPCA_OK) return s;
  s = launch_proj<TS>(ctx, P, l, S, Q, Z, ppart);
  if (s != FPCA_OK) return s;
  s = launch_cross_gram<TS>(ctx, P, l, Q, Z, part, A, "ritz_gram");
  if (s != FPCA_OK) return s;
  {
    fpca_status js = launch_jacobi_rr(ctx, l, A, V, rrs);
    if (js != FPCA_OK) return js;
  }
  k_eig_order<<<1, 1024, 0, ctx->stream>>>(l, A, order);
  FPCA_LAUNCHED(ctx, "eig_order");
  k_ritz_vectors<TS><<<(int)(((long long)P * k + 255) / 256), 256, 0, ctx->stream>>>(
      P, l, k, Q, V, order, evecs);
  FPCA_LAUNCHED(ctx, "ritz_vectors");
  k_finish<<<k, 1024, 0, ctx->stream>>>(P, l, k, dv, 1.0 / std::sqrt(dv), A, order, trace, evals,
                                        evecs, fve);
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
size_t rproj_ws_bytes(const fpca_ctx* ctx, int P, int l) {
  return 3 * WsCarve::round(sizeof(float) * (size_t)P * l) +
         4 * WsCarve::round(sizeof(double) * (size_t)l * l) + WsCarve::round(sizeof(double) * 4) +
         WsCarve::round(sizeof(int) * 3 * (size_t)l) +
         WsCarve::round(sizeof(double) * gram_part_doubles(P, l, ctx->num_sms)) +
         WsCarve::round(sizeof(double) * (5 * (size_t)l * l + l)) + 2048;
}

void rproj_ws_carve(const fpca_ctx* ctx, WsCarve& c, int P, int l, RprojWs& w) {
  w.Y = c.take<float>((size_t)P * l);
  w.Q = c.take<float>((size_t)P * l);
  w.Z = c.take<float>((size_t)P * l);
  w.G = c.take<double>((size_t)l * l);
  w.Rinv = c.take<double>((size_t)l * l);
  w.A = c.take<double>((size_t)l * l);
  w.V = c.take<double>((size_t)l * l);
  w.trace = c.take<double>(4);
  w.order = c.take<int>(3 * (size_t)l);
  w.part = c.take<double>(gram_part_doubles(P, l, ctx->num_sms));
  w.rr = c.take<double>(5 * (size_t)l * l + l);
}

fpca_status rproj_operator(fpca_ctx* ctx, int P, int l, int k, int power_iters, double dv,
                           const float* omega, RprojOp op, const RprojWs& w, double* evals,
                           double* evecs, double* fve) {
  fpca_status s = op.apply(op.self, omega, w.Y);
  if (s != FPCA_OK) return s;
  for (int it = 0; it < power_iters; ++it) {
    s = orth_cqr2<float>(ctx, P, l, w.Y, w.Q, w.Z, w.G, w.Rinv, w.part, 1);
    if (s != FPCA_OK) return s;
    s = op.apply(op.self, w.Q, w.Y);
    if (s != FPCA_OK) return s;
  }
  s = orth_cqr2<float>(ctx, P, l, w.Y, w.Q, w.Z, w.G, w.Rinv, w.part);
  if (s != FPCA_OK) return s;
  s = op.apply(op.self, w.Q, w.Z);
  if (s != FPCA_OK) return s;
  s = launch_cross_gram<float>(ctx, P, l, w.Q, w.Z, w.part, w.A, "ritz_gram");
  if (s != FPCA_OK) return s;
  s = launch_jacobi_rr(ctx, l, w.A, w.V, w.rr);
  if (s != FPCA_OK) return s;
  k_eig_order<<<1, 1024, 0, ctx->stream>>>(l, w.A, w.order);
  FPCA_LAUNCHED(ctx, "eig_order");
  k_ritz_vectors<float><<<(int)(((long long)P * k + 255) / 256), 256, 0, ctx->stream>>>(
      P, l, k, w.Q, w.V, w.order, evecs);
  FPCA_LAUNCHED(ctx, "ritz_vectors");
  k_finish<<<k, 1024, 0, ctx->stream>>>(P, l, k, dv, 1.0 / std::sqrt(dv), w.A, w.order, w.trace,
                                        evals, evecs, fve);
  FPCA_LAUNCHED(ctx, "eig_finish");
  return FPCA_OK;
}
