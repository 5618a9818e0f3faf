// Binning (Section 3.2) of the sums in Eq. (2.3) and Eq. (2.4).
//
// Mean bins carry, per grid bin b: the observation count, W_b = sum 1/N_i and
// V_b = sum Y_ij / N_i (V2 with Y^2).  Covariance bins carry, per ordered
// bin pair (p, q): the pair count, W = sum w_i, V = sum w_i R_ij R_il with
// w_i = 1/(N_i (N_i - 1)), over pairs j != l of one subject.
#include <cuda_bf16.h>

#include "fpca_internal.cuh"
#include "ff.cuh"

namespace {

__device__ __forceinline__ double load_y(const void* y, int prec, size_t idx) {
  return prec == FPCA_F64 ? static_cast<const double*>(y)[idx]
                          : static_cast<double>(static_cast<const float*>(y)[idx]);
}

__device__ __forceinline__ int bin_index(const double* t, int d, const int* m) {
  int flat = 0;
  for (int k = 0; k < d; ++k) {
    double x = floor(__dmul_rn(t[k], (double)m[k]));
    int ik = (int)fmin(fmax(x, 0.0), (double)(m[k] - 1));
    flat = flat * m[k] + ik;
  }
  return flat;
}

// N_i: observed nodes of subject i (mask row sum), one warp per subject; rows
// are read 16 bytes at a time when they are 16-byte aligned.
__global__ void k_subject_counts(int n, int P, const uint8_t* __restrict__ mask,
                                 int32_t* __restrict__ Ni) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (i >= n) return;
  int c = 0;
  if (!mask) {
    c = lane == 0 ? P : 0;
  } else if (P % 16 == 0 && (reinterpret_cast<uintptr_t>(mask) & 15) == 0) {
    const uint4* row = reinterpret_cast<const uint4*>(mask + (size_t)i * P);
    for (int q = lane; q < P / 16; q += 32) {
      const uint4 v = row[q];
      const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int k = 0; k < 4; ++k)  // count the nonzero bytes of w[k]
        c += __popc(__vcmpne4(w[k], 0u)) >> 3;
    }
  } else {
    const uint8_t* row = mask + (size_t)i * P;
    for (int p = lane; p < P; p += 32) c += row[p] != 0;
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if (lane == 0) Ni[i] = c;
}

// Dense mean bins: a block covers 32 nodes; its MB_SLICES thread rows take
// every MB_SLICES-th subject, and the partial sums are added by a fixed
// pairwise tree (deterministic).  Weights 1/N_i.
constexpr int MB_SLICES = 32;  // subject slices per block: short FP64 add chains
constexpr int MB_BATCH = 8;    // subjects whose loads are issued together (4 for FP64 y)
template <typename TY>
__global__ void __launch_bounds__(32 * MB_SLICES)
    k_bin_mean_dense(int n, int P, const TY* __restrict__ y, const uint8_t* __restrict__ mask,
                     const int32_t* __restrict__ Ni, int32_t* __restrict__ cnt,
                     double* __restrict__ w, double* __restrict__ v, double* __restrict__ v2) {
  __shared__ double ps[3][MB_SLICES][32];
  __shared__ int pc[MB_SLICES][32];
  __shared__ float winvh[32 * MB_SLICES], winvl[32 * MB_SLICES];
  const int p = blockIdx.x * 32 + threadIdx.x;
  int c = 0;
  // per-thread sums in float-float (about 48 bits from FP32 operations: FP64
  // adds are long-latency and low-throughput on this GPU), joined in FP64 below
  ff::F2 fw = ff::make(0.f), fv = ff::make(0.f), fv2 = ff::make(0.f);
  const int tid = threadIdx.y * 32 + threadIdx.x;
  for (int i0 = 0; i0 < n; i0 += 32 * MB_SLICES) {
    // 1/N_i for the next 32 * MB_SLICES subjects, one division per subject
    __syncthreads();
    {
      const int i = i0 + tid;
      const int N = i < n ? Ni[i] : 0;
      const double wd = N > 0 ? 1.0 / (double)N : 0.0;
      const float hi = (float)wd;
      winvh[tid] = hi;
      winvl[tid] = (float)(wd - (double)hi);
    }
    __syncthreads();
    if (p < P) {
      const int iend = min(n, i0 + 32 * MB_SLICES);
      constexpr int NB = sizeof(TY) == 8 ? MB_BATCH / 2 : MB_BATCH;
      for (int ib = i0 + threadIdx.y; ib < iend; ib += NB * MB_SLICES) {
        // the batch's loads first (independent of the sums), then the sums in
        // subject order
        TY yb[NB];
        bool ok[NB];
#pragma unroll
        for (int u = 0; u < NB; ++u) {
          const int i = ib + u * MB_SLICES;
          const size_t idx = (size_t)i * P + p;
          ok[u] = i < iend && (!mask || mask[idx]);
          yb[u] = i < iend ? y[idx] : TY(0);
        }
#pragma unroll
        for (int u = 0; u < NB; ++u) {
          const int i = ib + u * MB_SLICES;
          if (!ok[u]) continue;
          const ff::F2 wi = {winvh[i - i0], winvl[i - i0]};
          if (wi.hi == 0.f) continue;
          ff::F2 yy, y2;
          if constexpr (sizeof(TY) == 8) {
            const double yd = yb[u];
            const float hi = (float)yd;
            yy = {hi, (float)(yd - (double)hi)};
            y2 = ff::mul(yy, yy);
          } else {
            const float yf = yb[u];
            yy = ff::make(yf);
            y2 = ff::two_prod(yf, yf);  // exact
          }
          c += 1;
          fw = ff::add(fw, wi);
          fv = ff::add(fv, ff::mul(wi, yy));
          fv2 = ff::add(fv2, ff::mul(wi, y2));
        }
      }
    }
  }
  const double sw = ff::to_double(fw), sv = ff::to_double(fv), sv2 = ff::to_double(fv2);
  ps[0][threadIdx.y][threadIdx.x] = sw;
  ps[1][threadIdx.y][threadIdx.x] = sv;
  ps[2][threadIdx.y][threadIdx.x] = sv2;
  pc[threadIdx.y][threadIdx.x] = c;
  __syncthreads();
  // pairwise tree over the slices (fixed order; FP64 adds have a long latency)
  for (int h = MB_SLICES / 2; h >= 1; h >>= 1) {
    if (threadIdx.y < h) {
      pc[threadIdx.y][threadIdx.x] += pc[threadIdx.y + h][threadIdx.x];
#pragma unroll
      for (int a = 0; a < 3; ++a) ps[a][threadIdx.y][threadIdx.x] += ps[a][threadIdx.y + h][threadIdx.x];
    }
    __syncthreads();
  }
  if (threadIdx.y == 0 && p < P) {
    cnt[p] = pc[0][threadIdx.x];
    w[p] = ps[0][0][threadIdx.x];
    v[p] = ps[1][0][threadIdx.x];
    if (v2) v2[p] = ps[2][0][threadIdx.x];
  }
}

// Sparse mean bins: one thread per subject, atomic scatter into the bins.
__global__ void k_bin_mean_sparse(int n, long long N, int d, int m0, int m1, int m2,
                                  const int64_t* __restrict__ offs, const double* __restrict__ t,
                                  const double* __restrict__ y, int32_t* cnt, double* w,
                                  double* v, double* v2, int* __restrict__ err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int m[3] = {m0, m1, m2};
  const int64_t lo = offs[i], hi = offs[i + 1];
  if (lo < 0 || hi < lo || hi > N) {
    atomicExch(err, DERR_BOUNDS);
    return;
  }
  if (hi == lo) return;
  const double wi = 1.0 / (double)(hi - lo);
  for (int64_t j = lo; j < hi; ++j) {
    const int b = bin_index(t + j * d, d, m);
    const double yy = y[j];
    atomicAdd(cnt + b, 1);
    atomicAdd(w + b, wi);
    atomicAdd(v + b, __dmul_rn(wi, yy));
    if (v2) atomicAdd(v2 + b, __dmul_rn(wi, __dmul_rn(yy, yy)));
  }
}

// Operand planes of the tensor-core Gram products, K-major (subject index
// contiguous), BF16, zero-padded to Kpad subjects:
//   plane 0: M_ip                 (pair counts  C = M'M)
//   plane 1: w_i M_ip             (W = (wM)'M, exact 0/1 right operand)
//   plane 2: sqrt(w_i) R_ip M_ip  (V = R~'R~)
// A tile of 64 subjects x 32 nodes is transposed through shared memory: the
// reads run along the nodes (y, mask), the writes along the subjects as BF16
// pairs (128 bytes per node and plane).
template <typename TY>
__global__ void __launch_bounds__(256)
    k_cov_operands_bf16(int n, int P, int Kpad, const TY* __restrict__ y,
                        const uint8_t* __restrict__ mask, const int32_t* __restrict__ Ni,
                        const double* __restrict__ mu, int mode, __nv_bfloat162* __restrict__ ops) {
  __shared__ float tw[64][33], tr[64][33];
  __shared__ uint8_t tm[64][36];
  __shared__ float wsub[64], swsub[64], muf[32];
  const int i0 = blockIdx.y * 64, p0 = blockIdx.x * 32;
  const int tid = threadIdx.y * 32 + threadIdx.x;
  // per-subject weights w_i = 1/(N_i (N_i - 1)) and sqrt(w_i), and the mean at the
  // block's 32 nodes, once per block and in FP32: the operands are rounded to
  // BF16, so FP32 is ample (and FP64 operations are slow on this GPU)
  if (tid < 64) {
    const int i = i0 + tid;
    const int N = i < n ? Ni[i] : 0;
    const float wi = N >= 2 ? 1.f / ((float)N * (float)(N - 1)) : 0.f;
    wsub[tid] = wi;
    swsub[tid] = sqrtf(wi);
  } else if (tid < 96) {
    const int p = p0 + tid - 64;
    muf[tid - 64] = (p < P && mode == FPCA_COV_RESIDUAL) ? (float)mu[p] : 0.f;
  }
  // this thread's 8 observations, loads first (mask and y together)
  TY yv[8];
  uint8_t ob[8];
  const int p = p0 + threadIdx.x;
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int i = i0 + threadIdx.y + 8 * u;
    const bool in = i < n && p < P;
    const size_t idx = (size_t)i * P + p;
    ob[u] = in ? (mask ? mask[idx] : (uint8_t)1) : (uint8_t)0;
    yv[u] = in ? y[idx] : TY(0);
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    const int r = threadIdx.y + 8 * u;
    const bool obs = ob[u] != 0;
    tm[r][threadIdx.x] = obs ? 1 : 0;
    tw[r][threadIdx.x] = obs ? wsub[r] : 0.f;
    tr[r][threadIdx.x] = obs ? swsub[r] * ((float)yv[u] - muf[threadIdx.x]) : 0.f;
  }
  __syncthreads();
  // node p0 + c, subjects i0 + 2 lane and i0 + 2 lane + 1
  const size_t plane = (size_t)P * Kpad / 2;   // in BF16 pairs
  for (int c = threadIdx.y; c < 32; c += 8) {
    const int pn = p0 + c;
    if (pn >= P) continue;
    const int a = 2 * threadIdx.x;
    const size_t o = ((size_t)pn * Kpad + i0) / 2 + threadIdx.x;
    ops[o] = __floats2bfloat162_rn((float)tm[a][c], (float)tm[a + 1][c]);
    ops[plane + o] = __floats2bfloat162_rn(tw[a][c], tw[a + 1][c]);
    ops[2 * plane + o] = __floats2bfloat162_rn(tr[a][c], tr[a + 1][c]);
  }
}

// FP64 covariance bins of gridded data on CUDA cores: a 16 x 16 output tile
// per block, subjects streamed through shared memory in chunks of 16.
__global__ void k_cov_dense_f64(int n, int P, const void* __restrict__ y, int y_prec,
                                const uint8_t* __restrict__ mask, const int32_t* __restrict__ Ni,
                                const double* __restrict__ mu, int mode, int32_t* __restrict__ cnt,
                                double* __restrict__ w, double* __restrict__ v) {
  __shared__ double rp[16][17], rq[16][17], mp[16][17], mq[16][17], wsub[16];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int p = blockIdx.y * 16 + ty, q = blockIdx.x * 16 + tx;
  int c = 0;
  double sw = 0.0, sv = 0.0;
  for (int i0 = 0; i0 < n; i0 += 16) {
    // load subject chunk: rows i0..i0+15 for the 16 p and 16 q columns
    {
      const int i = i0 + ty;
      const int pc = blockIdx.y * 16 + tx, qc = blockIdx.x * 16 + tx;
      double obs_p = 0.0, obs_q = 0.0, r_p = 0.0, r_q = 0.0;
      if (i < n) {
        if (pc < P) {
          const size_t idx = (size_t)i * P + pc;
          obs_p = (mask ? mask[idx] != 0 : true) ? 1.0 : 0.0;
          if (obs_p != 0.0) {
            const double yy = load_y(y, y_prec, idx);
            r_p = mode == FPCA_COV_RESIDUAL ? yy - mu[pc] : yy;
          }
        }
        if (qc < P) {
          const size_t idx = (size_t)i * P + qc;
          obs_q = (mask ? mask[idx] != 0 : true) ? 1.0 : 0.0;
          if (obs_q != 0.0) {
            const double yy = load_y(y, y_prec, idx);
            r_q = mode == FPCA_COV_RESIDUAL ? yy - mu[qc] : yy;
          }
        }
      }
      mp[ty][tx] = obs_p;
      rp[ty][tx] = r_p;
      mq[ty][tx] = obs_q;
      rq[ty][tx] = r_q;
      if (tx == 0) {
        const int N = i < n ? Ni[i] : 0;
        wsub[ty] = N >= 2 ? 1.0 / ((double)N * (double)(N - 1)) : 0.0;
      }
    }
    __syncthreads();
    const int kmax = min(16, n - i0);
    for (int k = 0; k < kmax; ++k) {
      const double both = mp[k][ty] * mq[k][tx];
      c += both != 0.0;
      sw = __dadd_rn(sw, __dmul_rn(wsub[k], both));
      sv = __dadd_rn(sv, __dmul_rn(__dmul_rn(wsub[k], rp[k][ty]), rq[k][tx]));
    }
    __syncthreads();
  }
  if (p < P && q < P) {
    const size_t o = (size_t)p * P + q;
    const bool diag = p == q;
    cnt[o] = diag ? 0 : c;
    w[o] = diag ? 0.0 : sw;
    v[o] = diag ? 0.0 : sv;
  }
}

// Observation -> subject map for the sparse pair scatter.  Offsets outside
// 0 <= offs[i] <= offs[i+1] <= N are reported (DERR_BOUNDS) and the subject
// is skipped, here and in the scatter.
__global__ void k_obs_subject(int n, long long N, const int64_t* __restrict__ offs,
                              int32_t* __restrict__ subj, int* __restrict__ err) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t lo = offs[i], hi = offs[i + 1];
  if (lo < 0 || hi < lo || hi > N) {
    atomicExch(err, DERR_BOUNDS);
    return;
  }
  for (int64_t j = lo; j < hi; ++j) subj[j] = i;
}

// Per-observation bin and response (residual or raw).
__global__ void k_obs_prep(long long N, int d, int m0, int m1, int m2,
                           const double* __restrict__ t, const double* __restrict__ y,
                           const double* __restrict__ mu, int mode, int32_t* __restrict__ ob,
                           double* __restrict__ orr) {
  const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (j >= N) return;
  const int m[3] = {m0, m1, m2};
  const int b = bin_index(t + j * d, d, m);
  ob[j] = b;
  orr[j] = mode == FPCA_COV_RESIDUAL ? y[j] - mu[b] : y[j];
}

// Sparse covariance bins: thread per observation j, loop over its subject's
// other observations l; integer-exact atomic pair counts and atomic sums.
template <typename T>
__global__ void k_cov_sparse(long long N, int P, const int64_t* __restrict__ offs,
                             const int32_t* __restrict__ subj, const int32_t* __restrict__ ob,
                             const double* __restrict__ orr, const int32_t* __restrict__ fold,
                             int nfold, int32_t* cnt, T* w, T* v, T* q, int* __restrict__ err) {
  const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (j >= N) return;
  const int i = subj[j];
  if (i < 0) return;  // subject with invalid offsets
  const int64_t lo = offs[i], hi = offs[i + 1];
  const long long Ni = hi - lo;
  if (Ni < 2) return;
  if (nfold > 0 && (fold[i] < 0 || fold[i] >= nfold)) {
    atomicExch(err, DERR_BOUNDS);
    return;
  }
  const double wi = 1.0 / ((double)Ni * (double)(Ni - 1));
  const long long PP = (long long)P * P;
  const long long row = (nfold > 0 ? (long long)fold[i] : 0ll) * PP + (long long)ob[j] * P;
  const double rj = orr[j];
  for (int64_t l = lo; l < hi; ++l) {
    if (l == j) continue;
    const long long at = row + ob[l];
    const double prod = rj * orr[l];
    atomicAdd(cnt + at, 1);
    atomicAdd(w + at, (T)wi);
    atomicAdd(v + at, (T)(wi * prod));
    if (q) atomicAdd(q + at, (T)(wi * prod * prod));
  }
}


// ---------------------------------------------------------------------------
// FP32 covariance bins of gridded data, split by folds, on CUDA cores.
// Subjects with N_i >= 2 are put in fold order (stable); each one's row gives
// three operand rows in that order -- the mask M, the response R (zero where
// unobserved) and R^2 -- of stride Ps (P rounded up to the tile edge, zero
// beyond P), and its weight w_i = 1/(N_i(N_i - 1)).  Per fold f, with D_f the
// diagonal of the fold's weights,
//   C = M'M,  W = M' D_f M,  V = R' D_f R,  Q = (R^2)' D_f (R^2)
// are computed 128 x 128 outputs per block, for the tile pairs on and above the
// diagonal; the tile below is written as the transpose (all four are symmetric).
// ---------------------------------------------------------------------------
constexpr int FG_T = 128;   // output tile edge
constexpr int FG_K = 16;    // subjects per pipeline stage
constexpr int FG_NT = 256;  // threads: 16 x 16, 8 x 8 outputs each

__device__ __forceinline__ int fold_slot(int i, int F, const int32_t* __restrict__ fold,
                                         const int32_t* __restrict__ Ni, int* err) {
  if (Ni[i] < 2) return -1;  // no pairs
  if (!fold) return 0;
  const int f = fold[i];
  if (f < 0 || f >= F) {
    atomicExch(err, DERR_BOUNDS);
    return -1;
  }
  return f;
}

// Stable fold order (one block of 1024 threads): order[fstart[f] + r] is the r-th
// subject of fold f in index order; fstart[F] is the number of subjects kept.
__global__ void __launch_bounds__(1024)
    k_fold_order(int n, int F, const int32_t* __restrict__ fold, const int32_t* __restrict__ Ni,
                 int32_t* __restrict__ order, int32_t* __restrict__ fstart, int* err) {
  __shared__ int fcount[64];
  __shared__ int wpre[32][64];  // per warp and fold: count, then running position
  __shared__ int base[64];
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5;
  if (tid < 64) fcount[tid] = 0;
  __syncthreads();
  for (int i = tid; i < n; i += 1024) {
    const int f = fold_slot(i, F, fold, Ni, err);
    if (f >= 0) atomicAdd(&fcount[f], 1);
  }
  __syncthreads();
  if (tid == 0) {
    int s = 0;
    for (int f = 0; f < F; ++f) {
      base[f] = s;
      fstart[f] = s;
      s += fcount[f];
    }
    fstart[F] = s;
  }
  __syncthreads();
  for (int c0 = 0; c0 < n; c0 += 1024) {
    for (int e = tid; e < 32 * 64; e += 1024) (&wpre[0][0])[e] = 0;
    __syncthreads();
    const int i = c0 + tid;
    const int f = i < n ? fold_slot(i, F, fold, Ni, err) : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, f);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    if (f >= 0 && rank == 0) wpre[wp][f] = __popc(peers);
    __syncthreads();
    if (tid < F) {  // exclusive prefix over the warps, fold by fold
      int run = base[tid];
      for (int w2 = 0; w2 < 32; ++w2) {
        const int c = wpre[w2][tid];
        wpre[w2][tid] = run;
        run += c;
      }
      base[tid] = run;
    }
    __syncthreads();
    if (f >= 0) order[wpre[wp][f] + rank] = i;
    __syncthreads();
  }
}

// Operand rows in fold order (block k: row k), see above; rows past fstart[F] are
// left alone (the Gram kernel never reads them).
__global__ void k_fold_operands(int n, int P, int Ps, int F, const void* __restrict__ y,
                                int y_prec, const uint8_t* __restrict__ mask,
                                const int32_t* __restrict__ Ni, const double* __restrict__ mu,
                                int mode, const int32_t* __restrict__ order,
                                const int32_t* __restrict__ fstart, float* __restrict__ X,
                                float* __restrict__ ws) {
  const int k = blockIdx.x;
  if (k >= fstart[F]) return;
  const int i = order[k];
  const size_t plane = (size_t)n * Ps;
  for (int p = threadIdx.x; p < Ps; p += blockDim.x) {
    float m = 0.f, r = 0.f, r2 = 0.f;
    if (p < P) {
      const size_t idx = (size_t)i * P + p;
      if (!mask || mask[idx]) {
        const double yy = load_y(y, y_prec, idx);
        const double rd = mode == FPCA_COV_RESIDUAL ? yy - mu[p] : yy;
        m = 1.f;
        r = (float)rd;
        r2 = (float)(rd * rd);
      }
    }
    const size_t o = (size_t)k * Ps + p;
    X[o] = m;
    X[plane + o] = r;
    X[2 * plane + o] = r2;
  }
  if (threadIdx.x == 0) {
    const double N = (double)Ni[i];
    ws[k] = (float)(1.0 / (N * (N - 1.0)));
  }
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src),
               "r"(valid ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// blockIdx.x: tile pair (bi <= bj), y: fold, z: plane (0 C, 1 W, 2 V, 3 Q).
// Thread (ty, tx) owns rows {4ty..4ty+3, 64+4ty..} and columns {4tx.., 64+4tx..}
// of the tile, so its shared-memory reads are float4s of consecutive addresses.
__global__ void __launch_bounds__(FG_NT, 2)
    k_fold_gram(int n, int P, int Ps, const float* __restrict__ X, const float* __restrict__ ws,
                const int32_t* __restrict__ fstart, const int2* __restrict__ pairs,
                int32_t* __restrict__ cnt, float* __restrict__ w, float* __restrict__ v,
                float* __restrict__ q, int vec) {
  __shared__ __align__(16) float As[2][FG_K][FG_T];
  __shared__ __align__(16) float Bs[2][FG_K][FG_T];
  __shared__ float Ss[2][FG_K];
  const int2 pr = pairs[blockIdx.x];
  const int f = blockIdx.y, z = blockIdx.z;
  const int k0 = fstart[f], k1 = fstart[f + 1];
  const int plane = z <= 1 ? 0 : z - 1;  // C and W from M, V from R, Q from R^2
  const float* src = X + (size_t)plane * n * Ps;
  const bool scaled = z > 0;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int p0 = pr.x * FG_T, q0 = pr.y * FG_T;
  // stage loader: 16 rows x 128 columns of each operand, two float4 per thread each
  auto load = [&](int st, int kb) {
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int e = tid + u * FG_NT;       // 0..511
      const int r = e >> 5, c4 = e & 31;   // row, float4 column
      const int k = kb + r;
      const bool ok = k < k1;
      const float* rowp = src + (size_t)(ok ? k : 0) * Ps;
      cp_async16(smem_addr(&As[st][r][4 * c4]), rowp + p0 + 4 * c4, ok);
      cp_async16(smem_addr(&Bs[st][r][4 * c4]), rowp + q0 + 4 * c4, ok);
    }
    if (tid < FG_K) Ss[st][tid] = (kb + tid < k1 && scaled) ? ws[kb + tid] : 1.f;
  };
  float2 acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
  const int nchunk = (k1 - k0 + FG_K - 1) / FG_K;
  if (nchunk > 0) load(0, k0);
  cp_async_commit();
  for (int c = 0; c < nchunk; ++c) {
    const int st = c & 1;
    if (c + 1 < nchunk) load(st ^ 1, k0 + (c + 1) * FG_K);
    cp_async_commit();
    cp_async_wait1();
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < FG_K; ++k) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[st][k][4 * ty]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[st][k][64 + 4 * ty]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[st][k][4 * tx]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[st][k][64 + 4 * tx]);
      const float sk = Ss[st][k];
      const float a[8] = {a0.x * sk, a0.y * sk, a0.z * sk, a0.w * sk,
                          a1.x * sk, a1.y * sk, a1.z * sk, a1.w * sk};
      const float2 b[4] = {make_float2(b0.x, b0.y), make_float2(b0.z, b0.w),
                           make_float2(b1.x, b1.y), make_float2(b1.z, b1.w)};
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float2 ai = make_float2(a[i], a[i]);
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = __ffma2_rn(ai, b[j], acc[i][j]);
      }
    }
    __syncthreads();  // the stage is overwritten by the load after next
  }
  // epilogue: the tile (p, q) and, off the diagonal, its transpose (q, p); the
  // p == q entries hold only j == l pairs and are zero.  vec: P % 4 == 0 and the
  // outputs 16-byte aligned, so four consecutive columns are stored at once.
  const long long PP = (long long)P * P;
  const size_t fo = (size_t)f * PP;
  auto put4 = [&](int row, int col, float4 val) {  // columns col..col+3
    if (row >= P) return;
    const float x[4] = {row == col ? 0.f : val.x, row == col + 1 ? 0.f : val.y,
                        row == col + 2 ? 0.f : val.z, row == col + 3 ? 0.f : val.w};
    const size_t o = fo + (size_t)row * P + col;
    if (vec && col + 3 < P) {
      if (z == 0)
        *reinterpret_cast<int4*>(cnt + o) = make_int4(__float2int_rn(x[0]), __float2int_rn(x[1]),
                                                      __float2int_rn(x[2]), __float2int_rn(x[3]));
      else
        *reinterpret_cast<float4*>((z == 1 ? w : z == 2 ? v : q) + o) =
            make_float4(x[0], x[1], x[2], x[3]);
      return;
    }
    for (int u = 0; u < 4; ++u) {
      if (col + u >= P) break;
      if (z == 0)
        cnt[o + u] = __float2int_rn(x[u]);
      else
        (z == 1 ? w : z == 2 ? v : q)[o + u] = x[u];
    }
  };
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int row = p0 + (i < 4 ? 4 * ty + i : 64 + 4 * ty + (i - 4));
    put4(row, q0 + 4 * tx, make_float4(acc[i][0].x, acc[i][0].y, acc[i][1].x, acc[i][1].y));
    put4(row, q0 + 64 + 4 * tx, make_float4(acc[i][2].x, acc[i][2].y, acc[i][3].x, acc[i][3].y));
  }
  if (pr.x != pr.y) {
#pragma unroll
    for (int cc = 0; cc < 8; ++cc) {
      const int j = (cc & 3) >> 1, comp = cc & 1;
      const int jj = cc < 4 ? j : j + 2;
      const int row = q0 + (cc < 4 ? 4 * tx + cc : 64 + 4 * tx + (cc - 4));
      auto pick = [&](int i) { return comp ? acc[i][jj].y : acc[i][jj].x; };
      put4(row, p0 + 4 * ty, make_float4(pick(0), pick(1), pick(2), pick(3)));
      put4(row, p0 + 64 + 4 * ty, make_float4(pick(4), pick(5), pick(6), pick(7)));
    }
  }
}

}  // namespace

fpca_status launch_subject_counts_dense(fpca_ctx* ctx, int n, int P, const uint8_t* mask,
                                        int32_t* Ni) {
  k_subject_counts<<<(n + 7) / 8, 256, 0, ctx->stream>>>(n, P, mask, Ni);
  FPCA_LAUNCHED(ctx, "subject_counts");
  return FPCA_OK;
}

fpca_status launch_bin_mean_dense(fpca_ctx* ctx, int n, int P, const void* y, int y_prec,
                                  const uint8_t* mask, const int32_t* Ni, int32_t* cnt,
                                  double* w, double* v, double* v2) {
  if (y_prec == FPCA_F64)
    k_bin_mean_dense<double><<<(P + 31) / 32, dim3(32, MB_SLICES), 0, ctx->stream>>>(
        n, P, static_cast<const double*>(y), mask, Ni, cnt, w, v, v2);
  else
    k_bin_mean_dense<float><<<(P + 31) / 32, dim3(32, MB_SLICES), 0, ctx->stream>>>(
        n, P, static_cast<const float*>(y), mask, Ni, cnt, w, v, v2);
  FPCA_LAUNCHED(ctx, "bin_mean_dense");
  return FPCA_OK;
}

fpca_status launch_bin_mean_sparse(fpca_ctx* ctx, int n, const fpca_grid* g, const int64_t* offs,
                                   const double* t, const double* y, int32_t* cnt, double* w,
                                   double* v, double* v2) {
  const int P = grid_P(g);
  int64_t Nobs = 0;
  if (fpca_no_capture(ctx, "reading offs[n] of scattered data") != FPCA_OK) return FPCA_E_UNSUPPORTED;
  cudaError_t e = cudaMemcpyAsync(&Nobs, offs + n, sizeof(int64_t), cudaMemcpyDeviceToHost,
                                  ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return fpca_fail(ctx, FPCA_E_CUDA, "reading offs[n]: %s", cudaGetErrorString(e));
  if (Nobs < 0) return fpca_fail(ctx, FPCA_E_INVALID_ARG, "offs[n] = %lld", (long long)Nobs);
  cudaMemsetAsync(cnt, 0, sizeof(int32_t) * P, ctx->stream);
  cudaMemsetAsync(w, 0, sizeof(double) * P, ctx->stream);
  cudaMemsetAsync(v, 0, sizeof(double) * P, ctx->stream);
  if (v2) cudaMemsetAsync(v2, 0, sizeof(double) * P, ctx->stream);
  k_bin_mean_sparse<<<(n + 127) / 128, 128, 0, ctx->stream>>>(
      n, (long long)Nobs, g->d, g->m[0], g->d > 1 ? g->m[1] : 1, g->d > 2 ? g->m[2] : 1, offs, t,
      y, cnt, w, v, v2, ctx->d_err);
  FPCA_LAUNCHED(ctx, "bin_mean_sparse");
  return FPCA_OK;
}

fpca_status launch_cov_operands_bf16(fpca_ctx* ctx, int n, int P, int Kpad, const void* y,
                                     int y_prec, const uint8_t* mask, const int32_t* Ni,
                                     const double* mu, int mode, uint16_t* ops) {
  if (Kpad % 64 != 0) return fpca_fail(ctx, FPCA_E_INVALID_ARG, "Kpad = %d", Kpad);
  dim3 grid((P + 31) / 32, Kpad / 64);
  __nv_bfloat162* o2 = reinterpret_cast<__nv_bfloat162*>(ops);
  if (y_prec == FPCA_F64)
    k_cov_operands_bf16<double><<<grid, dim3(32, 8), 0, ctx->stream>>>(
        n, P, Kpad, static_cast<const double*>(y), mask, Ni, mu, mode, o2);
  else
    k_cov_operands_bf16<float><<<grid, dim3(32, 8), 0, ctx->stream>>>(
        n, P, Kpad, static_cast<const float*>(y), mask, Ni, mu, mode, o2);
  FPCA_LAUNCHED(ctx, "cov_operands_bf16");
  return FPCA_OK;
}

fpca_status launch_cov_dense_f64(fpca_ctx* ctx, int n, int P, const void* y, int y_prec,
                                 const uint8_t* mask, const int32_t* Ni, const double* mu,
                                 int mode, int32_t* cnt, double* w, double* v) {
  dim3 grid((P + 15) / 16, (P + 15) / 16);
  k_cov_dense_f64<<<grid, dim3(16, 16), 0, ctx->stream>>>(n, P, y, y_prec, mask, Ni, mu, mode,
                                                          cnt, w, v);
  FPCA_LAUNCHED(ctx, "cov_dense_f64");
  return FPCA_OK;
}

fpca_status launch_cov_sparse(fpca_ctx* ctx, int n, const fpca_grid* g, const int64_t* offs,
                              const double* t, const double* y, const double* mu, int mode,
                              const int32_t* fold, int nfold, int prec, int32_t* cnt, void* w,
                              void* v, void* q) {
  const int P = grid_P(g);
  const long long PP = (long long)P * P;
  const int F = nfold > 0 ? nfold : 1;
  // total observation count (offs[n]) is needed on the host to size the launch
  int64_t Nobs = 0;
  if (fpca_no_capture(ctx, "reading offs[n] of scattered data") != FPCA_OK) return FPCA_E_UNSUPPORTED;
  cudaError_t e = cudaMemcpyAsync(&Nobs, offs + n, sizeof(int64_t), cudaMemcpyDeviceToHost,
                                  ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return fpca_fail(ctx, FPCA_E_CUDA, "reading offs[n]: %s", cudaGetErrorString(e));
  if (Nobs < 0 || Nobs > (1ll << 31))
    return fpca_fail(ctx, FPCA_E_INVALID_ARG, "offs[n] = %lld out of range", (long long)Nobs);
  const size_t esz = prec == FPCA_F64 ? sizeof(double) : sizeof(float);
  cudaMemsetAsync(cnt, 0, sizeof(int32_t) * PP * F, ctx->stream);
  cudaMemsetAsync(w, 0, esz * PP * F, ctx->stream);
  cudaMemsetAsync(v, 0, esz * PP * F, ctx->stream);
  if (q) cudaMemsetAsync(q, 0, esz * PP * F, ctx->stream);
  if (Nobs == 0) return fpca_check_launch(ctx, "cov_sparse memset");
  void* ws = fpca_workspace(ctx, WsCarve::round(4 * Nobs) * 2 + WsCarve::round(8 * Nobs) + 1024);
  if (!ws) return fpca_fail(ctx, FPCA_E_OOM, "workspace");
  WsCarve carve(ws);
  int32_t* subj = carve.take<int32_t>(Nobs);
  int32_t* ob = carve.take<int32_t>(Nobs);
  double* orr = carve.take<double>(Nobs);
  cudaMemsetAsync(subj, 0xff, sizeof(int32_t) * Nobs, ctx->stream);  // -1: no valid subject
  k_obs_subject<<<(n + 127) / 128, 128, 0, ctx->stream>>>(n, Nobs, offs, subj, ctx->d_err);
  FPCA_LAUNCHED(ctx, "obs_subject");
  const int nb = (int)((Nobs + 255) / 256);
  k_obs_prep<<<nb, 256, 0, ctx->stream>>>(Nobs, g->d, g->m[0], g->d > 1 ? g->m[1] : 1,
                                          g->d > 2 ? g->m[2] : 1, t, y, mu, mode, ob, orr);
  FPCA_LAUNCHED(ctx, "obs_prep");
  if (prec == FPCA_F64) {
    k_cov_sparse<double><<<nb, 256, 0, ctx->stream>>>(Nobs, P, offs, subj, ob, orr, fold, nfold,
                                                      cnt, static_cast<double*>(w),
                                                      static_cast<double*>(v),
                                                      static_cast<double*>(q), ctx->d_err);
  } else {
    k_cov_sparse<float><<<nb, 256, 0, ctx->stream>>>(Nobs, P, offs, subj, ob, orr, fold, nfold,
                                                     cnt, static_cast<float*>(w),
                                                     static_cast<float*>(v),
                                                     static_cast<float*>(q), ctx->d_err);
  }
  FPCA_LAUNCHED(ctx, "cov_sparse");
  return FPCA_OK;
}

fpca_status launch_cov_dense_folds(fpca_ctx* ctx, int n, int P, const void* y, int y_prec,
                                   const uint8_t* mask, const double* mu, int mode,
                                   const int32_t* fold, int nfold, int32_t* cnt, float* w,
                                   float* v, float* q) {
  const int F = nfold > 0 ? nfold : 1;
  if (n == 0) {  // no subjects: every bin is empty
    const size_t PPF = (size_t)P * P * F;
    cudaMemsetAsync(cnt, 0, sizeof(int32_t) * PPF, ctx->stream);
    cudaMemsetAsync(w, 0, sizeof(float) * PPF, ctx->stream);
    cudaMemsetAsync(v, 0, sizeof(float) * PPF, ctx->stream);
    if (q) cudaMemsetAsync(q, 0, sizeof(float) * PPF, ctx->stream);
    return fpca_check_launch(ctx, "cov_fold_gram memset");
  }
  const int Ps = (P + FG_T - 1) / FG_T * FG_T;
  const int nt = Ps / FG_T;
  const size_t need = WsCarve::round(sizeof(int32_t) * (size_t)n) * 2 +
                      WsCarve::round(sizeof(int32_t) * 65) +
                      WsCarve::round(sizeof(float) * 3 * (size_t)n * Ps) +
                      WsCarve::round(sizeof(float) * (size_t)n) +
                      WsCarve::round(sizeof(int2) * (size_t)nt * (nt + 1) / 2) + 2048;
  void* wsp = fpca_workspace(ctx, need);
  if (!wsp) return fpca_fail(ctx, FPCA_E_OOM, "workspace (%zu bytes)", need);
  WsCarve carve(wsp);
  int32_t* Ni = carve.take<int32_t>(n);
  int32_t* order = carve.take<int32_t>(n);
  int32_t* fstart = carve.take<int32_t>(65);
  float* X = carve.take<float>(3 * (size_t)n * Ps);
  float* wsub = carve.take<float>(n);
  int2* pairs = carve.take<int2>((size_t)nt * (nt + 1) / 2);
  std::vector<int2> ph;
  ph.reserve((size_t)nt * (nt + 1) / 2);
  for (int bi = 0; bi < nt; ++bi)
    for (int bj = bi; bj < nt; ++bj) ph.push_back(make_int2(bi, bj));
  // pageable source: staged before the call returns (so not capturable)
  if (fpca_no_capture(ctx, "the fold-split binning of gridded data") != FPCA_OK)
    return FPCA_E_UNSUPPORTED;
  if (cudaMemcpyAsync(pairs, ph.data(), sizeof(int2) * ph.size(), cudaMemcpyHostToDevice,
                      ctx->stream) != cudaSuccess)
    return fpca_check_launch(ctx, "fold gram tile pairs");
  fpca_status s = launch_subject_counts_dense(ctx, n, P, mask, Ni);
  if (s != FPCA_OK) return s;
  k_fold_order<<<1, 1024, 0, ctx->stream>>>(n, F, nfold > 0 ? fold : nullptr, Ni, order, fstart,
                                            ctx->d_err);
  FPCA_LAUNCHED(ctx, "fold_order");
  k_fold_operands<<<n, 128, 0, ctx->stream>>>(n, P, Ps, F, y, y_prec, mask, Ni, mu, mode, order,
                                              fstart, X, wsub);
  FPCA_LAUNCHED(ctx, "fold_operands");
  const dim3 grid((unsigned)ph.size(), F, q ? 4 : 3);
  auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
  const int vec = (P % 4 == 0 && al16(cnt) && al16(w) && al16(v) && (!q || al16(q))) ? 1 : 0;
  k_fold_gram<<<grid, FG_NT, 0, ctx->stream>>>(n, P, Ps, X, wsub, fstart, pairs, cnt, w, v, q,
                                                vec);
  FPCA_LAUNCHED(ctx, "cov_fold_gram");
  return FPCA_OK;
}
