// Covariance binning of gridded data as Gram products on tcgen05 tensor cores.
//
// For data on the grid nodes, the binned sums of Eq. (2.4) over ordered pairs
// j != l of one subject are Gram matrices of the n x P subject-by-node
// planes (Section 3.2 binning, diagonal p == q dropped):
//   C = M'M,   W = (w M)'M,   V = R~'R~,   R~_ip = sqrt(w_i) R_ip M_ip.
// Operands are BF16 in K-major layout (subject index contiguous) and stream
// through a TMA -> shared memory -> tcgen05.mma pipeline; the 128 x 128
// accumulator lives in tensor memory (TMEM) and the epilogue reads it back
// with tcgen05.ld.  All three products are symmetric, so only output tiles
// with tile_row <= tile_col are computed and each is written twice (direct
// and mirrored).  0/1 products accumulate exactly in FP32 below 2^24 terms,
// so the pair counts are exact integers.
#include <cuda_bf16.h>

#include "ptx.cuh"

namespace {

constexpr int BM = 128, BN = 128, BK = 64;  // BK bf16 = 128 bytes = one swizzle row
constexpr int STAGES = 3;  // three stages: two CTAs per SM, one's epilogue overlapping the other's MMAs
constexpr int TILE_BYTES = BM * BK * 2;
constexpr int STAGE_BYTES = 2 * TILE_BYTES;
constexpr uint32_t TMEM_COLS = 128;
constexpr uint32_t IDESC = ptx::idesc_f32acc(1u /*BF16*/, BM, BN);
constexpr size_t SMEM_BYTES = STAGES * STAGE_BYTES + 1024 /*align*/ + 256 /*barriers*/;

struct GramJob {
  int a_plane, b_plane;  // operand planes (rows a_plane*P .. of the [3P x Kpad] tensor)
  void* out;             // P x P
  int out_int;           // 1: int32 counts, 0: float
};
struct GramJobs {
  GramJob j[3];
};

__global__ void __launch_bounds__(128, 2)
    k_gram_tc(const __grid_constant__ CUtensorMap tmap, int P, int Kpad, GramJobs jobs, int* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* done = empty + STAGES;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // upper-triangle tile (tm <= tn) from the linear block index
  const int L = blockIdx.x;
  int tn = 0;
  while ((tn + 1) * (tn + 2) / 2 <= L) ++tn;
  const int tm = L - tn * (tn + 1) / 2;
  const GramJob job = jobs.j[blockIdx.y];
  const int nk = Kpad / BK;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      ptx::mbar_init(ptx::smem_u32(&full[s]), 1);
      ptx::mbar_init(ptx::smem_u32(&empty[s]), 1);
    }
    ptx::mbar_init(ptx::smem_u32(done), 1);
    ptx::fence_mbar_init();
  }
  if (warp == 2) {
    ptx::tmem_alloc(ptx::smem_u32(tslot), TMEM_COLS);
    ptx::tmem_relinquish();
  }
  ptx::tc_fence_before();
  __syncthreads();
  ptx::tc_fence_after();
  const uint32_t tmem = *tslot;

  if (warp == 0 && lane == 0) {
    // TMA producer
    const int rowA = job.a_plane * P + tm * BM;
    const int rowB = job.b_plane * P + tn * BN;
    int issued = 0;
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      const uint32_t ph = (kb / STAGES) & 1;
      if (!ptx::mbar_wait(ptx::smem_u32(&empty[s]), ph ^ 1u, err)) break;
      const uint32_t fb = ptx::smem_u32(&full[s]);
      ptx::mbar_arrive_expect_tx(fb, STAGE_BYTES);
      const uint32_t dst = ptx::smem_u32(smem + s * STAGE_BYTES);
      ptx::tma_load_2d(dst, &tmap, fb, kb * BK, rowA);
      ptx::tma_load_2d(dst + TILE_BYTES, &tmap, fb, kb * BK, rowB);
      issued = kb + 1;
    }
    if (issued < nk) {
      // gave up: let the copies already issued land before the CTA exits
      for (int kb = (issued > STAGES ? issued - STAGES : 0); kb < issued; ++kb)
        ptx::mbar_wait(ptx::smem_u32(&full[kb % STAGES]), (kb / STAGES) & 1, err);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer: one thread drives the tensor core
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % STAGES;
      const uint32_t ph = (kb / STAGES) & 1;
      if (!ptx::mbar_wait(ptx::smem_u32(&full[s]), ph, err)) break;
      ptx::tc_fence_after();
      const uint32_t a = ptx::smem_u32(smem + s * STAGE_BYTES);
      const uint32_t b = a + TILE_BYTES;
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) {
        ptx::tc_mma_f16(tmem, ptx::sdesc_kmajor_sw128(a + kk * 32),
                        ptx::sdesc_kmajor_sw128(b + kk * 32), IDESC, (kb | kk) != 0);
      }
      ptx::tc_commit(ptx::smem_u32(&empty[s]));
    }
    ptx::tc_commit(ptx::smem_u32(done));
  }
  __syncwarp();

  // Epilogue: warp w owns accumulator rows (TMEM lanes) 32w .. 32w+31.
  const bool have = ptx::mbar_wait(ptx::smem_u32(done), 0, err);
  __syncwarp();
  ptx::tc_fence_after();
  if (have) {
    // The operand stages are free once every MMA has completed: each warp takes a
    // 32 x 33 word scratch there to turn its rows around, so that the direct tile,
    // like the mirrored one, is written 32 consecutive words per store instruction.
    uint32_t* scr = reinterpret_cast<uint32_t*>(smem) + warp * 32 * 33;
    const int row0 = tm * BM + warp * 32;
    const int row = row0 + lane;
#pragma unroll 1
    for (int c = 0; c < BN / 32; ++c) {
      uint32_t r[32];
      ptx::tmem_ld_32x32b_x32(tmem + (static_cast<uint32_t>(warp * 32) << 16) + c * 32, r);
      ptx::tmem_ld_wait();
      const int col0 = tn * BN + c * 32;
      uint32_t bits[32];  // the output words of row `row`, columns col0 .. col0 + 31
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const float x = (row == col0 + j) ? 0.f : __uint_as_float(r[j]);
        bits[j] = job.out_int ? static_cast<uint32_t>(__float2int_rn(x)) : __float_as_uint(x);
      }
      uint32_t* out = static_cast<uint32_t*>(job.out);
      if (tm != tn) {  // mirrored tile: lanes are consecutive rows = consecutive columns there
#pragma unroll
        for (int j = 0; j < 32; ++j) out[(size_t)(col0 + j) * P + row] = bits[j];
      }
#pragma unroll
      for (int j = 0; j < 32; ++j) scr[lane * 33 + j] = bits[j];
      __syncwarp();
#pragma unroll 4
      for (int rr = 0; rr < 32; ++rr)
        out[(size_t)(row0 + rr) * P + col0 + lane] = scr[rr * 33 + lane];
      __syncwarp();
    }
  }
  ptx::tc_fence_before();
  __syncthreads();
  if (warp == 2) ptx::tmem_dealloc(tmem, TMEM_COLS);
}

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

}  // namespace

fpca_status launch_gram_tc(fpca_ctx* ctx, int P, int Kpad, const uint16_t* ops, int32_t* cnt,
                           float* w, float* v) {
  if (P % BM != 0 || Kpad % BK != 0)
    return fpca_fail(ctx, FPCA_E_UNSUPPORTED, "gram_tc needs P %% 128 == 0 and Kpad %% 64 == 0");
  EncodeTiledFn enc = encode_fn();
  if (!enc) return fpca_fail(ctx, FPCA_E_CUDA, "cuTensorMapEncodeTiled is unavailable");
  CUtensorMap map;
  const cuuint64_t dims[2] = {(cuuint64_t)Kpad, (cuuint64_t)3 * P};
  const cuuint64_t strides[1] = {(cuuint64_t)Kpad * 2};
  const cuuint32_t box[2] = {BK, BM};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<uint16_t*>(ops), dims,
                   strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                   CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fpca_fail(ctx, FPCA_E_CUDA, "tensor map encode failed (%d)", (int)r);
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
    attr_set = true;
  }
  GramJobs jobs;
  jobs.j[0] = GramJob{0, 0, cnt, 1};
  jobs.j[1] = GramJob{1, 0, w, 0};
  jobs.j[2] = GramJob{2, 2, v, 0};
  const int T = P / BM;
  dim3 grid(T * (T + 1) / 2, 3);
  k_gram_tc<<<grid, 128, SMEM_BYTES, ctx->stream>>>(map, P, Kpad, jobs, ctx->d_err);
  FPCA_LAUNCHED(ctx, "gram_tc");
  return FPCA_OK;
}
