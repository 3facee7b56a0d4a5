// gemm_tc.cu -- dense products on the tcgen05 tensor cores for the learned
// warm start's width-256 network: C (M x N, FP32, row-major) = A (M x K) .
// B (N x K)^T, with A and B row-major BF16 (K contiguous) and the products
// accumulated in FP32 in tensor memory.
//
// One CTA computes rows [128 bx, +128) and columns [nt by, +nt) of C over the
// K chunks (64 BF16, 128 bytes per row) [kcs bz, kcs (bz + 1)): blockIdx.z
// splits K, the partial products then being added into C atomically.  All
// threads copy a chunk's operand rows into one of two stages with 16-byte
// cp.async copies (zero-filled past M, N and K) in the canonical K-major
// layout; thread 0 issues the chunk's four MMAs (K = 16 each) and commits to
// the stage's barrier, and the next chunk is copied into the other stage
// while they run.  Warps 0-3 read the accumulator (TMEM lane quarter = their
// 32 rows) and store or add C with 16-byte accesses.  Every wait is bounded;
// a timeout sets *err and skips the epilogue.
#include <cuda_bf16.h>

#include <algorithm>

#include "internal.h"
#include "tc.cuh"

namespace tdbem {

using namespace tc;

namespace {
constexpr int kGThreads = 256;
constexpr int kGStageA = 16384;  // 128 rows x 128 bytes
constexpr int kGStageB = 32768;  // up to 256 rows x 128 bytes
constexpr int kGSmem = 2 * (kGStageA + kGStageB);
}  // namespace

__global__ void __launch_bounds__(kGThreads) k_gemm_bf16(const __nv_bfloat16* A, int64_t lda,
                                                         const __nv_bfloat16* B, int64_t ldb, float* C, int64_t ldc,
                                                         int M, int N, int K, int nt, int kcs, int add,
                                                         int32_t* err) {
  extern __shared__ __align__(1024) uint8_t dsm[];
  __shared__ __align__(8) uint64_t mma_done[2];
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * 128, n0 = blockIdx.y * nt;
  const int nch = (K + 63) / 64;
  const int kc0 = blockIdx.z * kcs, kc1 = min(nch, kc0 + kcs);
  if (tid == 0) {
    for (int s = 0; s < 2; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mma_done[s])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(256u));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = idesc_f32acc(1u, nt);  // BF16 operands
  bool ok = true;
  int i = 0;
  for (int ch = kc0; ch < kc1; ++ch, ++i) {
    const int st = i & 1;
    // the stage was last read by the MMAs of chunk i - 2
    if (i >= 2 && !__syncthreads_and(mbar_wait(smem_u32(&mma_done[st]), (uint32_t)(((i >> 1) - 1) & 1)))) {
      ok = false;
      break;
    }
    uint8_t* sa = dsm + st * (kGStageA + kGStageB);
    uint8_t* sb = sa + kGStageA;
    for (int u = tid; u < 1024 + nt * 8; u += kGThreads) {
      const bool isA = u < 1024;
      const int uu = isA ? u : u - 1024;
      const int r = unit_row(uu), kk = ch * 64 + unit_k16(uu) * 8;
      const int grow = (isA ? m0 : n0) + r;
      const bool v = grow < (isA ? M : N) && kk < K;
      const __nv_bfloat16* src = v ? (isA ? A + grow * lda + kk : B + grow * ldb + kk) : A;
      cp_async16_zfill(smem_u32((isA ? sa : sb) + uu * 16), src, v ? 16u : 0u);
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(sa), b0 = smem_u32(sb);
      for (int ks = 0; ks < 4; ++ks) {
        const uint32_t off = 256u * ks;  // 32 bytes of K per instruction
        mma_f16(tmem, make_desc(a0 + off), make_desc(b0 + off), idesc, (i > 0 || ks > 0) ? 1u : 0u);
      }
      mma_commit(smem_u32(&mma_done[st]));
    }
  }
  // the last commit covers every MMA issued
  if (i > 0 && !mbar_wait(smem_u32(&mma_done[(i - 1) & 1]), (uint32_t)(((i - 1) >> 1) & 1))) ok = false;
  ok = __syncthreads_and(ok) != 0;
  tc_fence_after();
  if (!ok) {
    if (tid == 0) atomicExch(err, 1);
  } else if (warp < 4 && i > 0) {
    const int r = m0 + warp * 32 + lane;
    for (int j0 = 0; j0 < nt; j0 += 16) {
      uint32_t v[16];
      const uint32_t addr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)j0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
          "%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(addr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (r < M) {
#pragma unroll
        for (int q = 0; q < 16; q += 4) {
          const int n = n0 + j0 + q;
          if (n < N) {
            const float4 val = make_float4(__uint_as_float(v[q]), __uint_as_float(v[q + 1]),
                                           __uint_as_float(v[q + 2]), __uint_as_float(v[q + 3]));
            float4* dst = (float4*)(C + (int64_t)r * ldc + n);
            if (add)
              atomicAdd(dst, val);
            else
              *dst = val;
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256u));
}

}  // namespace tdbem

// C = A . B^T (add = 0) or C += A . B^T (add = 1), K split over ksplit CTAs
// (ksplit > 1 needs add = 1).  Requirements, checked here: K, lda and ldb
// multiples of 8 and A, B 16-byte aligned (16-byte operand copies); N and ldc
// multiples of 4 and C 16-byte aligned (16-byte epilogue accesses).
tdbem_status tdbem_gemm_bf16(tdbem_ctx* c, cudaStream_t st, const __nv_bfloat16* A, int64_t lda,
                             const __nv_bfloat16* B, int64_t ldb, float* C, int64_t ldc, int M, int N, int K, int add,
                             int ksplit, int32_t* err) {
  using namespace tdbem;
  static bool attr = false;
  if (!attr) {
    TDBEM_CUDA_TRY(c, cudaFuncSetAttribute(k_gemm_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, kGSmem));
    attr = true;
  }
  if (M <= 0 || N <= 0 || K <= 0) return TDBEM_OK;
  if (K % 8 || lda % 8 || ldb % 8 || N % 4 || ldc % 4 || ((uintptr_t)A & 15) || ((uintptr_t)B & 15) ||
      ((uintptr_t)C & 15) || (ksplit > 1 && !add) || ksplit < 1) {
    c->set_error("gemm: operand shapes or alignment");
    return TDBEM_EINVAL;
  }
  const int nt = std::min(256, (N + 15) / 16 * 16);
  const int nch = (K + 63) / 64;
  const int ks = std::min(ksplit, nch);
  const int kcs = (nch + ks - 1) / ks;
  const dim3 grid((unsigned)((M + 127) / 128), (unsigned)((N + nt - 1) / nt), (unsigned)((nch + kcs - 1) / kcs));
  k_gemm_bf16<<<grid, kGThreads, kGSmem, st>>>(A, lda, B, ldb, C, ldc, M, N, K, nt, kcs, add, err);
  TDBEM_CUDA_TRY(c, cudaGetLastError());
  return TDBEM_OK;
}
