// m2l_tc.cu -- M2L on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// The M2L of one level and one gating event is a batch of dense products
// (paper section 3.6.1, eq. m2l_matrix): for every canonical offset class and
// lag q, C (P x N) += K_{c,q} (P x P) . B (P x N), where the columns of B are
// the moments (one component each) of all interaction pairs of the class,
// gathered through the pair's cube-symmetry node map, and the columns of C are
// added to the target clusters' local coefficients of interval k+q.
//
// One CTA computes a 128 x 128 tile of C.  Per K chunk (128 bytes per row)
// the 256 threads load the operator rows and the gathered moment columns,
// round them to the tensor-core type (TF32, BF16, or BF16 hi + lo for the
// split-precision form) and store them in shared memory in the canonical
// K-major layout without swizzle (8-row x 16-byte core matrices; LBO = 128 B
// between core matrices along K, SBO = 1024 B between 8-row groups).  One
// thread issues tcgen05.mma into a 128-column TMEM accumulator and commits to
// an mbarrier; every wait on it is bounded and records a timeout in the error
// word.  The epilogue reads TMEM with tcgen05.ld (32 lanes x 16 columns per
// warp and call) and adds each group of pt = 4 consecutive rows -- the four
// time nodes of one spatial node, contiguous in the local coefficients --
// with one vector reduction red.global.add.v4.f32.
#include <cuda_bf16.h>

#include <cstdint>

#include "internal.h"

namespace tdbem {

namespace {

constexpr int kTileM = 128, kTileN = 128, kThreads = 256;
constexpr uint32_t kTmemCols = 128;
constexpr int kNCmp = 7;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);   // start address
  d |= (uint64_t)(128 >> 4) << 16;           // leading byte offset: next core matrix along K
  d |= (uint64_t)(1024 >> 4) << 32;          // stride byte offset: next 8-row group
  d |= (uint64_t)1 << 46;                    // descriptor version (sm_100 family)
  return d;                                  // base offset 0, no swizzle
}

// instruction descriptor: D = F32, A/B format fmt (1 = BF16 in kind::f16,
// 2 = TF32 in kind::tf32), both K-major, N = 128, M = 128
__device__ __forceinline__ uint32_t make_idesc(uint32_t fmt) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(kTileN >> 3) << 17) | ((uint32_t)(kTileM >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait; false on timeout
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (uint32_t i = 0; i < (1u << 20); ++i)
    if (mbar_try_wait(mbar, parity)) return true;
  return false;
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ uint32_t f32_to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// byte offset of (row, byte-in-row) in a 128-row x 128-byte K-major tile
__device__ __forceinline__ uint32_t tile_off(int row, int kbyte) {
  return (uint32_t)((row >> 3) * 1024 + (kbyte >> 4) * 128 + (row & 7) * 16 + (kbyte & 15));
}

}  // namespace

// prec: 1 = TF32, 2 = BF16, 3 = BF16 x 3, 4 = TF32 x 3 (split: hi*hi + hi*lo + lo*hi)
__global__ void __launch_bounds__(kThreads) k_m2l_tc(const int4* gemm, const int4* tiles, const float* ops, int P,
                                                     int pt, int PS, const int32_t* pO, const int32_t* pS,
                                                     const int16_t* psym, const int16_t* smap, const float* mom,
                                                     int k, float* loc, int Q, int prec, int32_t* err) {
  extern __shared__ __align__(1024) uint8_t dsm[];
  __shared__ int64_t src_off[kTileN];
  __shared__ int64_t dst_off[kTileN];
  __shared__ int32_t map_off[kTileN];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  // shared tiles (16 KB each): A hi, B hi, A lo, B lo
  uint8_t* tA = dsm;
  uint8_t* tB = dsm + 16384;
  uint8_t* tA2 = dsm + 32768;
  uint8_t* tB2 = dsm + 49152;

  const int4 tl = tiles[blockIdx.x];
  const int4 gd = gemm[tl.x];
  const int kind = gd.w & 0xff, q = (gd.w >> 8) & 0xff, qhi = (gd.w >> 16) & 0xff;
  const int nk = kind == 0 ? 3 : 4, c0 = kind == 0 ? 0 : 3;
  const int var = (q == qhi) ? 1 : 0;
  const float* A = ops + ((int64_t)gd.x * 2 + kind) * P * P;
  const int row0 = tl.y * kTileM, col0 = tl.z * kTileN;
  const int ncol = gd.z * nk;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool split = prec == 3 || prec == 4;
  const bool tf = prec == 1 || prec == 4;
  const int es = tf ? 4 : 2;  // bytes per element in shared memory
  const int KC = 128 / es;           // K elements per chunk

  if (tid < kTileN) {
    int gcol = col0 + tid;
    if (gcol < ncol) {
      int pr = gd.y + gcol / nk, c = c0 + gcol % nk;
      src_off[tid] = (((int64_t)pS[pr] * 2 + (k & 1)) * 2 * kNCmp + (int64_t)var * kNCmp + c) * P;
      dst_off[tid] = (((int64_t)pO[pr] * Q + ((k + q) % Q)) * kNCmp + c) * P;
      map_off[tid] = (int32_t)psym[pr] * PS;
    } else {
      src_off[tid] = -1;
    }
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = make_idesc(tf ? 2u : 1u);
  const uint32_t mb = smem_u32(&mbar);
  bool ok = true;

  const int nchunks = (P + KC - 1) / KC;
  for (int ch = 0; ch < nchunks && ok; ++ch) {
    const int k0 = ch * KC;
    // operator rows: 4 consecutive K values per task
    for (int e = tid; e < kTileM * (KC / 4); e += kThreads) {
      int r = e / (KC / 4), g = e % (KC / 4);
      int row = row0 + r, kk = k0 + 4 * g;
      float x[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) x[u] = (row < P && kk + u < P) ? A[(int64_t)row * P + kk + u] : 0.f;
      if (tf) {
        uint4 w = make_uint4(f32_to_tf32(x[0]), f32_to_tf32(x[1]), f32_to_tf32(x[2]), f32_to_tf32(x[3]));
        *(uint4*)(tA + tile_off(r, 16 * g)) = w;
        if (split) {
          uint4 l = make_uint4(f32_to_tf32(x[0] - __uint_as_float(w.x)), f32_to_tf32(x[1] - __uint_as_float(w.y)),
                               f32_to_tf32(x[2] - __uint_as_float(w.z)), f32_to_tf32(x[3] - __uint_as_float(w.w)));
          *(uint4*)(tA2 + tile_off(r, 16 * g)) = l;
        }
      } else {
        __nv_bfloat16 h[4], l[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          h[u] = __float2bfloat16_rn(x[u]);
          l[u] = __float2bfloat16_rn(x[u] - __bfloat162float(h[u]));
        }
        *(uint2*)(tA + tile_off(r, 8 * g)) = *(uint2*)h;
        if (split) *(uint2*)(tA2 + tile_off(r, 8 * g)) = *(uint2*)l;
      }
    }
    // moment columns, gathered through the symmetry map
    for (int e = tid; e < kTileN * (KC / 4); e += kThreads) {
      int n = e / (KC / 4), g = e % (KC / 4);
      int kk = k0 + 4 * g;
      float x[4] = {0.f, 0.f, 0.f, 0.f};
      int64_t so = src_off[n];
      if (so >= 0) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          int kq = kk + u;
          if (kq < P) {
            int bp = kq / pt, nt = kq - bp * pt;
            x[u] = mom[so + (int64_t)smap[map_off[n] + bp] * pt + nt];
          }
        }
      }
      if (tf) {
        uint4 w = make_uint4(f32_to_tf32(x[0]), f32_to_tf32(x[1]), f32_to_tf32(x[2]), f32_to_tf32(x[3]));
        *(uint4*)(tB + tile_off(n, 16 * g)) = w;
        if (split) {
          uint4 l = make_uint4(f32_to_tf32(x[0] - __uint_as_float(w.x)), f32_to_tf32(x[1] - __uint_as_float(w.y)),
                               f32_to_tf32(x[2] - __uint_as_float(w.z)), f32_to_tf32(x[3] - __uint_as_float(w.w)));
          *(uint4*)(tB2 + tile_off(n, 16 * g)) = l;
        }
      } else {
        __nv_bfloat16 h[4], l[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          h[u] = __float2bfloat16_rn(x[u]);
          l[u] = __float2bfloat16_rn(x[u] - __bfloat162float(h[u]));
        }
        *(uint2*)(tB + tile_off(n, 8 * g)) = *(uint2*)h;
        if (split) *(uint2*)(tB2 + tile_off(n, 8 * g)) = *(uint2*)l;
      }
    }
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t a0 = smem_u32(tA), b0 = smem_u32(tB), a1 = smem_u32(tA2), b1 = smem_u32(tB2);
      for (int s = 0; s < 4; ++s) {
        uint32_t acc = (ch > 0 || s > 0) ? 1u : 0u;
        uint32_t off = 256u * s;  // two core matrices (32 bytes of K) per instruction
        if (tf) {
          mma_tf32(tmem, make_desc(a0 + off), make_desc(b0 + off), idesc, acc);
          if (split) {
            mma_tf32(tmem, make_desc(a0 + off), make_desc(b1 + off), idesc, 1u);
            mma_tf32(tmem, make_desc(a1 + off), make_desc(b0 + off), idesc, 1u);
          }
        } else {
          mma_f16(tmem, make_desc(a0 + off), make_desc(b0 + off), idesc, acc);
          if (split) {
            mma_f16(tmem, make_desc(a0 + off), make_desc(b1 + off), idesc, 1u);
            mma_f16(tmem, make_desc(a1 + off), make_desc(b0 + off), idesc, 1u);
          }
        }
      }
      mma_commit(mb);
    }
    // the next chunk overwrites the tiles: wait for the MMAs to finish; the
    // verdict is made uniform across the CTA before anyone acts on it
    bool mine = mbar_wait(mb, (uint32_t)(ch & 1));
    ok = __syncthreads_and(mine) != 0;
    if (!ok && tid == 0) atomicExch(err, 1);
  }
  if (!ok) {
    // give the tensor core a last bounded chance to drain before TMEM is freed
    mbar_wait(mb, (uint32_t)((nchunks - 1) & 1));
  }
  tc_fence_after();
  if (ok) {
    const int q4 = warp & 3, cb = (warp >> 2) * 64;
    const int r = row0 + q4 * 32 + lane;
    for (int j0 = 0; j0 < 64; j0 += 16) {
      uint32_t v[16];
      uint32_t addr = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(cb + j0);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
          "%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(addr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int jj = 0; jj < 16; ++jj) {
        const int n = cb + j0 + jj;
        float val = __uint_as_float(v[jj]);
        const bool col_ok = col0 + n < ncol;
        if (pt == 4) {
          float v1 = __shfl_down_sync(0xffffffffu, val, 1);
          float v2 = __shfl_down_sync(0xffffffffu, val, 2);
          float v3 = __shfl_down_sync(0xffffffffu, val, 3);
          if (col_ok && (lane & 3) == 0 && r < P) {
            int ap = r >> 2;
            float* dst = loc + dst_off[n] + (int64_t)smap[map_off[n] + ap] * 4;
            atomicAdd((float4*)dst, make_float4(val, v1, v2, v3));
          }
        } else if (col_ok && r < P) {
          int ap = r / pt, m = r - ap * pt;
          atomicAdd(loc + dst_off[n] + (int64_t)smap[map_off[n] + ap] * pt + m, val);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

}  // namespace tdbem

// Launch the tensor-core M2L of one level event.
tdbem_status tdbem_m2l_tc(tdbem_ctx* c, const int4* gemm, const int4* tiles, int ntiles, const float* ops, int P,
                          int pt, int PS, const int32_t* pO, const int32_t* pS, const int16_t* psym,
                          const int16_t* smap, const float* mom, int k, float* loc, int Q, int prec, int32_t* err) {
  using namespace tdbem;
  static bool attr = false;
  if (!attr) {
    TDBEM_CUDA_TRY(c, cudaFuncSetAttribute(k_m2l_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 65536 + 1024));
    attr = true;
  }
  if (ntiles == 0) return TDBEM_OK;
  k_m2l_tc<<<ntiles, kThreads, 65536 + 1024, c->stream>>>(gemm, tiles, ops, P, pt, PS, pO, pS, psym, smap, mom, k,
                                                          loc, Q, prec, err);
  TDBEM_CUDA_TRY(c, cudaGetLastError());
  return TDBEM_OK;
}
