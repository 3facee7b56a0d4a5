// m2l_tc.cu -- M2L on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// The M2L of one level and one gating event is a batch of dense products
// (paper section 3.6.1, eq. m2l_matrix): for every canonical offset class and
// lag q, C (P x N) += K_{c,q} (P x P) . B (P x N), where the columns of B are
// the moments (one component each) of all interaction pairs of the class,
// gathered through the pair's cube-symmetry node map, and the columns of C are
// added to the target clusters' local coefficients of interval k+q.
//
// One CTA computes two 128 x 128 tiles of C that share their columns (the
// two 128-row halves of a 256-row operator), so each gathered moment chunk
// feeds both: the gathers, which bound the kernel, are halved per output.
// Operand tiles live in shared
// memory in the canonical K-major layout without swizzle: 8-row x 16-byte
// core matrices, LBO = 128 B between core matrices along K, SBO = 1024 B
// between 8-row groups.  With 128 bytes of K per row that layout is a linear
// run of 1024 16-byte units, unit u holding row 8(u >> 6) + (u & 7) and K
// bytes 16((u >> 3) & 7) .. +15, so thread t writing units t, t+256, ... is
// free of bank conflicts.  The operators are converted once at setup into
// exactly these images (TF32, BF16, or hi and lo parts for the split forms,
// zero-padded past P) and brought in by TMA bulk copies (cp.async.bulk, one
// per row tile and chunk, completing on an mbarrier); the moment columns
// are gathered through the symmetry map one spatial node (pt = 4 time
// coefficients, one 16-byte load) at a time and converted on the fly.  One
// thread issues tcgen05.mma into a 128-column TMEM accumulator per row tile and commits to
// an mbarrier; every wait on it is bounded and records a timeout in the error
// word.  The epilogue reads TMEM with tcgen05.ld (32 lanes x 16 columns per
// warp and call) and adds each group of pt = 4 consecutive rows -- the four
// time nodes of one spatial node, contiguous in the local coefficients --
// with one vector reduction red.global.add.v4.f32.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>

#include "internal.h"
#include "tc.cuh"

namespace tdbem {

using namespace tc;

namespace {

constexpr int kTileM = 128, kTileN = 128, kThreads = 256;
constexpr int kTileBytes = 16384;  // one 128 x 128-byte operand tile
// per CTA: kMT 128-row operator tiles sharing one gathered B, one 128-column
// TMEM accumulator each; shared memory A hi/lo per row tile, then B hi/lo
template <int kMT>
constexpr int smem_tiles() { return (2 * kMT + 2) * kTileBytes; }
constexpr int kNCmp = 7;
constexpr int kSmapSmem = 24 * 1024;  // largest symmetry-map table staged in shared memory

// instruction descriptor: D = F32, A/B format fmt (1 = BF16 in kind::f16,
// 2 = TF32 in kind::tf32), both K-major, N = 128, M = 128
__device__ __forceinline__ uint32_t make_idesc(uint32_t fmt) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(kTileN >> 3) << 17) | ((uint32_t)(kTileM >> 4) << 24);
}

__device__ __forceinline__ uint32_t f32_to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}


// operand formats of the tensor-core forms
enum { kFmtTf32 = 0, kFmtBf16 = 1, kFmtF16 = 2 };

// hi (and lo = residual) parts of E consecutive values in the tensor-core type
template <int kFmt>
__device__ __forceinline__ void split_unit(const float* x, uint4& hi, uint4& lo) {
  if (kFmt == kFmtTf32) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      h[u] = f32_to_tf32(x[u]);
      l[u] = f32_to_tf32(x[u] - __uint_as_float(h[u]));
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
  } else if (kFmt == kFmtF16) {
    __align__(16) __half h[8], l[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      h[u] = __float2half_rn(x[u]);
      l[u] = __float2half_rn(x[u] - __half2float(h[u]));
    }
    hi = *(uint4*)h;
    lo = *(uint4*)l;
  } else {
    __align__(16) __nv_bfloat16 h[8], l[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      h[u] = __float2bfloat16_rn(x[u]);
      l[u] = __float2bfloat16_rn(x[u] - __bfloat162float(h[u]));
    }
    hi = *(uint4*)h;
    lo = *(uint4*)l;
  }
}

__device__ __forceinline__ void split_any(int fmt, const float* x, uint4& hi, uint4& lo) {
  if (fmt == kFmtTf32)
    split_unit<kFmtTf32>(x, hi, lo);
  else if (fmt == kFmtF16)
    split_unit<kFmtF16>(x, hi, lo);
  else
    split_unit<kFmtBf16>(x, hi, lo);
}

// Power-of-two scale that brings the largest magnitude m of a block of
// values into [2^14, 2^15) for the FP16 form (clamped so that the scale and
// its inverse are normal FP32 numbers; 1 for an all-zero block).
__device__ __forceinline__ int f16_scale_exp(float m) {
  if (!(m > 0.f)) return 0;
  int e;
  frexpf(m, &e);  // m = f 2^e, f in [0.5, 1)
  return max(-126, min(126, 15 - e));
}

}  // namespace

// Operator scales of the FP16 form: for every operator ops[opk] (P x P), the
// power of two 2^s that brings its largest magnitude into [2^14, 2^15), and
// 2^-s.  One block per operator.
__global__ void k_m2l_opscale(const float* ops, int P, float* scale, float* inv) {
  const int64_t opk = blockIdx.x;
  const float* o = ops + opk * P * P;
  float m = 0.f;
  for (int64_t i = threadIdx.x; i < (int64_t)P * P; i += blockDim.x) m = fmaxf(m, fabsf(o[i]));
  for (int d = 16; d > 0; d >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, d));
  __shared__ float wm[32];
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, wm[w]);
    m = fmaxf(m, wm[0]);
    const int sx = f16_scale_exp(m);
    scale[opk] = ldexpf(1.f, sx);
    inv[opk] = ldexpf(1.f, -sx);
  }
}

// Operator images: img[((((op*2 + kind)*nrt + rt)*nch + ch)*nparts + part)*1024 + u]
// is unit u of row tile rt, K chunk ch, part (0 hi, 1 lo) of operator
// ops[op][kind] (P x P, row-major FP32).  One thread per unit.
__global__ void k_m2l_images(const float* ops, int64_t nunits, int P, int nrt, int nch, int nparts, int fmt,
                             const float* scale, uint4* img) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nunits) return;
  const int u = (int)(t & 1023);
  int64_t rest = t >> 10;
  const int part = (int)(rest % nparts);
  rest /= nparts;
  const int ch = (int)(rest % nch);
  rest /= nch;
  const int rt = (int)(rest % nrt);
  const int64_t opk = rest / nrt;  // op * 2 + kind
  const bool tf = fmt == kFmtTf32;
  const int E = tf ? 4 : 8, KC = tf ? 32 : 64;
  const int row = rt * kTileM + unit_row(u);
  const int k0 = ch * KC + unit_k16(u) * E;
  const float sc = scale ? scale[opk] : 1.f;
  float x[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    int kk = k0 + e;
    x[e] = (e < E && row < P && kk < P) ? sc * ops[(opk * P + row) * P + kk] : 0.f;
  }
  uint4 hi, lo;
  split_any(fmt, x, hi, lo);
  img[t] = part == 0 ? hi : lo;
}

// prec: 1 = TF32, 2 = BF16, 3 = BF16 x 3, 4 = TF32 x 3 (split: hi*hi + hi*lo + lo*hi)
template <int kMT>
__global__ void __launch_bounds__(kThreads) k_m2l_tc(const int4* gemm, const int4* tiles, const uint4* img, int P,
                                                     int pt, int PS, const int32_t* pO, const int32_t* pC,
                                                     const int16_t* psym, const int16_t* smap, const float* pk,
                                                     int k, float* loc, int Q, int R, int prec, const float* opinv,
                                                     const float* pkinv, int32_t* err) {
  constexpr uint32_t kTmemCols = 128 * kMT;
  extern __shared__ __align__(1024) uint8_t dsm[];
  __shared__ int64_t src_off[kTileN];
  __shared__ int64_t dst_off[kTileN];
  __shared__ int32_t map_off[kTileN];
  __shared__ float col_inv[kTileN];  // the FP16 form's inverse column scales
  __shared__ __align__(8) uint64_t mbar;   // MMA completion
  __shared__ __align__(8) uint64_t abar;   // operator tiles landed
  __shared__ uint32_t tmem_base;
  // shared tiles (16 KB each): A hi, A lo of each row tile, then B hi, B lo
  uint8_t* tB = dsm + 2 * kMT * kTileBytes;
  uint8_t* tB2 = tB + kTileBytes;

  // the symmetry node maps, staged in shared memory when they fit
  const int16_t* smp = smap;
  if (48 * PS * 2 <= kSmapSmem) {
    int16_t* st = (int16_t*)(dsm + smem_tiles<kMT>());
    for (int u = threadIdx.x; u < 48 * PS; u += kThreads) st[u] = smap[u];
    smp = st;
  }
  const int4 tl = tiles[blockIdx.x];
  const int4 gd = gemm[tl.x];
  const int kind = gd.w & 0xff, q = (gd.w >> 8) & 0xff, qhi = (gd.w >> 16) & 0xff;
  const int nk = kind == 0 ? 3 : 4, c0 = kind == 0 ? 0 : 3;
  const int var = (q == qhi) ? 1 : 0;
  // row tiles kMT*tl.y .. +kMT-1 (those below P)
  const int rt0 = tl.y * kMT, col0 = tl.z * kTileN;
  const int row0 = rt0 * kTileM;
  const int ncol = gd.z * nk * R;  // columns (pair, right-hand side, component)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool split = prec == 3 || prec == 4 || prec == 5;
  const int fmt = (prec == 1 || prec == 4) ? kFmtTf32 : (prec == 5 ? kFmtF16 : kFmtBf16);
  const bool tf = fmt == kFmtTf32;
  const int E = tf ? 4 : 8;    // K elements per 16-byte unit
  const int KC = 8 * E;        // K elements per chunk (128 bytes per row)

  if (tid < kTileN) {
    int gcol = col0 + tid;
    if (gcol < ncol) {
      int pr = gd.y + gcol / (nk * R), rem = gcol % (nk * R), rhs = rem / nk, c = c0 + rem % nk;
      const int64_t prow = (((int64_t)pC[pr] * 2 + var) * R + rhs) * kNCmp + c;  // packed row
      src_off[tid] = prow * P;
      col_inv[tid] = pkinv ? pkinv[prow] : 1.f;
      dst_off[tid] = ((((int64_t)pO[pr] * Q + ((k + q) % Q)) * R + rhs) * kNCmp + c) * P;
      map_off[tid] = (int32_t)psym[pr] * PS;
    } else {
      src_off[tid] = -1;
      dst_off[tid] = -1;
      map_off[tid] = 0;
      col_inv[tid] = 1.f;
    }
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&abar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = make_idesc(tf ? 2u : (fmt == kFmtF16 ? 0u : 1u));
  const float op_inv = opinv ? opinv[gd.x * 2 + kind] : 1.f;
  const uint32_t mb = smem_u32(&mbar), ab = smem_u32(&abar);
  bool ok = true;
  bool a_pending = false;  // thread 0: an operator copy not yet seen complete

  const int nchunks = (P + KC - 1) / KC;
  const int nrt = (P + kTileM - 1) / kTileM;
  const int nmt = min(kMT, nrt - rt0);  // row tiles of this CTA
  const int nparts = split ? 2 : 1;
  // moment columns: rows of the packed, already permuted moments, so each
  // column's chunk is a contiguous run.  With P a multiple of 4 every thread
  // loads its four 16-byte units of a chunk into registers; the loads of
  // chunk ch + 1 are issued as soon as the MMAs of chunk ch are, so their
  // latency overlaps the tensor-core work.
  constexpr int kU = 1024 / kThreads;
  const bool vec = (P & 3) == 0;
  float4 v[kU][2];
  auto load_b = [&](int chunk) {
    const int kb = chunk * KC;
#pragma unroll
    for (int j = 0; j < kU; ++j) {
      const int u = tid + j * kThreads;
      const int64_t so = src_off[unit_row(u)];
      const int kk = kb + unit_k16(u) * E;
#pragma unroll
      for (int g = 0; g < 2; ++g) {
        const int kq = kk + 4 * g;
        v[j][g] = (so >= 0 && 4 * g < E && kq < P) ? __ldg((const float4*)(pk + so + kq))
                                                    : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
  };
  if (vec) load_b(0);
  for (int ch = 0; ch < nchunks && ok; ++ch) {
    const int k0 = ch * KC;
    // operator rows: the pre-converted images of this chunk (hi and lo parts
    // contiguous, nparts x 16 KB per row tile) brought in by the TMA bulk-copy
    // engine while the threads gather the moments; the previous chunk's MMAs
    // have completed, so the tiles are free
    if (tid == 0) {
      mbar_expect_tx(ab, (uint32_t)(nmt * nparts * kTileBytes));
      for (int mt = 0; mt < nmt; ++mt) {
        const uint4* src = img + ((((int64_t)gd.x * 2 + kind) * nrt + rt0 + mt) * nchunks + ch) * nparts * 1024;
        bulk_g2s(smem_u32(dsm + 2 * mt * kTileBytes), src, (uint32_t)(nparts * kTileBytes), ab);
      }
      a_pending = true;
    }
    // convert and store this chunk's moment columns (already in registers
    // when P is a multiple of 4)
    if (vec) {
#pragma unroll
      for (int j = 0; j < kU; ++j) {
        const int u = tid + j * kThreads;
        const float x[8] = {v[j][0].x, v[j][0].y, v[j][0].z, v[j][0].w, v[j][1].x, v[j][1].y, v[j][1].z, v[j][1].w};
        uint4 hi, lo;
        split_any(fmt, x, hi, lo);
        ((uint4*)tB)[u] = hi;
        if (split) ((uint4*)tB2)[u] = lo;
      }
    } else {
      for (int u = tid; u < 1024; u += kThreads) {
        const int64_t so = src_off[unit_row(u)];
        const int kk = k0 + unit_k16(u) * E;
        float x[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) x[e] = (so >= 0 && e < E && kk + e < P) ? pk[so + kk + e] : 0.f;
        uint4 hi, lo;
        split_any(fmt, x, hi, lo);
        ((uint4*)tB)[u] = hi;
        if (split) ((uint4*)tB2)[u] = lo;
      }
    }
    fence_async_smem();
    __syncthreads();
    bool a_ok = true;
    if (tid == 0) {
      a_ok = mbar_wait(ab, (uint32_t)(ch & 1));
      a_pending = !a_ok;
      tc_fence_after();
      const uint32_t b0 = smem_u32(tB), b1 = smem_u32(tB2);
      for (int mt = 0; a_ok && mt < nmt; ++mt) {
        const uint32_t a0 = smem_u32(dsm + 2 * mt * kTileBytes), a1 = a0 + kTileBytes;
        const uint32_t d = tmem + (uint32_t)(mt * kTileN);  // this row tile's accumulator columns
        for (int s = 0; s < 4; ++s) {
          uint32_t acc = (ch > 0 || s > 0) ? 1u : 0u;
          uint32_t off = 256u * s;  // two core matrices (32 bytes of K) per instruction
          if (tf) {
            mma_tf32(d, make_desc(a0 + off), make_desc(b0 + off), idesc, acc);
            if (split) {
              mma_tf32(d, make_desc(a0 + off), make_desc(b1 + off), idesc, 1u);
              mma_tf32(d, make_desc(a1 + off), make_desc(b0 + off), idesc, 1u);
            }
          } else {
            mma_f16(d, make_desc(a0 + off), make_desc(b0 + off), idesc, acc);
            if (split) {
              mma_f16(d, make_desc(a0 + off), make_desc(b1 + off), idesc, 1u);
              mma_f16(d, make_desc(a1 + off), make_desc(b0 + off), idesc, 1u);
            }
          }
        }
      }
      mma_commit(mb);
    }
    if (vec && ch + 1 < nchunks) load_b(ch + 1);
    // the next chunk overwrites the tiles: wait for the MMAs to finish; the
    // verdict is made uniform across the CTA before anyone acts on it
    // (with no MMA issued the commit arrives at once)
    bool mine = mbar_wait(mb, (uint32_t)(ch & 1)) && a_ok;
    ok = __syncthreads_and(mine) != 0;
    if (!ok) {
      if (tid == 0) atomicExch(err, 1);
      // give the tensor core and the copy engine a last bounded chance to
      // drain this chunk before TMEM is freed and the CTA exits
      mbar_wait(mb, (uint32_t)(ch & 1));
      if (tid == 0 && a_pending) mbar_wait(ab, (uint32_t)(ch & 1));
    }
  }
  tc_fence_after();
  // With both 128-row tiles of a 256-row operator in this CTA every column's
  // P outputs are here: they are placed, unscaled and un-permuted, into a
  // staging row of P floats in the (now free) operand tiles, and each
  // column's row is added to the local coefficients with one bulk reduction
  // by the copy engine (cp.reduce.async.bulk ... add.f32), in place of P / 4
  // 16-byte atomics.  64 columns are staged at a time.
  // (a tile with few valid columns, the last of a small GEMM, keeps the
  // per-column atomics: the staging's cost does not shrink with the columns)
  const bool bulk = kMT == 2 && pt == 4 && nmt * kTileM >= P && (int64_t)P * 4 * 64 <= smem_tiles<kMT>() &&
                    ncol - col0 >= 32;
  if (ok && bulk) {
    float* stage = (float*)dsm;  // [64][P]
    const int q4 = warp & 3, mt = warp >> 2;
    const int r = row0 + mt * kTileM + q4 * 32 + lane;
    for (int h = 0; h < 2; ++h) {
      if (mt < nmt) {
        for (int j0 = 0; j0 < 64; j0 += 16) {
          uint32_t v[16];
          const uint32_t addr = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(mt * kTileN + 64 * h + j0);
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
              "%14, %15}, [%16];"
              : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
              : "r"(addr));
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          if (r < P) {
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) {
              const int n = 64 * h + j0 + jj;
              if (col0 + n < ncol)  // a column past the GEMM has no target (and is not added)
                stage[(j0 + jj) * P + smp[map_off[n] + (r >> 2)] * 4 + (r & 3)] =
                    __uint_as_float(v[jj]) * (op_inv * col_inv[n]);
            }
          }
        }
      }
      fence_async_smem();
      __syncthreads();
      if (tid < 64) {
        const int n = 64 * h + tid;
        if (col0 + n < ncol) bulk_reduce_add_f32(loc + dst_off[n], smem_u32(stage + tid * P), (uint32_t)(P * 4));
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");  // the stage may be overwritten
      }
      __syncthreads();
    }
    if (tid < 64) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  }
  for (int mt = 0; ok && !bulk && mt < nmt; ++mt) {
    const int q4 = warp & 3, cb = (warp >> 2) * 64;
    const int r = row0 + mt * kTileM + q4 * 32 + lane;
    for (int j0 = 0; j0 < 64; j0 += 16) {
      uint32_t v[16];
      uint32_t addr = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(mt * kTileN + cb + j0);
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
        float val = __uint_as_float(v[jj]) * (op_inv * col_inv[n]);
        const bool col_ok = col0 + n < ncol;
        if (pt == 4) {
          float v1 = __shfl_down_sync(0xffffffffu, val, 1);
          float v2 = __shfl_down_sync(0xffffffffu, val, 2);
          float v3 = __shfl_down_sync(0xffffffffu, val, 3);
          if (col_ok && (lane & 3) == 0 && r < P) {
            int ap = r >> 2;
            float* dst = loc + dst_off[n] + (int64_t)smp[map_off[n] + ap] * 4;
            atomicAdd((float4*)dst, make_float4(val, v1, v2, v3));
          }
        } else if (col_ok && r < P) {
          int ap = r / pt, m = r - ap * pt;
          atomicAdd(loc + dst_off[n] + (int64_t)smp[map_off[n] + ap] * pt + m, val);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

// Symmetry-permuted moments of one gating event.  Row
// ((combo * 2 + var) * R + rhs) * kNC + c of pk is the B column shared by
// every interaction pair whose source cell and cube symmetry are those of
// combo: pk[row][node * pt + t] = mom[S][k & 1][var][rhs][c][smap[sym][node] * pt + t].
// One thread per (row, spatial node); the writes of a warp are contiguous.
__global__ void k_m2l_pack(const int32_t* cS, const int16_t* csym, int64_t nrows, const int16_t* smap,
                           const float* mom, int k, int R, int PS, int pt, float* pk) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= nrows * PS) return;
  const int64_t row = g / PS;
  const int node = (int)(g - row * PS);
  const int64_t per = 2LL * R * kNCmp;  // rows per combo: (var, rhs, component)
  const int64_t combo = row / per, rem = row - combo * per;
  const int P = PS * pt;
  const float* src =
      mom + (((int64_t)cS[combo] * 2 + (k & 1)) * per + rem) * P + (int64_t)smap[csym[combo] * PS + node] * pt;
  float* dst = pk + row * P + (int64_t)node * pt;
  if (pt == 4) {
    *(float4*)dst = __ldg((const float4*)src);
  } else {
    for (int t = 0; t < pt; ++t) dst[t] = src[t];
  }
}

// The same for the FP16 form, with each row scaled by the power of two that
// brings its largest magnitude into [2^14, 2^15) (exact); pkinv[row] receives
// the inverse.  One warp per row: the lanes find the row's largest magnitude,
// then write the scaled row.
__global__ void k_m2l_pack_scaled(const int32_t* cS, const int16_t* csym, int64_t nrows, const int16_t* smap,
                                  const float* mom, int k, int R, int PS, int pt, float* pk, float* pkinv) {
  const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= nrows) return;  // whole warps: a warp's lanes share their row
  const int64_t per = 2LL * R * kNCmp;
  const int64_t combo = row / per, rem = row - combo * per;
  const int P = PS * pt;
  const float* base = mom + (((int64_t)cS[combo] * 2 + (k & 1)) * per + rem) * P;
  const int16_t* sm = smap + csym[combo] * PS;
  float m = 0.f;
  for (int node = lane; node < PS; node += 32) {
    const float* src = base + (int64_t)sm[node] * pt;
    for (int t = 0; t < pt; ++t) m = fmaxf(m, fabsf(src[t]));
  }
  for (int d = 16; d > 0; d >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, d));
  const int sx = f16_scale_exp(m);
  const float sc = ldexpf(1.f, sx);
  float* dst = pk + row * P;
  for (int node = lane; node < PS; node += 32) {
    const float* src = base + (int64_t)sm[node] * pt;
    if (pt == 4) {
      const float4 v = __ldg((const float4*)src);
      *(float4*)(dst + node * 4) = make_float4(sc * v.x, sc * v.y, sc * v.z, sc * v.w);
    } else {
      for (int t = 0; t < pt; ++t) dst[node * pt + t] = sc * src[t];
    }
  }
  if (lane == 0) pkinv[row] = ldexpf(1.f, -sx);
}

// ---------------------------------------------------------------------------
// The FP16 form with the operator resident in shared memory (P <= 256).
//
// A work unit is one 128-row tile of one operator (GEMM g, row tile rt) and a
// run of up to kResRun consecutive 128-column tiles of its B.  The CTA brings
// the unit's operator rows in once (hi and lo parts of every K chunk, by TMA
// bulk copies) and streams the column tiles through a three-stage ring:
//  - warps 0-3 copy each (column tile, K chunk) item of the packed moments,
//    already scaled and split into FP16 hi and lo by k_m2l_pack_f16, into a
//    ring stage with 16-byte cp.async copies, up to three items ahead of the
//    tensor core; each thread's copies arrive on the stage's barrier when
//    they land (cp.async.mbarrier.arrive), so the producers never wait on
//    their own copies;
//  - one thread of warp 4 issues the item's tcgen05 MMAs into one of two
//    128-column TMEM accumulators, commits to the stage's barrier (which frees
//    the stage), and after a tile's last chunk to the accumulator's barrier;
//  - warps 5-8 drain each finished accumulator (tcgen05.ld), unscale, and add
//    it to the local coefficients while the next tile accumulates in the other.
// The CTA is persistent over units blockIdx.x, blockIdx.x + gridDim.x, ...
// Every wait is bounded; a timeout sets *err, raises a shared abort flag
// that ends every role's loop, and the CTA drains its copies and MMAs before
// freeing TMEM.
constexpr int kResThreads = 288;
constexpr int kResMaxCh = 4;  // K chunks of 64 halves: P <= 256
constexpr int kResStages = 3;
constexpr int kResStage = 2 * kTileBytes;
constexpr int kResSmem = kResMaxCh * 2 * kTileBytes + kResStages * kResStage;

struct ResUnit {
  int g, rt, ct0, nct;
  int op, kind, q, nk, c0, var, ncol, pbase;
};
__device__ __forceinline__ ResUnit res_unit(const int4* gemm, const int4* units, int u, int R) {
  ResUnit U;
  const int4 un = units[u];
  U.g = un.x;
  U.rt = un.y;
  U.ct0 = un.z;
  U.nct = un.w;
  const int4 gd = gemm[U.g];
  U.op = gd.x;
  U.pbase = gd.y;
  U.kind = gd.w & 0xff;
  U.q = (gd.w >> 8) & 0xff;
  const int qhi = (gd.w >> 16) & 0xff;
  U.nk = U.kind == 0 ? 3 : 4;
  U.c0 = U.kind == 0 ? 0 : 3;
  U.var = U.q == qhi ? 1 : 0;
  U.ncol = gd.z * U.nk * R;
  return U;
}

__global__ void __launch_bounds__(kResThreads, 1)
    k_m2l_res(const int4* gemm, const int4* units, int nunits, const uint4* img, int P, int P16, int pt, int PS,
              const int32_t* pO, const int32_t* pC, const int16_t* psym, const int16_t* smap, const __half* pk16,
              int k, float* loc, int Q, int R, const float* opinv, const float* pkinv, int32_t* err) {
  extern __shared__ __align__(1024) uint8_t dsm[];
  uint8_t* sA = dsm;                               // [chunk][hi, lo][16 KB]
  uint8_t* sB = dsm + kResMaxCh * 2 * kTileBytes;  // [stage][hi, lo][16 KB]
  __shared__ __align__(8) uint64_t a_full, b_full[kResStages], mma_done[kResStages], acc_full[2], acc_empty[2];
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nch = P16 / 64, nrt = (P + kTileM - 1) / kTileM;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&a_full)));
    for (int i = 0; i < kResStages; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" ::"r"(smem_u32(&b_full[i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mma_done[i])));
    }
    for (int i = 0; i < 2; ++i) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&acc_full[i])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" ::"r"(smem_u32(&acc_empty[i])));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_flag = 0;
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
  auto fail = [&]() {
    if (!abort_flag) {
      abort_flag = 1;
      atomicExch(err, 1);
    }
  };

  if (warp < 4) {
    // ---- producers: cp.async of the packed FP16 moments into the ring ----
    const int tid = threadIdx.x;
    const int k16 = (tid >> 3) & 7;  // this thread's 16-byte column along K (the same for its 8 units)
    int64_t g_item = 0;
    for (int u = blockIdx.x; u < nunits && !abort_flag; u += gridDim.x) {
      const ResUnit U = res_unit(gemm, units, u, R);
      for (int t = 0; t < U.nct && !abort_flag; ++t) {
        const int col0 = (U.ct0 + t) * kTileN;
        // units tid + 128 i (i < 8) of a part: row ((tid >> 6) + 2 i) * 8 + (tid & 7)
        int64_t srow[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int r = (((tid >> 6) + 2 * i) << 3) | (tid & 7);
          const int gcol = col0 + r;
          srow[i] = -1;
          if (gcol < U.ncol) {
            const int pr = U.pbase + gcol / (U.nk * R), rem = gcol % (U.nk * R);
            const int64_t prow = (((int64_t)pC[pr] * 2 + U.var) * R + rem / U.nk) * kNCmp + U.c0 + rem % U.nk;
            srow[i] = prow * 2 * P16;
          }
        }
        for (int ch = 0; ch < nch && !abort_flag; ++ch, ++g_item) {
          const int st = (int)(g_item % kResStages);
          const uint32_t ph = (uint32_t)((g_item / kResStages) & 1);  // this use's phase of the stage
          // the stage was last read by the MMAs of item g_item - kResStages
          if (g_item >= kResStages && !mbar_wait(smem_u32(&mma_done[st]), ph ^ 1u)) {
            fail();
            break;
          }
          const uint32_t base = smem_u32(sB + st * kResStage);
#pragma unroll
          for (int part = 0; part < 2; ++part)
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              const int uu = tid + 128 * i;
              const bool v = srow[i] >= 0;
              const __half* src = v ? pk16 + srow[i] + part * P16 + ch * 64 + k16 * 8 : pk16;
              cp_async16_zfill(base + part * kTileBytes + uu * 16, src, v ? 16u : 0u);
            }
          // arrive on the stage's barrier once this thread's copies have landed
          asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(&b_full[st]))
                       : "memory");
        }
      }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
  } else if (warp == 4) {
    // ---- the MMA issuer: the whole warp runs the loop (its waits and their
    // verdicts agreed by vote), lane 0 issues the copies, MMAs and commits ----
    const uint32_t idesc = make_idesc(0u);  // FP16 operands in kind::f16
    auto wait_all = [&](uint64_t* bar, uint32_t parity) {
      return __all_sync(0xffffffffu, mbar_wait(smem_u32(bar), parity));
    };
    int64_t g_item = 0, j = 0;
    uint32_t a_par = 0;
    bool issued = false;  // an MMA commit may be outstanding
    for (int u = blockIdx.x; u < nunits && !__any_sync(0xffffffffu, abort_flag != 0); u += gridDim.x) {
      const ResUnit U = res_unit(gemm, units, u, R);
      // the operator rows are overwritten only after the previous unit's MMAs
      if (g_item > 0 &&
          !wait_all(&mma_done[(g_item - 1) % kResStages], (uint32_t)(((g_item - 1) / kResStages) & 1))) {
        fail();
        break;
      }
      if (lane == 0) {
        const uint4* src = img + (((int64_t)U.op * 2 + U.kind) * nrt + U.rt) * nch * 2 * 1024;
        mbar_expect_tx(smem_u32(&a_full), (uint32_t)(nch * 2 * kTileBytes));
        for (int ch = 0; ch < nch; ++ch)
          bulk_g2s(smem_u32(sA + ch * 2 * kTileBytes), src + (int64_t)ch * 2 * 1024, 2 * kTileBytes,
                   smem_u32(&a_full));
      }
      __syncwarp();
      if (!wait_all(&a_full, a_par)) {
        fail();
        // the copy engine may still write the operator tiles: give it a last bounded chance
        wait_all(&a_full, a_par);
        break;
      }
      a_par ^= 1;
      bool stop = false;
      for (int t = 0; t < U.nct && !stop; ++t, ++j) {
        const int b = (int)(j & 1);
        // the accumulator was last drained by the epilogue of tile j - 2
        if (j >= 2 && !wait_all(&acc_empty[b], (uint32_t)(((j >> 1) - 1) & 1))) {
          fail();
          stop = true;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(b * kTileN);
        for (int ch = 0; ch < nch; ++ch, ++g_item) {
          const int st = (int)(g_item % kResStages);
          if (!wait_all(&b_full[st], (uint32_t)((g_item / kResStages) & 1))) {
            fail();
            stop = true;
            break;
          }
          // the producers' copies (generic proxy) are read by the tensor core (async proxy)
          fence_async_smem();
          tc_fence_after();
          if (lane == 0) {
            // D[column][operator row] += moments . operator^T: the moment
            // columns are the MMA's M side, the resident operator rows its N side
            const uint32_t o0 = smem_u32(sA + ch * 2 * kTileBytes), o1 = o0 + kTileBytes;
            const uint32_t m0 = smem_u32(sB + st * kResStage), m1 = m0 + kTileBytes;
            for (int ks = 0; ks < 4; ++ks) {
              const uint32_t off = 256u * ks;  // 32 bytes of K per instruction
              mma_f16(d, make_desc(m0 + off), make_desc(o0 + off), idesc, (ch > 0 || ks > 0) ? 1u : 0u);
              mma_f16(d, make_desc(m1 + off), make_desc(o0 + off), idesc, 1u);
              mma_f16(d, make_desc(m0 + off), make_desc(o1 + off), idesc, 1u);
            }
            mma_commit(smem_u32(&mma_done[st]));
            if (ch == nch - 1) mma_commit(smem_u32(&acc_full[b]));
          }
          __syncwarp();
          issued = true;
        }
      }
      if (stop) break;
    }
    // drain: the last commit covers every MMA issued
    if (issued) wait_all(&mma_done[(g_item - 1) % kResStages], (uint32_t)(((g_item - 1) / kResStages) & 1));
  } else {
    // ---- epilogue: TMEM -> unscale -> local coefficients.  TMEM lane =
    // moment column of the tile, TMEM column = operator row, so each lane adds
    // its own column's rows: pt consecutive rows (the time nodes of one
    // spatial node) are contiguous in the local coefficients.  Control flow
    // stays uniform across each warp (tcgen05.ld is .sync.aligned): the abort
    // flag and every wait's verdict are agreed by vote ----
    const int q4 = warp & 3;  // TMEM lane quarter this warp may read
    int64_t j = 0;
    for (int u = blockIdx.x; u < nunits && !__any_sync(0xffffffffu, abort_flag != 0); u += gridDim.x) {
      const ResUnit U = res_unit(gemm, units, u, R);
      const float op_inv = opinv[U.op * 2 + U.kind];
      const int row0 = U.rt * kTileM;
      for (int t = 0; t < U.nct && !__any_sync(0xffffffffu, abort_flag != 0); ++t, ++j) {
        const int b = (int)(j & 1);
        const int gcol = (U.ct0 + t) * kTileN + q4 * 32 + lane;  // this lane's column
        int64_t dst_off = -1;
        int32_t map_off = 0;
        float ci = 0.f;
        if (gcol < U.ncol) {
          const int pr = U.pbase + gcol / (U.nk * R), rem = gcol % (U.nk * R), rhs = rem / U.nk, c = U.c0 + rem % U.nk;
          const int64_t prow = (((int64_t)pC[pr] * 2 + U.var) * R + rhs) * kNCmp + c;
          dst_off = ((((int64_t)pO[pr] * Q + ((k + U.q) % Q)) * R + rhs) * kNCmp + c) * P;
          map_off = (int32_t)psym[pr] * PS;
          ci = op_inv * pkinv[prow];
        }
        if (!__all_sync(0xffffffffu, mbar_wait(smem_u32(&acc_full[b]), (uint32_t)((j >> 1) & 1)))) {
          fail();
          break;
        }
        tc_fence_after();
        for (int j0 = 0; j0 < kTileN; j0 += 16) {
          __syncwarp();  // the lanes leave the previous group's adds at different points
          uint32_t v[16];
          const uint32_t addr = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)(b * kTileN + j0);
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
              "%14, %15}, [%16];"
              : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
              : "r"(addr));
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          const int rb = row0 + j0;  // operator row of v[0]
          if (dst_off < 0) {
          } else if (pt == 4) {
#pragma unroll
            for (int gi = 0; gi < 4; ++gi) {
              const int r = rb + 4 * gi;
              if (r < P) {
                float* dst = loc + dst_off + (int64_t)smap[map_off + (r >> 2)] * 4;
                atomicAdd((float4*)dst, make_float4(__uint_as_float(v[4 * gi]) * ci, __uint_as_float(v[4 * gi + 1]) * ci,
                                                    __uint_as_float(v[4 * gi + 2]) * ci,
                                                    __uint_as_float(v[4 * gi + 3]) * ci));
              }
            }
          } else {
#pragma unroll
            for (int jj = 0; jj < 16; ++jj) {
              const int r = rb + jj;
              if (r < P) {
                const int ap = r / pt, m = r - ap * pt;
                atomicAdd(loc + dst_off + (int64_t)smap[map_off + ap] * pt + m, __uint_as_float(v[jj]) * ci);
              }
            }
          }
        }
        tc_fence_before();
        mbar_arrive(smem_u32(&acc_empty[b]));
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256u));
}

// Packed moments of the FP16 form for k_m2l_res: row (as in k_m2l_pack) scaled
// by a power of two (k_m2l_pack_scaled) and split into FP16 hi and lo parts,
// pk16[(row * 2 + part) * P16 + e], zero past P up to P16 (a multiple of 64).
// One warp per row.
__global__ void k_m2l_pack_f16(const int32_t* cS, const int16_t* csym, int64_t nrows, const int16_t* smap,
                               const float* mom, int k, int R, int PS, int pt, int P16, __half* pk16,
                               float* pkinv) {
  const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= nrows) return;  // whole warps: a warp's lanes share their row
  const int64_t per = 2LL * R * kNCmp;
  const int64_t combo = row / per, rem = row - combo * per;
  const int P = PS * pt;
  const float* base = mom + (((int64_t)cS[combo] * 2 + (k & 1)) * per + rem) * P;
  const int16_t* sm = smap + csym[combo] * PS;
  float m = 0.f;
  for (int e = lane; e < P; e += 32) m = fmaxf(m, fabsf(base[(int64_t)sm[e / pt] * pt + e % pt]));
  for (int d = 16; d > 0; d >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, d));
  const int sx = f16_scale_exp(m);
  const float sc = ldexpf(1.f, sx);
  __half* hi = pk16 + row * 2 * P16;
  __half* lo = hi + P16;
  for (int e = lane; e < P16; e += 32) {
    const float x = e < P ? sc * base[(int64_t)sm[e / pt] * pt + e % pt] : 0.f;
    const __half h = __float2half_rn(x);
    hi[e] = h;
    lo[e] = __float2half_rn(x - __half2float(h));
  }
  if (lane == 0) pkinv[row] = ldexpf(1.f, -sx);
}

}  // namespace tdbem

// Launch the tensor-core M2L of one level event with mt (1 or 2) 128-row
// operator tiles per CTA; tiles must be the list planned for that mt.
template <int kMT>
static tdbem_status launch_m2l_tc(tdbem_ctx* c, const int4* gemm, const int4* tiles, int ntiles, const uint4* img,
                                  int P, int pt, int PS, const int32_t* pO, const int32_t* pC, const int16_t* psym,
                                  const int16_t* smap, const float* pk, int k, float* loc, int Q, int R, int prec,
                                  const float* opinv, const float* pkinv, int32_t* err) {
  using namespace tdbem;
  static bool attr = false;
  if (!attr) {
    TDBEM_CUDA_TRY(c, cudaFuncSetAttribute(k_m2l_tc<kMT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           smem_tiles<kMT>() + kSmapSmem + 1024));
    attr = true;
  }
  if (ntiles == 0) return TDBEM_OK;
  const size_t smem = smem_tiles<kMT>() + (48 * PS * 2 <= kSmapSmem ? 48 * PS * 2 : 0) + 1024;
  k_m2l_tc<kMT><<<ntiles, kThreads, smem, c->stream>>>(gemm, tiles, img, P, pt, PS, pO, pC, psym, smap, pk, k, loc,
                                                        Q, R, prec, opinv, pkinv, err);
  TDBEM_CUDA_TRY(c, cudaGetLastError());
  return TDBEM_OK;
}

tdbem_status tdbem_m2l_tc(tdbem_ctx* c, int mt, const int4* gemm, const int4* tiles, int ntiles, const uint4* img,
                          int P, int pt, int PS, const int32_t* pO, const int32_t* pC, const int16_t* psym,
                          const int16_t* smap, const float* pk, int k, float* loc, int Q, int R, int prec,
                          const float* opinv, const float* pkinv, int32_t* err) {
  if (mt == 2)
    return launch_m2l_tc<2>(c, gemm, tiles, ntiles, img, P, pt, PS, pO, pC, psym, smap, pk, k, loc, Q, R, prec, opinv,
                            pkinv, err);
  return launch_m2l_tc<1>(c, gemm, tiles, ntiles, img, P, pt, PS, pO, pC, psym, smap, pk, k, loc, Q, R, prec, opinv,
                          pkinv, err);
}

// Convert the FP32 operators of one level into the tensor-core images read by
// k_m2l_tc (allocated here, owned by the context).  The FP16 form scales each
// operator by a power of two first; *opinv (allocated here, 2 nop floats)
// then holds the inverse scales, and is null for the other forms.
tdbem_status tdbem_m2l_tc_images(tdbem_ctx* c, const float* ops, int nop, int P, int prec, uint4** img,
                                 float** opinv) {
  using namespace tdbem;
  *img = nullptr;
  *opinv = nullptr;
  if (nop == 0) return TDBEM_OK;
  const int fmt = (prec == TDBEM_P_TF32 || prec == TDBEM_P_TF32X3) ? kFmtTf32
                                                                      : (prec == TDBEM_P_F16X3 ? kFmtF16 : kFmtBf16);
  const bool split = prec == TDBEM_P_TF32X3 || prec == TDBEM_P_BF16X3 || prec == TDBEM_P_F16X3;
  const int KC = fmt == kFmtTf32 ? 32 : 64;
  const int nrt = (P + kTileM - 1) / kTileM, nch = (P + KC - 1) / KC, nparts = split ? 2 : 1;
  const int64_t nunits = (int64_t)nop * 2 * nrt * nch * nparts * 1024;
  tdbem_status s = c->dalloc(img, nunits);
  if (s) return s;
  float* scale = nullptr;
  if (fmt == kFmtF16) {
    if ((s = c->dalloc(&scale, 2 * (int64_t)nop)) || (s = c->dalloc(opinv, 2 * (int64_t)nop))) return s;
    k_m2l_opscale<<<(unsigned)(2 * nop), 256, 0, c->stream>>>(ops, P, scale, *opinv);
    TDBEM_CUDA_TRY(c, cudaGetLastError());
  }
  k_m2l_images<<<(unsigned)((nunits + 255) / 256), 256, 0, c->stream>>>(ops, nunits, P, nrt, nch, nparts, fmt, scale,
                                                                        *img);
  TDBEM_CUDA_TRY(c, cudaGetLastError());
  return TDBEM_OK;
}

// Pack the moments of one level event for k_m2l_tc: ncombo (source cell,
// symmetry) combinations, rows of P floats each (see k_m2l_pack).
tdbem_status tdbem_m2l_pack(tdbem_ctx* c, const int32_t* cS, const int16_t* csym, int ncombo, const int16_t* smap,
                            const float* mom, int k, int R, int PS, int pt, float* pk, float* pkinv) {
  using namespace tdbem;
  const int64_t nrows = (int64_t)ncombo * 2 * R * kNCmp;
  if (nrows == 0) return TDBEM_OK;
  if (pkinv) {
    k_m2l_pack_scaled<<<(unsigned)((nrows * 32 + 255) / 256), 256, 0, c->stream>>>(cS, csym, nrows, smap, mom, k, R,
                                                                                   PS, pt, pk, pkinv);
    TDBEM_CUDA_TRY(c, cudaGetLastError());
    return TDBEM_OK;
  }
  const int64_t nth = nrows * PS;
  k_m2l_pack<<<(unsigned)((nth + 255) / 256), 256, 0, c->stream>>>(cS, csym, nrows, smap, mom, k, R, PS, pt, pk);
  TDBEM_CUDA_TRY(c, cudaGetLastError());
  return TDBEM_OK;
}

// The FP16 form with resident operator rows (k_m2l_res): units [u0, u0 + n) of
// the level's unit list, on a persistent grid of at most one CTA per SM and at
// most max_ctas CTAs (0: no further limit), or with max_ctas < 0 one CTA per
// unit (the hardware then schedules the units among other streams' work).
tdbem_status tdbem_m2l_res(tdbem_ctx* c, const int4* gemm, const int4* units, int u0, int n, const uint4* img, int P,
                           int pt, int PS, const int32_t* pO, const int32_t* pC, const int16_t* psym,
                           const int16_t* smap, const __half* pk16, int k, float* loc, int Q, int R,
                           const float* opinv, const float* pkinv, int32_t* err, int max_ctas) {
  using namespace tdbem;
  static bool attr = false;
  static int nsm = 0;
  if (!attr) {
    TDBEM_CUDA_TRY(c, cudaFuncSetAttribute(k_m2l_res, cudaFuncAttributeMaxDynamicSharedMemorySize, kResSmem));
    TDBEM_CUDA_TRY(c, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device));
    attr = true;
  }
  if (n <= 0) return TDBEM_OK;
  const int P16 = (P + 63) / 64 * 64;
  if (P16 > 64 * kResMaxCh) {
    c->set_error("fast: resident-operator M2L needs P <= 256");
    return TDBEM_EINVAL;
  }
  const int grid = max_ctas < 0 ? n : std::min(n, max_ctas > 0 ? std::min(max_ctas, nsm) : nsm);
  k_m2l_res<<<grid, kResThreads, kResSmem, c->stream>>>(gemm, units + u0, n, img, P, P16, pt, PS, pO, pC, psym, smap,
                                                         pk16, k, loc, Q, R, opinv, pkinv, err);
  TDBEM_CUDA_TRY(c, cudaGetLastError());
  return TDBEM_OK;
}

tdbem_status tdbem_m2l_pack_f16(tdbem_ctx* c, const int32_t* cS, const int16_t* csym, int ncombo,
                                const int16_t* smap, const float* mom, int k, int R, int PS, int pt, __half* pk16,
                                float* pkinv) {
  using namespace tdbem;
  const int64_t nrows = (int64_t)ncombo * 2 * R * kNCmp;
  if (nrows == 0) return TDBEM_OK;
  const int P16 = (PS * pt + 63) / 64 * 64;
  k_m2l_pack_f16<<<(unsigned)((nrows * 32 + 255) / 256), 256, 0, c->stream>>>(cS, csym, nrows, smap, mom, k, R, PS,
                                                                              pt, P16, pk16, pkinv);
  TDBEM_CUDA_TRY(c, cudaGetLastError());
  return TDBEM_OK;
}
