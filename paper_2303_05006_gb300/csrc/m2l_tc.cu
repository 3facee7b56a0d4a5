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

namespace tdbem {

namespace {

constexpr int kTileM = 128, kTileN = 128, kThreads = 256;
constexpr int kTileBytes = 16384;  // one 128 x 128-byte operand tile
// per CTA: kMT 128-row operator tiles sharing one gathered B, one 128-column
// TMEM accumulator each; shared memory A hi/lo per row tile, then B hi/lo
template <int kMT>
constexpr int smem_tiles() { return (2 * kMT + 2) * kTileBytes; }
constexpr int kNCmp = 7;
constexpr int kSmapSmem = 24 * 1024;  // largest symmetry-map table staged in shared memory

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

// arrive on mbar (one of its expected arrivals) and add bytes to the
// transaction count the current phase waits for
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

// bulk copy (TMA, no tensor map) of bytes from global to this CTA's shared
// memory, counted on mbar; both addresses 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ uint32_t f32_to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// 16-byte unit u of a 128-row x 128-byte K-major tile: its row and its
// 16-byte column along K (the unit's byte offset in the tile is 16 u)
__device__ __forceinline__ int unit_row(int u) { return ((u >> 6) << 3) | (u & 7); }
__device__ __forceinline__ int unit_k16(int u) { return (u >> 3) & 7; }

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
  for (int mt = 0; ok && mt < nmt; ++mt) {
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
