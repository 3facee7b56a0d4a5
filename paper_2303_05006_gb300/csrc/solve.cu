// solve.cu -- the per-step solve Z0 J^{alpha-1} = R^{alpha-1} (paper eq. solve).
//
// Z0 = Zt^(1) couples only edges whose supports come within c dt of each other
// (tau = 1 - r/(c dt) > 0), so it is sparse and close to diagonal (section
// 2.6).  It is stored in CSR and solved with Jacobi-preconditioned BiCGStab to
// a relative residual solve_tol, starting from the cubic extrapolation of the
// last four currents.
//
// The whole Krylov loop runs in ONE launch of a thread-block cluster: each of
// the cluster's CTAs owns a contiguous block of rows, vectors live in global
// memory (L2-resident), and every reduction is combined through distributed
// shared memory after a hardware cluster barrier.  There is no host round trip
// and no software spin-wait; all CTAs take identical branch decisions because
// they read the same reduced values.
#include <cooperative_groups.h>

#include <algorithm>
#include <vector>

#include "internal.h"

namespace cg = cooperative_groups;

namespace tdbem {

constexpr int kSolveThreads = 512;

__global__ void k_z0_count(const int16_t* m_lo, const uint8_t* nlag, int64_t ne, int32_t* cnt) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= ne) return;
  int c = 0;
  for (int64_t j = 0; j < ne; ++j) {
    int64_t p = i * ne + j;
    if (m_lo[p] == 1 && nlag[p] > 0) ++c;
  }
  cnt[i] = c;
}

__global__ void k_z0_fill(const int16_t* m_lo, const uint8_t* nlag, const int64_t* off, const double* val, int64_t ne,
                          const int32_t* ptr, int32_t* col, double* z, double* inv_diag) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= ne) return;
  int k = ptr[i];
  double dg = 0.0;
  for (int64_t j = 0; j < ne; ++j) {
    int64_t p = i * ne + j;
    if (m_lo[p] == 1 && nlag[p] > 0) {
      col[k] = (int32_t)j;
      z[k] = val[off[p]];
      if (j == i) dg = z[k];
      ++k;
    }
  }
  inv_diag[i] = (dg != 0.0) ? 1.0 / dg : 1.0;
}

__global__ void k_z0_csr(const int64_t* row_ptr, const int32_t* col, const int16_t* m_lo, const uint8_t* nlag,
                         const int64_t* off, const double* val, int64_t ne, const int32_t* ptr, int32_t* zcol, double* z,
                         double* inv_diag, int32_t* cnt, int fill) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= ne) return;
  int k = fill ? ptr[i] : 0;
  double dg = 0.0;
  for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
    if (m_lo[p] != 1 || nlag[p] == 0) continue;
    if (fill) {
      zcol[k] = col[p];
      z[k] = val[off[p]];
      if (col[p] == i) dg = z[k];
    }
    ++k;
  }
  if (fill)
    inv_diag[i] = (dg != 0.0) ? 1.0 / dg : 1.0;
  else
    cnt[i] = k;
}

struct SolveArgs {
  const int32_t* ptr;
  const int32_t* col;
  const double* val;      // Z0, FP64 (outer residual)
  const float* val32;     // Z0, FP32 (inner iterations)
  const float* inv_diag;  // Jacobi preconditioner
  const double* b;
  double* x;        // solution (also written to the ring)
  double* ring;     // [ne][L]
  int32_t L;
  int32_t alpha;    // solving J^{alpha-1}
  int32_t warm;     // 1: cubic extrapolation of J^{alpha-2..alpha-5}
  double* w;        // FP64 residual [ne], then 9 FP32 vectors [9][ne]
  int64_t ne;
  double tol;
  int32_t maxit;    // cap on the total inner iterations
  int32_t* status;  // [0] inner iterations, [1] converged flag, [2] misses, [3] iteration total
  double* resid;    // [0] final relative residual
};

// Block sums of NV values; the totals end up in thread 0.
template <int NV>
__device__ __forceinline__ void block_sums(double (&v)[NV], double* sm) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k)
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) sm[wid * NV + k] = v[k];
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = (lane < nw) ? sm[lane * NV + k] : 0.0;
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      v[k] = s;
    }
  }
  __syncthreads();
}

// Cluster-wide sums: thread 0 publishes its block totals in this CTA's slot
// (two alternating slots, so a slot is rewritten only after one more cluster
// barrier than its readers have passed); after the hardware cluster barrier,
// lane r of warp 0 reads CTA r's slot through distributed shared memory, the
// warp sums them in a fixed order and broadcasts through shared memory.
template <int NV>
__device__ __forceinline__ void cluster_sums(cg::cluster_group& cl, double (&v)[NV], double (*slots)[4],
                                             double* bc, int& phase) {
  double* slot = slots[phase & 1];
  ++phase;
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) slot[k] = v[k];
  cl.sync();
  if (threadIdx.x < 32) {
    unsigned nb = cl.num_blocks();
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double s = threadIdx.x < nb ? cl.map_shared_rank(slot, threadIdx.x)[k] : 0.0;
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if (threadIdx.x == 0) bc[k] = s;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = bc[k];
}

__device__ __forceinline__ double spmv_row64(const SolveArgs& A, int64_t i, const double* x) {
  double s = 0.0;
  for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) s += A.val[k] * x[A.col[k]];
  return s;
}

__device__ __forceinline__ float spmv_row32(const SolveArgs& A, int64_t i, const float* x) {
  float s0 = 0.f, s1 = 0.f;
  int k = A.ptr[i], e = A.ptr[i + 1];
  for (; k + 1 < e; k += 2) {
    s0 += A.val32[k] * x[A.col[k]];
    s1 += A.val32[k + 1] * x[A.col[k + 1]];
  }
  if (k < e) s0 += A.val32[k] * x[A.col[k]];
  return s0 + s1;
}

// Mixed-precision solve of Z0 x = b: FP64 residual r = b - Z0 x (iterative
// refinement) around an FP32 Jacobi-preconditioned BiCGStab for the
// correction, inner relative tolerance 1e-5.  Z0 is well conditioned (about 2
// on the test spheres), so each refinement gains five to six digits and two to
// three refinements reach 1e-13.
__global__ void __launch_bounds__(kSolveThreads) k_bicgstab(SolveArgs A) {
  cg::cluster_group cl = cg::this_cluster();
  __shared__ double red[32 * 4];
  __shared__ double slots[2][4];
  __shared__ double bc[4];
  int phase = 0;
  const int64_t ne = A.ne;
  const unsigned nb = cl.num_blocks(), rk = cl.block_rank();
  const int64_t rows = (ne + nb - 1) / nb;
  const int64_t r0 = rk * rows, r1 = min(ne, r0 + rows);
  double* r64 = A.w;
  float* f = (float*)(A.w + ne);
  float* r = f;
  float* rh = f + ne;
  float* p = f + 2 * ne;
  float* v = f + 3 * ne;
  float* s = f + 4 * ne;
  float* t = f + 5 * ne;
  float* ph = f + 6 * ne;
  float* sh = f + 7 * ne;
  float* d = f + 8 * ne;
  const int L = A.L, msk = A.L - 1;
  for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
    double x0 = 0.0;
    if (A.warm) {
      const double* J = A.ring + i * L;
      int b = A.alpha - 2;  // J^{alpha-2}, J^{alpha-3}, ... (zero before step 0)
      double j1 = b >= 0 ? J[b & msk] : 0.0, j2 = b >= 1 ? J[(b - 1) & msk] : 0.0;
      double j3 = b >= 2 ? J[(b - 2) & msk] : 0.0, j4 = b >= 3 ? J[(b - 3) & msk] : 0.0;
      x0 = 4.0 * j1 - 6.0 * j2 + 4.0 * j3 - j4;
    }
    A.x[i] = x0;
  }
  cl.sync();
  double bb = -1.0, rr = 0.0;
  int inner_total = 0;
  bool conv = false;
  for (int outer = 0; outer < 8; ++outer) {
    // FP64 residual
    double q2[2] = {0.0, 0.0};
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      double ri = A.b[i] - spmv_row64(A, i, A.x);
      r64[i] = ri;
      q2[0] += ri * ri;
      q2[1] += A.b[i] * A.b[i];
    }
    block_sums<2>(q2, red);
    cluster_sums<2>(cl, q2, slots, bc, phase);
    rr = q2[0];
    if (bb < 0) bb = q2[1];
    if (rr <= A.tol * A.tol * bb) {
      conv = true;
      break;
    }
    if (inner_total >= A.maxit) break;
    // FP32 BiCGStab for Z0 d = r64, relative tolerance 1e-5
    double q1[2] = {0.0, 0.0};
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      float ri = (float)(r64[i] * (1.0 / sqrt(rr)));  // unit-norm right-hand side
      r[i] = ri;
      rh[i] = ri;
      p[i] = 0.f;
      v[i] = 0.f;
      d[i] = 0.f;
      q1[0] += (double)ri * ri;
    }
    block_sums<1>(*(double(*)[1])q1, red);
    cluster_sums<1>(cl, *(double(*)[1])q1, slots, bc, phase);
    double rho = q1[0], rho_old = 1.0, alp = 1.0, om = 1.0;
    const double tin2 = 1e-10 * q1[0];
    for (int it = 0; it < 40 && inner_total < A.maxit; ++it) {
      ++inner_total;
      if (rho == 0.0) break;
      float beta = (float)((rho / rho_old) * (alp / om));
      float omf = (float)om;
      for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        float pi = r[i] + beta * (p[i] - omf * v[i]);
        p[i] = pi;
        ph[i] = pi * A.inv_diag[i];
      }
      cl.sync();
      double e1[1] = {0.0};
      for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        float vi = spmv_row32(A, i, ph);
        v[i] = vi;
        e1[0] += (double)(rh[i] * vi);
      }
      block_sums<1>(e1, red);
      cluster_sums<1>(cl, e1, slots, bc, phase);
      if (e1[0] == 0.0) break;
      alp = rho / e1[0];
      float alf = (float)alp;
      double e2[1] = {0.0};
      for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        float si = r[i] - alf * v[i];
        s[i] = si;
        sh[i] = si * A.inv_diag[i];
        e2[0] += (double)(si * si);
      }
      block_sums<1>(e2, red);
      cluster_sums<1>(cl, e2, slots, bc, phase);  // also orders sh for the SpMV below
      if (e2[0] <= tin2) {
        for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) d[i] += alf * ph[i];
        break;
      }
      double e3[2] = {0.0, 0.0};
      for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        float ti = spmv_row32(A, i, sh);
        t[i] = ti;
        e3[0] += (double)(ti * s[i]);
        e3[1] += (double)(ti * ti);
      }
      block_sums<2>(e3, red);
      cluster_sums<2>(cl, e3, slots, bc, phase);
      if (e3[1] == 0.0) break;
      om = e3[0] / e3[1];
      omf = (float)om;
      double e4[2] = {0.0, 0.0};
      for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        d[i] += alf * ph[i] + omf * sh[i];
        float ri = s[i] - omf * t[i];
        r[i] = ri;
        e4[0] += (double)(ri * ri);
        e4[1] += (double)(rh[i] * ri);
      }
      block_sums<2>(e4, red);
      cluster_sums<2>(cl, e4, slots, bc, phase);
      rho_old = rho;
      rho = e4[1];
      if (e4[0] <= tin2 || om == 0.0) break;
    }
    // x += |r| d (own rows), then a barrier before the next residual reads x
    const double sc = sqrt(rr);
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) A.x[i] += sc * (double)d[i];
    cl.sync();
  }
  for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) A.ring[i * L + ((A.alpha - 1) & msk)] = A.x[i];
  if (rk == 0 && threadIdx.x == 0) {
    A.status[0] = inner_total;
    A.status[1] = conv ? 1 : 0;
    A.status[2] += conv ? 0 : 1;  // solves that missed the tolerance since the last reset
    A.status[3] += inner_total;   // iterations since the last reset
    A.resid[0] = bb > 0 ? sqrt(rr / bb) : 0.0;
  }
  cl.sync();  // keep every CTA's shared slots alive until all remote reads are done
}

// ---------------------------------------------------------------------------
// Batched form: R right-hand sides at once (vectors [ne][R], RHS fastest).
// The grid is a row of thread-block clusters; cluster g solves the contiguous
// RHS slice [g*Rc, min(R, (g+1)*Rc)), Rc = ceil(R / clusters), with the same
// mixed-precision scheme as k_bicgstab and per-RHS scalars (an RHS that has
// converged keeps its iterate: its updates are masked).  Reductions are
// per-RHS: shared-memory atomics per CTA, then CTA slot r of every cluster
// member is summed through DSMEM in rank order.  The status words are
// combined over clusters with atomics; the last cluster to finish publishes
// the step's verdict (status[0] must be zero at launch).
constexpr int kMaxRhs = 64;

struct MultiArgs {
  const int32_t* ptr;
  const int32_t* col;
  const double* val;
  const float* val32;
  const float* inv_diag;
  const double* b;   // [ne][R]
  double* x;         // [ne][R]
  double* ring;      // [ne][L][R]
  int32_t L, alpha, warm, R;
  double* w;         // FP64 residual [ne][R], then 9 FP32 vectors [9][ne][R]
  int64_t ne;
  double tol;
  int32_t maxit;
  int32_t* status;   // [0] max inner iterations, [1] all converged, [2] misses, [3] total, [4..5] scratch
};

// Sum over the cluster of the per-CTA partial sums part[0..n) into out[];
// part[] is cleared for the next use.  All threads of every CTA call it.
__device__ __forceinline__ void multi_reduce(cg::cluster_group& cl, double* part, double (*slot)[kMaxRhs],
                                             double* out, int n, int& phase) {
  double* sl = slot[phase & 1];  // alternate slots: a slot is not rewritten before every CTA has read it
  ++phase;
  for (int r = threadIdx.x; r < n; r += blockDim.x) sl[r] = part[r];
  cl.sync();
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    double sacc = 0.0;
    for (unsigned k = 0; k < cl.num_blocks(); ++k) sacc += cl.map_shared_rank(sl, k)[r];
    out[r] = sacc;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < n; r += blockDim.x) part[r] = 0.0;
  __syncthreads();
}

__global__ void __launch_bounds__(kSolveThreads) k_bicgstab_multi(MultiArgs A) {
  cg::cluster_group cl = cg::this_cluster();
  __shared__ double part[kMaxRhs], part2[kMaxRhs], red1[kMaxRhs], red2[kMaxRhs];
  __shared__ double slots[2][kMaxRhs], slots2[2][kMaxRhs];
  __shared__ double rho[kMaxRhs], rho_old[kMaxRhs], alp[kMaxRhs], om[kMaxRhs], bb[kMaxRhs], nr[kMaxRhs];
  __shared__ int act[kMaxRhs], conv[kMaxRhs];
  int phase = 0, phase2 = 0;
  const int R = A.R;
  const unsigned nb = cl.num_blocks(), rk = cl.block_rank();
  const int ncl = gridDim.x / nb, cid = blockIdx.x / nb;
  const int Rc = (R + ncl - 1) / ncl;
  const int rb = cid * Rc, Rl = max(0, min(R, rb + Rc) - rb);  // this cluster's RHS slice
  const int64_t ne = A.ne;
  const int64_t rows = (ne + nb - 1) / nb;
  const int64_t r0 = rk * rows, r1 = min(ne, r0 + rows);
  const int64_t nloc = (r1 > r0 ? r1 - r0 : 0) * Rl;
  const int64_t NR = ne * R;
  double* r64 = A.w;
  float* f = (float*)(A.w + NR);
  float *rv = f, *rh = f + NR, *pv = f + 2 * NR, *vv = f + 3 * NR, *sv = f + 4 * NR, *tv = f + 5 * NR,
        *ph = f + 6 * NR, *sh = f + 7 * NR, *dv = f + 8 * NR;
  const int L = A.L, msk = L - 1;
  // element e of this CTA: row i = r0 + e / Rl, right-hand side rb + e % Rl, vector index q = i R + r
#define ELEM(e, i, l, q)            \
  const int64_t i = r0 + (e) / Rl;  \
  const int l = (int)((e) % Rl);    \
  const int64_t q = i * R + rb + l;
  for (int l = threadIdx.x; l < kMaxRhs; l += blockDim.x) {
    part[l] = part2[l] = 0.0;
    bb[l] = -1.0;
    conv[l] = 0;
    act[l] = 0;
  }
  __syncthreads();
  for (int64_t e = threadIdx.x; e < nloc; e += blockDim.x) {
    ELEM(e, i, l, q)
    double x0 = 0.0;
    if (A.warm) {
      const double* J = A.ring + i * L * R + rb + l;
      int b = A.alpha - 2;
      double j1 = b >= 0 ? J[(int64_t)(b & msk) * R] : 0.0, j2 = b >= 1 ? J[(int64_t)((b - 1) & msk) * R] : 0.0;
      double j3 = b >= 2 ? J[(int64_t)((b - 2) & msk) * R] : 0.0, j4 = b >= 3 ? J[(int64_t)((b - 3) & msk) * R] : 0.0;
      x0 = 4.0 * j1 - 6.0 * j2 + 4.0 * j3 - j4;
    }
    A.x[q] = x0;
  }
  cl.sync();
  int inner_total = 0;
  for (int outer = 0;; ++outer) {
    // FP64 residual of every RHS of the slice
    for (int64_t e = threadIdx.x; e < nloc; e += blockDim.x) {
      ELEM(e, i, l, q)
      double sacc = 0.0;
      for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) sacc += A.val[k] * A.x[(int64_t)A.col[k] * R + rb + l];
      double bi = A.b[q], ri = bi - sacc;
      r64[q] = ri;
      atomicAdd(&part[l], ri * ri);
      atomicAdd(&part2[l], bi * bi);
    }
    __syncthreads();
    multi_reduce(cl, part, slots, red1, Rl, phase);
    multi_reduce(cl, part2, slots2, red2, Rl, phase2);
    for (int l = threadIdx.x; l < Rl; l += blockDim.x) {
      if (bb[l] < 0) bb[l] = red2[l];
      nr[l] = red1[l];
      conv[l] = red1[l] <= A.tol * A.tol * bb[l];
      act[l] = !conv[l];
    }
    __syncthreads();
    int all = 1;
    for (int l = 0; l < Rl; ++l) all &= conv[l];
    if (all || outer == 8 || inner_total >= A.maxit) break;
    // FP32 Jacobi-preconditioned BiCGStab on the unit-norm residuals, relative tolerance 1e-5
    for (int64_t e = threadIdx.x; e < nloc; e += blockDim.x) {
      ELEM(e, i, l, q)
      float ri = nr[l] > 0 ? (float)(r64[q] / sqrt(nr[l])) : 0.f;
      rv[q] = ri;
      rh[q] = ri;
      pv[q] = vv[q] = dv[q] = 0.f;
      atomicAdd(&part[l], (double)ri * ri);
    }
    __syncthreads();
    multi_reduce(cl, part, slots, red1, Rl, phase);
    for (int l = threadIdx.x; l < Rl; l += blockDim.x) {
      rho[l] = red1[l];
      rho_old[l] = alp[l] = om[l] = 1.0;
      act[l] = act[l] && rho[l] > 0.0;
    }
    __syncthreads();
    for (int it = 0; it < 40 && inner_total < A.maxit; ++it) {
      int any = 0;
      for (int l = 0; l < Rl; ++l) any |= act[l];
      if (!any) break;
      ++inner_total;
      for (int64_t e = threadIdx.x; e < nloc; e += blockDim.x) {
        ELEM(e, i, l, q)
        if (!act[l]) continue;
        float beta = (float)((rho[l] / rho_old[l]) * (alp[l] / om[l]));
        float pi = rv[q] + beta * (pv[q] - (float)om[l] * vv[q]);
        pv[q] = pi;
        ph[q] = pi * A.inv_diag[i];
      }
      cl.sync();
      for (int64_t e = threadIdx.x; e < nloc; e += blockDim.x) {
        ELEM(e, i, l, q)
        if (!act[l]) continue;
        float sacc = 0.f;
        for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) sacc += A.val32[k] * ph[(int64_t)A.col[k] * R + rb + l];
        vv[q] = sacc;
        atomicAdd(&part[l], (double)(rh[q] * sacc));
      }
      __syncthreads();
      multi_reduce(cl, part, slots, red1, Rl, phase);
      for (int l = threadIdx.x; l < Rl; l += blockDim.x) {
        if (act[l] && red1[l] == 0.0) act[l] = 0;
        if (act[l]) alp[l] = rho[l] / red1[l];
      }
      __syncthreads();
      for (int64_t e = threadIdx.x; e < nloc; e += blockDim.x) {
        ELEM(e, i, l, q)
        if (!act[l]) continue;
        float si = rv[q] - (float)alp[l] * vv[q];
        sv[q] = si;
        sh[q] = si * A.inv_diag[i];
        atomicAdd(&part[l], (double)(si * si));
      }
      __syncthreads();
      multi_reduce(cl, part, slots, red1, Rl, phase);  // its cluster barrier also publishes sh
      for (int l = threadIdx.x; l < Rl; l += blockDim.x) conv[l] = act[l] && red1[l] <= 1e-10;
      __syncthreads();
      for (int64_t e = threadIdx.x; e < nloc; e += blockDim.x) {
        ELEM(e, i, l, q)
        if (!act[l]) continue;
        if (conv[l]) {
          dv[q] += (float)alp[l] * ph[q];
          continue;
        }
        float sacc = 0.f;
        for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) sacc += A.val32[k] * sh[(int64_t)A.col[k] * R + rb + l];
        tv[q] = sacc;
        atomicAdd(&part[l], (double)(sacc * sv[q]));
        atomicAdd(&part2[l], (double)(sacc * sacc));
      }
      __syncthreads();
      multi_reduce(cl, part, slots, red1, Rl, phase);
      multi_reduce(cl, part2, slots2, red2, Rl, phase2);
      for (int l = threadIdx.x; l < Rl; l += blockDim.x) {
        if (conv[l]) act[l] = 0;
        if (act[l] && red2[l] == 0.0) act[l] = 0;
        if (act[l]) om[l] = red1[l] / red2[l];
      }
      __syncthreads();
      for (int64_t e = threadIdx.x; e < nloc; e += blockDim.x) {
        ELEM(e, i, l, q)
        if (!act[l]) continue;
        dv[q] += (float)alp[l] * ph[q] + (float)om[l] * sh[q];
        float ri = sv[q] - (float)om[l] * tv[q];
        rv[q] = ri;
        atomicAdd(&part[l], (double)(ri * ri));
        atomicAdd(&part2[l], (double)(rh[q] * ri));
      }
      __syncthreads();
      multi_reduce(cl, part, slots, red1, Rl, phase);
      multi_reduce(cl, part2, slots2, red2, Rl, phase2);
      for (int l = threadIdx.x; l < Rl; l += blockDim.x) {
        if (!act[l]) continue;
        rho_old[l] = rho[l];
        rho[l] = red2[l];
        if (red1[l] <= 1e-10 || om[l] == 0.0 || rho[l] == 0.0) act[l] = 0;
      }
      __syncthreads();
    }
    for (int64_t e = threadIdx.x; e < nloc; e += blockDim.x) {
      ELEM(e, i, l, q)
      A.x[q] += sqrt(nr[l]) * (double)dv[q];
    }
    cl.sync();
  }
  int nconv = 0;
  for (int l = 0; l < Rl; ++l) nconv += conv[l] ? 1 : 0;
  for (int64_t e = threadIdx.x; e < nloc; e += blockDim.x) {
    ELEM(e, i, l, q)
    A.ring[(i * L + ((A.alpha - 1) & msk)) * R + rb + l] = A.x[q];
  }
#undef ELEM
  if (rk == 0 && threadIdx.x == 0) {
    atomicMax(&A.status[0], inner_total);
    if (nconv < Rl) atomicAdd(&A.status[4], 1);
    __threadfence();
    if (atomicAdd(&A.status[5], 1) == ncl - 1) {  // last cluster: publish the verdict
      __threadfence();
      int miss = atomicAdd(&A.status[4], 0);
      int it = atomicAdd(&A.status[0], 0);
      A.status[1] = miss == 0 ? 1 : 0;
      A.status[2] += miss == 0 ? 0 : 1;
      A.status[3] += it;
      A.status[4] = 0;
      A.status[5] = 0;
    }
  }
  cl.sync();
}

__global__ void k_z0_f32(const double* z, const double* inv_diag, int64_t nnz, int64_t ne, float* z32, float* inv32) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < nnz) z32[i] = (float)z[i];
  if (i < ne) inv32[i] = (float)inv_diag[i];
}

}  // namespace tdbem

using namespace tdbem;

static int g_cluster = 0;

static tdbem_status tdbem_z0_f32(tdbem_ctx* c) {
  tdbem_status s;
  if ((s = c->dalloc(&c->d_z0_val32, c->z0_nnz)) || (s = c->dalloc(&c->d_z0_inv32, c->ne))) return s;
  int64_t n = std::max<int64_t>(c->z0_nnz, c->ne);
  k_z0_f32<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(c->d_z0_val, c->d_z0_inv_diag, c->z0_nnz, c->ne,
                                                               c->d_z0_val32, c->d_z0_inv32);
  TDBEM_CUDA_TRY(c, cudaGetLastError());
  TDBEM_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return TDBEM_OK;
}

tdbem_status tdbem_build_z0(tdbem_ctx* c) {
  const int64_t ne = c->ne;
  const PairStore& st = c->direct;
  int32_t* d_cnt = nullptr;
  tdbem_status s;
  if ((s = c->dalloc(&d_cnt, ne)) || (s = c->dalloc(&c->d_z0_ptr, ne + 1)) ||
      (s = c->dalloc(&c->d_z0_inv_diag, ne)))
    return s;
  k_z0_count<<<(unsigned)((ne + 127) / 128), 128, 0, c->stream>>>(st.m_lo, st.nlag, ne, d_cnt);
  TDBEM_CUDA_TRY(c, cudaGetLastError());
  std::vector<int32_t> cnt(ne), ptr(ne + 1);
  TDBEM_CUDA_TRY(c, cudaMemcpyAsync(cnt.data(), d_cnt, ne * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
  TDBEM_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  ptr[0] = 0;
  for (int64_t i = 0; i < ne; ++i) ptr[i + 1] = ptr[i] + cnt[i];
  c->z0_nnz = ptr[ne];
  if ((s = c->dalloc(&c->d_z0_col, c->z0_nnz)) || (s = c->dalloc(&c->d_z0_val, c->z0_nnz))) return s;
  TDBEM_CUDA_TRY(c, cudaMemcpyAsync(c->d_z0_ptr, ptr.data(), (ne + 1) * sizeof(int32_t), cudaMemcpyHostToDevice,
                                    c->stream));
  k_z0_fill<<<(unsigned)((ne + 127) / 128), 128, 0, c->stream>>>(st.m_lo, st.nlag, st.off, st.val, ne, c->d_z0_ptr,
                                                                 c->d_z0_col, c->d_z0_val, c->d_z0_inv_diag);
  TDBEM_CUDA_TRY(c, cudaGetLastError());
  if ((s = c->dalloc(&c->d_work, 8 * ne * c->R)) || (s = c->dalloc(&c->d_status, 8)) || (s = c->dalloc(&c->d_dots, 4)))
    return s;
  return tdbem_z0_f32(c);
}

tdbem_status tdbem_build_z0_csr(tdbem_ctx* c) {
  const int64_t ne = c->ne;
  const int64_t* rp;
  const int32_t* col;
  const int16_t* ml;
  const uint8_t* nl;
  const int64_t* off;
  const double* val;
  tdbem_fast_z0_source(c, &rp, &col, &ml, &nl, &off, &val);
  int32_t* d_cnt = nullptr;
  tdbem_status s;
  if ((s = c->dalloc(&d_cnt, ne)) || (s = c->dalloc(&c->d_z0_ptr, ne + 1)) ||
      (s = c->dalloc(&c->d_z0_inv_diag, ne)))
    return s;
  k_z0_csr<<<(unsigned)((ne + 127) / 128), 128, 0, c->stream>>>(rp, col, ml, nl, off, val, ne, nullptr, nullptr,
                                                                nullptr, nullptr, d_cnt, 0);
  TDBEM_CUDA_TRY(c, cudaGetLastError());
  std::vector<int32_t> cnt(ne), ptr(ne + 1);
  TDBEM_CUDA_TRY(c, cudaMemcpyAsync(cnt.data(), d_cnt, ne * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
  TDBEM_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  ptr[0] = 0;
  for (int64_t i = 0; i < ne; ++i) ptr[i + 1] = ptr[i] + cnt[i];
  c->z0_nnz = ptr[ne];
  if ((s = c->dalloc(&c->d_z0_col, c->z0_nnz)) || (s = c->dalloc(&c->d_z0_val, c->z0_nnz))) return s;
  TDBEM_CUDA_TRY(c, cudaMemcpyAsync(c->d_z0_ptr, ptr.data(), (ne + 1) * sizeof(int32_t), cudaMemcpyHostToDevice,
                                    c->stream));
  k_z0_csr<<<(unsigned)((ne + 127) / 128), 128, 0, c->stream>>>(rp, col, ml, nl, off, val, ne, c->d_z0_ptr,
                                                                c->d_z0_col, c->d_z0_val, c->d_z0_inv_diag, nullptr, 1);
  TDBEM_CUDA_TRY(c, cudaGetLastError());
  if ((s = c->dalloc(&c->d_work, 8 * ne * c->R)) || (s = c->dalloc(&c->d_status, 8)) || (s = c->dalloc(&c->d_dots, 4)))
    return s;
  return tdbem_z0_f32(c);
}

static tdbem_status pick_cluster(tdbem_ctx* c) {
  if (g_cluster) return TDBEM_OK;
  TDBEM_CUDA_TRY(c, cudaFuncSetAttribute(k_bicgstab, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  for (int cs : {16, 8, 4, 2, 1}) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(kSolveThreads);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int ncl = 0;
    cudaError_t oe = cudaOccupancyMaxActiveClusters(&ncl, k_bicgstab, &cfg);
    if (oe == cudaSuccess && ncl > 0) {
      g_cluster = cs;
      return TDBEM_OK;
    }
    cudaGetLastError();
    c->set_error(std::string("solve: cluster of ") + std::to_string(cs) + " not schedulable: " +
                 cudaGetErrorString(oe) + ", max active " + std::to_string(ncl));
  }
  return TDBEM_ECUDA;
}

// Batched solver: the cluster size of the single-RHS solver and as many
// co-resident clusters as there are right-hand sides, up to what fits.
static int g_multi_ncl = 0;
static tdbem_status pick_multi(tdbem_ctx* c) {
  if (g_multi_ncl) return TDBEM_OK;
  tdbem_status s = pick_cluster(c);
  if (s) return s;
  TDBEM_CUDA_TRY(c, cudaFuncSetAttribute(k_bicgstab_multi, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(g_cluster);
  cfg.blockDim = dim3(kSolveThreads);
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = g_cluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int ncl = 0;
  TDBEM_CUDA_TRY(c, cudaOccupancyMaxActiveClusters(&ncl, k_bicgstab_multi, &cfg));
  if (ncl < 1) {
    c->set_error("solve: no cluster of the batched solver is schedulable");
    return TDBEM_ECUDA;
  }
  g_multi_ncl = ncl;
  return TDBEM_OK;
}

static tdbem_status solve_multi(tdbem_ctx* c, int32_t alpha) {
  tdbem_status s;
  if ((s = pick_multi(c))) return s;
  MultiArgs A;
  A.ptr = c->d_z0_ptr;
  A.col = c->d_z0_col;
  A.val = c->d_z0_val;
  A.val32 = c->d_z0_val32;
  A.inv_diag = c->d_z0_inv32;
  A.b = c->d_R;
  A.x = c->d_J;
  A.ring = c->d_Jring;
  A.L = c->L;
  A.alpha = alpha;
  A.warm = c->p.warm_start ? 1 : 0;
  A.R = c->R;
  A.w = c->d_work;
  A.ne = c->ne;
  A.tol = c->p.solve_tol;
  A.maxit = c->p.solve_maxit;
  A.status = c->d_status;
  // every cluster must hold at most kMaxRhs right-hand sides
  int ncl = std::min(g_multi_ncl, c->R);
  if ((c->R + ncl - 1) / ncl > kMaxRhs) {
    c->set_error("solve: too many right-hand sides for the co-resident solver clusters");
    return TDBEM_EINVAL;
  }
  c->cluster = g_cluster;
  TDBEM_CUDA_TRY(c, cudaMemsetAsync(c->d_status, 0, sizeof(int32_t), c->stream));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(g_cluster * ncl);
  cfg.blockDim = dim3(kSolveThreads);
  cfg.stream = c->stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = g_cluster;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  TDBEM_CUDA_TRY(c, cudaLaunchKernelEx(&cfg, k_bicgstab_multi, A));
  return TDBEM_OK;
}

tdbem_status tdbem_solve_z0(tdbem_ctx* c, int32_t alpha, int32_t* iters) {
  tdbem_status s;
  if (c->R > 1) {
    if ((s = solve_multi(c, alpha))) return s;
  } else {
    if ((s = pick_cluster(c))) return s;
    SolveArgs A;
    A.ptr = c->d_z0_ptr;
    A.col = c->d_z0_col;
    A.val = c->d_z0_val;
    A.val32 = c->d_z0_val32;
    A.inv_diag = c->d_z0_inv32;
    A.b = c->d_R;
    A.x = c->d_J;
    A.ring = c->d_Jring;
    A.L = c->L;
    A.alpha = alpha;
    A.warm = c->p.warm_start ? 1 : 0;
    A.w = c->d_work;
    A.ne = c->ne;
    A.tol = c->p.solve_tol;
    A.maxit = c->p.solve_maxit;
    A.status = c->d_status;
    A.resid = c->d_dots;
    c->cluster = g_cluster;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(g_cluster);
    cfg.blockDim = dim3(kSolveThreads);
    cfg.stream = c->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = g_cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    TDBEM_CUDA_TRY(c, cudaLaunchKernelEx(&cfg, k_bicgstab, A));
  }
  if (iters) {
    int32_t h[2];
    TDBEM_CUDA_TRY(c, cudaMemcpyAsync(h, c->d_status, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    TDBEM_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    *iters = h[0];
    c->total_iters += h[0];
    if (!h[1]) {
      c->set_error("solve: Z0 tolerance not reached within solve_maxit");
      return TDBEM_ENOCONV;
    }
  }
  return TDBEM_OK;
}
