// solve.cu -- the per-step solve Z0 J^{alpha-1} = R^{alpha-1} (paper eq. solve).
//
// Z0 = Zt^(1) couples only edges whose supports come within c dt of each other
// (tau = 1 - r/(c dt) > 0), so it is sparse and close to diagonal (section
// 2.6).  It is built in CSR, kept for the solver in column-major ELL, and
// solved with Jacobi-preconditioned BiCGStab to
// a relative residual solve_tol, starting from the cubic extrapolation of the
// last four currents.
//
// The whole Krylov loop runs in ONE launch of a thread-block cluster: each of
// the cluster's CTAs owns a contiguous block of rows, vectors live in global
// memory (L2-resident), and every reduction is combined through distributed
// shared memory after a hardware cluster barrier.  There is no host round trip
// and no software spin-wait; all CTAs take identical branch decisions because
// they read the same reduced values.  Large meshes (kGridSolveRows) run the
// same loop over a cooperative grid of every SM, meeting at grid barriers.
#include <cooperative_groups.h>

#include <algorithm>
#include <vector>

#include "internal.h"

namespace cg = cooperative_groups;

namespace tdbem {

constexpr int kSolveThreads = 512;
constexpr int kPc = 5;  // entries per row of the triangle-block preconditioner
// squared relative residual at which an inner FP32 BiCGStab stops (1e-5 in
// norm; 1e-6 measured 4% fewer iterations and no faster solve, the batched
// solve slower)
constexpr double kInner2 = 1e-10;
// iterations of one inner FP32 solve: a few on well-shaped meshes, ~100 where
// slivers (a cone tip, the poles of a UV mesh) worsen the conditioning of Z0
constexpr int kInnerMax = 80;
constexpr double kJacRatio = 0.7;  // largest residual ratio per Jacobi sweep that keeps sweeping

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
  // Z0 as column-major ELL: row i has len[i] entries, entry k at [k*ne + i]
  const int32_t* len;
  const int32_t* col;
  const double* val;      // Z0, FP64 (residuals, Jacobi sweeps)
  const float* val32;     // Z0, FP32 (inner iterations)
  const float* inv_diag;  // Jacobi preconditioner
  const int32_t* pc_col;  // triangle-block preconditioner P as ELL [kPc][ne] (null: Jacobi)
  const float* pc_val;
  const double* b;
  double* x;        // solution (also written to the ring)
  double* ring;     // [ne][L]
  int32_t L;
  int32_t alpha;    // solving J^{alpha-1}
  int32_t warm;     // 1: cubic extrapolation of J^{alpha-2..alpha-5}; 2: x holds another guess,
                    //    kept unless the extrapolation has the smaller residual
  double* w;        // FP64 residual [ne], then 9 FP32 vectors [9][ne]
  int64_t ne;
  double tol;
  int32_t maxit;    // cap on the total inner iterations
  int32_t jacobi;   // max FP64 Jacobi sweeps before the Krylov refinement (0: none)
  int32_t* status;  // [0] inner iterations, [1] converged flag, [2] misses, [3] iteration total,
                    // [6] Jacobi sweeps of this solve, [7] Jacobi sweeps since the last reset
  double* resid;    // [0] final relative residual
  double* gslots;   // grid-wide form: [2][gridDim][4] per-block partial sums
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

// Where the solve's CTAs meet.  ClusterSync: one thread-block cluster, the
// sums combined through distributed shared memory.  GridSync: a cooperative
// grid over the whole GPU (large meshes, where one cluster's 16 SMs are too
// few), the per-block partials published in global memory and read back with
// L2-only loads after the grid barrier, summed by every block in the same
// fixed order.
struct ClusterSync {
  cg::cluster_group cl;
  double (*slots)[4];
  double* bc;
  int phase = 0;
  __device__ unsigned nblocks() const { return cl.num_blocks(); }
  __device__ unsigned rank() const { return cl.block_rank(); }
  __device__ void sync() { cl.sync(); }
  template <int NV>
  __device__ void sums(double (&v)[NV]) {
    cluster_sums<NV>(cl, v, slots, bc, phase);
  }
};

struct GridSync {
  cg::grid_group g;
  double* gslots;  // [2][gridDim.x][4]
  double* bc;
  int phase = 0;
  __device__ unsigned nblocks() const { return gridDim.x; }
  __device__ unsigned rank() const { return blockIdx.x; }
  __device__ void sync() { g.sync(); }
  template <int NV>
  __device__ void sums(double (&v)[NV]) {
    double* slot = gslots + (int64_t)(phase & 1) * gridDim.x * 4;
    ++phase;
    if (threadIdx.x == 0)
#pragma unroll
      for (int k = 0; k < NV; ++k) slot[(int64_t)blockIdx.x * 4 + k] = v[k];
    g.sync();
    if (threadIdx.x < 32) {
#pragma unroll
      for (int k = 0; k < NV; ++k) {
        double s = 0.0;
        for (unsigned b = threadIdx.x; b < gridDim.x; b += 32) s += __ldcg(slot + (int64_t)b * 4 + k);
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) bc[k] = s;
      }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = bc[k];
  }
};

// Row i of Z0 times x (x[j*R + rl]: column rl of an [ne][R] block).  With the
// column-major ELL layout consecutive rows (threads) read consecutive
// addresses, and four independent products per step keep loads in flight.
template <class T, class V>
__device__ __forceinline__ V ell_row(const int32_t* len, const int32_t* col, const T* val, int64_t ne, int64_t i,
                                     const V* x, int R, int rl) {
  V s0 = 0, s1 = 0, s2 = 0, s3 = 0;
  const int n = len[i];
  int k = 0;
  for (; k + 3 < n; k += 4) {
    const int64_t a = (int64_t)k * ne + i;
    const int c0 = col[a], c1 = col[a + ne], c2 = col[a + 2 * ne], c3 = col[a + 3 * ne];
    const V v0 = (V)val[a], v1 = (V)val[a + ne], v2 = (V)val[a + 2 * ne], v3 = (V)val[a + 3 * ne];
    s0 += v0 * x[(int64_t)c0 * R + rl];
    s1 += v1 * x[(int64_t)c1 * R + rl];
    s2 += v2 * x[(int64_t)c2 * R + rl];
    s3 += v3 * x[(int64_t)c3 * R + rl];
  }
  for (; k < n; ++k) {
    const int64_t a = (int64_t)k * ne + i;
    s0 += (V)val[a] * x[(int64_t)col[a] * R + rl];
  }
  return (s0 + s1) + (s2 + s3);
}

__device__ __forceinline__ double spmv_row64(const SolveArgs& A, int64_t i, const double* x) {
  return ell_row<double, double>(A.len, A.col, A.val, A.ne, i, x, 1, 0);
}

__device__ __forceinline__ float spmv_row32(const SolveArgs& A, int64_t i, const float* x) {
  return ell_row<float, float>(A.len, A.col, A.val32, A.ne, i, x, 1, 0);
}

// The same for column rl of an [ne][R] block
__device__ __forceinline__ float precond_row_r(const int32_t* pcol, const float* pval, int64_t ne, int64_t i,
                                               const float* x, int R, int rl) {
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kPc; ++k) s += pval[k * ne + i] * x[(int64_t)pcol[k * ne + i] * R + rl];
  return s;
}

// Row i of the triangle-block preconditioner times x (kPc entries: the edge
// and its four RWG neighbours; unused slots hold a zero value).
__device__ __forceinline__ float precond_row(const SolveArgs& A, int64_t i, const float* x) {
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < kPc; ++k) s += A.pc_val[k * A.ne + i] * x[A.pc_col[k * A.ne + i]];
  return s;
}

// Mixed-precision solve of Z0 x = b: FP64 residual r = b - Z0 x (iterative
// refinement) around an FP32 preconditioned BiCGStab for the correction, run
// to the reduction the outer tolerance still needs, at most 1e-5 (kInner2).
// Z0 is well conditioned (about 2 on the test spheres), so each refinement
// gains five to six digits and two to three refinements reach 1e-13.
template <class Sync>
__device__ __forceinline__ void bicgstab_body(const SolveArgs& A, Sync& cl, double* red) {
  const int64_t ne = A.ne;
  const unsigned nb = cl.nblocks(), rk = cl.rank();
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
  // warm 1: the extrapolation goes to x; warm 2: to r64, beside the guess in x
  double* xc_dst = A.warm == 2 ? r64 : A.x;
  for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
    double x0 = 0.0;
    if (A.warm) {
      const double* J = A.ring + i * L;
      int b = A.alpha - 2;  // J^{alpha-2}, J^{alpha-3}, ... (zero before step 0)
      double j1 = b >= 0 ? J[b & msk] : 0.0, j2 = b >= 1 ? J[(b - 1) & msk] : 0.0;
      double j3 = b >= 2 ? J[(b - 2) & msk] : 0.0, j4 = b >= 3 ? J[(b - 3) & msk] : 0.0;
      x0 = 4.0 * j1 - 6.0 * j2 + 4.0 * j3 - j4;
    }
    xc_dst[i] = x0;
  }
  cl.sync();
  if (A.warm == 2) {
    // keep the guess only if its FP64 residual is smaller (a NaN never is)
    double q2[2] = {0.0, 0.0};
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      const double rg = A.b[i] - spmv_row64(A, i, A.x), rc = A.b[i] - spmv_row64(A, i, r64);
      q2[0] += rg * rg;
      q2[1] += rc * rc;
    }
    block_sums<2>(q2, red);
    cl.template sums<2>(q2);
    const bool keep = q2[0] < q2[1];
    if (!keep) {
      for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) A.x[i] = r64[i];
    }
    if (rk == 0 && threadIdx.x == 0) A.status[keep ? 8 : 9] += 1;
    cl.sync();
  }
  double bb = -1.0, rr = 0.0;
  int inner_total = 0;
  bool conv = false;
  // Stage 1: FP64 Jacobi sweeps x <- x + D^{-1}(b - Z0 x).  Z0 is strongly
  // diagonal (spectral radius of I - D^{-1} Z0 about 0.27 on the test
  // meshes), so each sweep gains about half a digit for one SpMV and one
  // cluster reduction.  The sweep that finds a residual norm above kJacRatio
  // times the previous one hands the iterate to the Krylov stage instead.
  int sweeps = 0;
  {
    double* cur = A.x;
    double* nxt = r64;  // the residual buffer is free until the Krylov stage
    double rr_prev = -1.0;
    for (int k = 0; k < A.jacobi; ++k) {
      double q2[2] = {0.0, 0.0};
      for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        double ri = A.b[i] - spmv_row64(A, i, cur);
        nxt[i] = cur[i] + ri * (double)A.inv_diag[i];
        q2[0] += ri * ri;
        q2[1] += A.b[i] * A.b[i];
      }
      block_sums<2>(q2, red);
      cl.template sums<2>(q2);  // its cluster barrier also publishes nxt
      if (bb < 0) bb = q2[1];
      rr = q2[0];
      if (rr <= A.tol * A.tol * bb) {  // cur is the solution
        conv = true;
        break;
      }
      if (rr_prev >= 0.0 && rr > kJacRatio * kJacRatio * rr_prev) break;  // not contracting: keep cur
      rr_prev = rr;
      double* t = cur;
      cur = nxt;
      nxt = t;
      ++sweeps;
    }
    if (cur != A.x) {
      for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) A.x[i] = cur[i];
      cl.sync();
    }
  }
  for (int outer = 0; outer < 8 && !conv; ++outer) {
    // FP64 residual
    double q2[2] = {0.0, 0.0};
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      double ri = A.b[i] - spmv_row64(A, i, A.x);
      r64[i] = ri;
      q2[0] += ri * ri;
      q2[1] += A.b[i] * A.b[i];
    }
    block_sums<2>(q2, red);
    cl.template sums<2>(q2);
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
    cl.template sums<1>(*(double(*)[1])q1);
    double rho = q1[0], rho_old = 1.0, alp = 1.0, om = 1.0;
    // inner target: the reduction that brings the FP64 residual to half the
    // outer tolerance, within [1e-5, 0.5] (1e-5: what FP32 reliably reaches)
    const double want2 = 0.25 * A.tol * A.tol * bb / rr;
    const double tin2 = fmin(fmax(want2, kInner2), 0.25) * q1[0];
    for (int it = 0; it < kInnerMax && inner_total < A.maxit; ++it) {
      ++inner_total;
      if (rho == 0.0) break;
      float beta = (float)((rho / rho_old) * (alp / om));
      float omf = (float)om;
      for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        float pi = r[i] + beta * (p[i] - omf * v[i]);
        p[i] = pi;
        if (!A.pc_val) ph[i] = pi * A.inv_diag[i];
      }
      cl.sync();
      if (A.pc_val) {  // ph = P p needs the neighbours' p: published by the barrier above
        for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) ph[i] = precond_row(A, i, p);
        cl.sync();
      }
      double e1[1] = {0.0};
      for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        float vi = spmv_row32(A, i, ph);
        v[i] = vi;
        e1[0] += (double)(rh[i] * vi);
      }
      block_sums<1>(e1, red);
      cl.template sums<1>(e1);
      if (e1[0] == 0.0) break;
      alp = rho / e1[0];
      float alf = (float)alp;
      double e2[1] = {0.0};
      for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        float si = r[i] - alf * v[i];
        s[i] = si;
        if (!A.pc_val) sh[i] = si * A.inv_diag[i];
        e2[0] += (double)(si * si);
      }
      block_sums<1>(e2, red);
      cl.template sums<1>(e2);  // also orders sh (or s) for what follows
      if (e2[0] <= tin2) {
        for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) d[i] += alf * ph[i];
        break;
      }
      if (A.pc_val) {
        for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) sh[i] = precond_row(A, i, s);
        cl.sync();
      }
      double e3[2] = {0.0, 0.0};
      for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        float ti = spmv_row32(A, i, sh);
        t[i] = ti;
        e3[0] += (double)(ti * s[i]);
        e3[1] += (double)(ti * ti);
      }
      block_sums<2>(e3, red);
      cl.template sums<2>(e3);
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
      cl.template sums<2>(e4);
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
    A.status[6] = sweeps;
    A.status[7] += sweeps;
    A.status[1] = conv ? 1 : 0;
    A.status[2] += conv ? 0 : 1;  // solves that missed the tolerance since the last reset
    A.status[3] += inner_total;   // iterations since the last reset
    A.resid[0] = bb > 0 ? sqrt(rr / bb) : 0.0;
  }
  cl.sync();  // keep every CTA's shared slots alive until all remote reads are done
}

__global__ void __launch_bounds__(kSolveThreads) k_bicgstab(SolveArgs A) {
  __shared__ double red[32 * 4];
  __shared__ double slots[2][4];
  __shared__ double bc[4];
  ClusterSync S{cg::this_cluster(), slots, bc};
  bicgstab_body(A, S, red);
}

// The same solve over a cooperative grid (launched with
// cudaLaunchCooperativeKernel, every block resident).
__global__ void __launch_bounds__(kSolveThreads) k_bicgstab_grid(SolveArgs A) {
  __shared__ double red[32 * 4];
  __shared__ double bc[4];
  GridSync S{cg::this_grid(), A.gslots, bc};
  bicgstab_body(A, S, red);
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
  const int32_t* len;  // Z0 as column-major ELL (see SolveArgs)
  const int32_t* pc_col;  // triangle-block preconditioner (see SolveArgs; null: Jacobi)
  const float* pc_val;
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
  int32_t jacobi;    // max FP64 Jacobi sweeps before the Krylov refinement
  int32_t* status;   // [0] max inner iterations, [1] all converged, [2] misses, [3] total, [4..5] scratch,
                     // [6] max Jacobi sweeps of this solve, [7] their running total
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

// Add a thread's partial sum v (of right-hand side l = lane mod Rp) into
// part[l]: lanes of one RHS are combined by shuffles first, so each warp
// issues at most 32 shared atomics per reduction.
__device__ __forceinline__ void seg_add(double v, int Rp, bool act, double* part, int l) {
  for (int o = 16; o >= Rp; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (act && (threadIdx.x & 31) < Rp) atomicAdd(&part[l], v);
}

// Element map: the cluster's RHS slice (Rl right-hand sides) is padded to
// Rp = a power of two <= kMaxRhs; thread t always takes RHS l = t mod Rp
// (active when l < Rl) and rows r0 + t / Rp, stepping by blockDim / Rp, so
// its partial sums are per-RHS registers.
__global__ void __launch_bounds__(kSolveThreads) k_bicgstab_multi(MultiArgs A) {
  cg::cluster_group cl = cg::this_cluster();
  __shared__ double part[kMaxRhs], part2[kMaxRhs], red1[kMaxRhs], red2[kMaxRhs];
  __shared__ double slots[2][kMaxRhs], slots2[2][kMaxRhs];
  __shared__ double rho[kMaxRhs], rho_old[kMaxRhs], alp[kMaxRhs], om[kMaxRhs], bb[kMaxRhs], nr[kMaxRhs];
  __shared__ double rprev[kMaxRhs];
  __shared__ int act[kMaxRhs], conv[kMaxRhs], jac[kMaxRhs];
  int phase = 0, phase2 = 0;
  const int R = A.R;
  const unsigned nb = cl.num_blocks(), rk = cl.block_rank();
  const int ncl = gridDim.x / nb, cid = blockIdx.x / nb;
  const int Rc = (R + ncl - 1) / ncl;
  const int rb = cid * Rc, Rl = max(0, min(R, rb + Rc) - rb);  // this cluster's RHS slice
  int sh = 0;
  while ((1 << sh) < Rl) ++sh;
  const int Rp = 1 << sh;
  const int l = threadIdx.x & (Rp - 1);
  const bool lane_on = l < Rl;
  const int rstep = blockDim.x >> sh;
  const int64_t ne = A.ne;
  const int64_t rows = (ne + nb - 1) / nb;
  const int64_t r0 = rk * rows, r1 = min(ne, r0 + rows);
  const int64_t i0 = r0 + (threadIdx.x >> sh);
  const int64_t NR = ne * R;
  double* r64 = A.w;
  float* f = (float*)(A.w + NR);
  float *rv = f, *rh = f + NR, *pv = f + 2 * NR, *vv = f + 3 * NR, *sv = f + 4 * NR, *tv = f + 5 * NR,
        *ph = f + 6 * NR, *shv = f + 7 * NR, *dv = f + 8 * NR;
  const int L = A.L, msk = L - 1;
  const int rl = rb + l;  // this thread's right-hand side (valid when lane_on)
#define ROWS for (int64_t i = lane_on ? i0 : r1; i < r1; i += rstep)
  for (int k = threadIdx.x; k < kMaxRhs; k += blockDim.x) {
    part[k] = part2[k] = 0.0;
    bb[k] = -1.0;
    rprev[k] = -1.0;
    conv[k] = act[k] = 0;
    jac[k] = 1;
  }
  __syncthreads();
  double* xc_dst = A.warm == 2 ? r64 : A.x;  // as in k_bicgstab
  ROWS {
    double x0 = 0.0;
    if (A.warm) {
      const double* J = A.ring + i * L * R + rl;
      int b = A.alpha - 2;
      double j1 = b >= 0 ? J[(int64_t)(b & msk) * R] : 0.0, j2 = b >= 1 ? J[(int64_t)((b - 1) & msk) * R] : 0.0;
      double j3 = b >= 2 ? J[(int64_t)((b - 2) & msk) * R] : 0.0, j4 = b >= 3 ? J[(int64_t)((b - 3) & msk) * R] : 0.0;
      x0 = 4.0 * j1 - 6.0 * j2 + 4.0 * j3 - j4;
    }
    xc_dst[i * R + rl] = x0;
  }
  cl.sync();
  if (A.warm == 2) {
    double q1 = 0.0, q2 = 0.0;
    ROWS {
      const double bi = A.b[i * R + rl];
      const double rg = bi - ell_row<double, double>(A.len, A.col, A.val, A.ne, i, A.x, R, rl);
      const double rc = bi - ell_row<double, double>(A.len, A.col, A.val, A.ne, i, r64, R, rl);
      q1 += rg * rg;
      q2 += rc * rc;
    }
    seg_add(q1, Rp, lane_on, part, l);
    seg_add(q2, Rp, lane_on, part2, l);
    __syncthreads();
    multi_reduce(cl, part, slots, red1, Rl, phase);
    multi_reduce(cl, part2, slots2, red2, Rl, phase2);
    if (lane_on && !(red1[l] < red2[l])) {
      ROWS A.x[i * R + rl] = r64[i * R + rl];
    }
    if (rk == 0 && threadIdx.x == 0) {
      int kept = 0;
      for (int m = 0; m < Rl; ++m) kept += red1[m] < red2[m] ? 1 : 0;
      atomicAdd(&A.status[8], kept);
      atomicAdd(&A.status[9], Rl - kept);
    }
    cl.sync();
  }
  int inner_total = 0, sweeps = 0;
  // Stage 1: FP64 Jacobi sweeps per RHS (as in k_bicgstab).  An RHS leaves
  // the stage when it converges or stops contracting; its iterate is then
  // carried along unchanged (jac: 1 sweeping, 2 stopping now, 0 stopped).
  {
    double* cur = A.x;
    double* nxt = r64;
    for (int k = 0; k < A.jacobi; ++k) {
      int any = 0;
      for (int m = 0; m < Rl; ++m) any |= (jac[m] == 1);
      if (!any) break;
      double q1 = 0.0, q2 = 0.0;
      const bool on = lane_on && jac[l] == 1;
      ROWS {
        const int64_t q = i * R + rl;
        if (!on) {
          nxt[q] = cur[q];
          continue;
        }
        double sacc = 0.0;
        sacc = ell_row<double, double>(A.len, A.col, A.val, A.ne, i, cur, R, rl);
        const double bi = A.b[q], ri = bi - sacc;
        nxt[q] = cur[q] + ri * (double)A.inv_diag[i];
        q1 += ri * ri;
        q2 += bi * bi;
      }
      seg_add(q1, Rp, on, part, l);
      seg_add(q2, Rp, on, part2, l);
      __syncthreads();
      multi_reduce(cl, part, slots, red1, Rl, phase);  // its cluster barrier also publishes nxt
      multi_reduce(cl, part2, slots2, red2, Rl, phase2);
      for (int m = threadIdx.x; m < Rl; m += blockDim.x) {
        if (jac[m] != 1) continue;
        if (bb[m] < 0) bb[m] = red2[m];
        const bool done = red1[m] <= A.tol * A.tol * bb[m];
        const bool slow = rprev[m] >= 0.0 && red1[m] > kJacRatio * kJacRatio * rprev[m];
        rprev[m] = red1[m];
        if (done || slow) jac[m] = 2;  // keeps cur: its nxt is reset below
      }
      __syncthreads();
      if (lane_on && jac[l] == 2) {
        ROWS nxt[i * R + rl] = cur[i * R + rl];
      }
      __syncthreads();
      for (int m = threadIdx.x; m < Rl; m += blockDim.x)
        if (jac[m] == 2) jac[m] = 0;
      cl.sync();  // reverted values and flags visible before the next sweep
      double* t = cur;
      cur = nxt;
      nxt = t;
      ++sweeps;
    }
    if (cur != A.x) {
      ROWS A.x[i * R + rl] = cur[i * R + rl];
    }
    for (int m = threadIdx.x; m < kMaxRhs; m += blockDim.x) bb[m] = -1.0;
    cl.sync();
  }
  // Stage 2: mixed-precision refinement as in k_bicgstab, per RHS.
  for (int outer = 0;; ++outer) {
    {
      double q1 = 0.0, q2 = 0.0;
      ROWS {
        const int64_t q = i * R + rl;
        double sacc = 0.0;
        sacc = ell_row<double, double>(A.len, A.col, A.val, A.ne, i, A.x, R, rl);
        const double bi = A.b[q], ri = bi - sacc;
        r64[q] = ri;
        q1 += ri * ri;
        q2 += bi * bi;
      }
      seg_add(q1, Rp, lane_on, part, l);
      seg_add(q2, Rp, lane_on, part2, l);
    }
    __syncthreads();
    multi_reduce(cl, part, slots, red1, Rl, phase);
    multi_reduce(cl, part2, slots2, red2, Rl, phase2);
    for (int m = threadIdx.x; m < Rl; m += blockDim.x) {
      if (bb[m] < 0) bb[m] = red2[m];
      nr[m] = red1[m];
      conv[m] = red1[m] <= A.tol * A.tol * bb[m];
      act[m] = !conv[m];
    }
    __syncthreads();
    int all = 1;
    for (int m = 0; m < Rl; ++m) all &= conv[m];
    if (all || outer == 8 || inner_total >= A.maxit) break;
    // FP32 Jacobi-preconditioned BiCGStab on the unit-norm residuals, relative tolerance 1e-5
    {
      double q1 = 0.0;
      const double inv = (lane_on && nr[l] > 0) ? 1.0 / sqrt(nr[l]) : 0.0;
      ROWS {
        const int64_t q = i * R + rl;
        const float ri = (float)(r64[q] * inv);
        rv[q] = ri;
        rh[q] = ri;
        pv[q] = vv[q] = dv[q] = 0.f;
        q1 += (double)ri * ri;
      }
      seg_add(q1, Rp, lane_on, part, l);
    }
    __syncthreads();
    multi_reduce(cl, part, slots, red1, Rl, phase);
    for (int m = threadIdx.x; m < Rl; m += blockDim.x) {
      rho[m] = red1[m];
      rho_old[m] = alp[m] = om[m] = 1.0;
      act[m] = act[m] && rho[m] > 0.0;
    }
    __syncthreads();
    for (int it = 0; it < kInnerMax && inner_total < A.maxit; ++it) {
      int any = 0;
      for (int m = 0; m < Rl; ++m) any |= act[m];
      if (!any) break;
      ++inner_total;
      bool on = lane_on && act[l];
      if (on) {
        const float beta = (float)((rho[l] / rho_old[l]) * (alp[l] / om[l])), omf = (float)om[l];
        ROWS {
          const int64_t q = i * R + rl;
          const float pi = rv[q] + beta * (pv[q] - omf * vv[q]);
          pv[q] = pi;
          if (!A.pc_val) ph[q] = pi * A.inv_diag[i];
        }
      }
      cl.sync();
      if (A.pc_val) {  // ph = P p: the neighbours' p were published by the barrier above
        if (on) {
          ROWS ph[i * R + rl] = precond_row_r(A.pc_col, A.pc_val, A.ne, i, pv, R, rl);
        }
        cl.sync();
      }
      {
        double e1 = 0.0;
        if (on) {
          ROWS {
            const int64_t q = i * R + rl;
            float sacc = 0.f;
            sacc = ell_row<float, float>(A.len, A.col, A.val32, A.ne, i, ph, R, rl);
            vv[q] = sacc;
            e1 += (double)(rh[q] * sacc);
          }
        }
        seg_add(e1, Rp, on, part, l);
      }
      __syncthreads();
      multi_reduce(cl, part, slots, red1, Rl, phase);
      for (int m = threadIdx.x; m < Rl; m += blockDim.x) {
        if (act[m] && red1[m] == 0.0) act[m] = 0;
        if (act[m]) alp[m] = rho[m] / red1[m];
      }
      __syncthreads();
      on = lane_on && act[l];
      {
        double e2 = 0.0;
        if (on) {
          const float alf = (float)alp[l];
          ROWS {
            const int64_t q = i * R + rl;
            const float si = rv[q] - alf * vv[q];
            sv[q] = si;
            if (!A.pc_val) shv[q] = si * A.inv_diag[i];
            e2 += (double)(si * si);
          }
        }
        seg_add(e2, Rp, on, part, l);
      }
      __syncthreads();
      multi_reduce(cl, part, slots, red1, Rl, phase);  // its cluster barrier also publishes shv
      for (int m = threadIdx.x; m < Rl; m += blockDim.x) conv[m] = act[m] && red1[m] <= kInner2;
      __syncthreads();
      if (A.pc_val) {  // shv = P s for the right-hand sides still iterating
        if (on && !conv[l]) {
          ROWS shv[i * R + rl] = precond_row_r(A.pc_col, A.pc_val, A.ne, i, sv, R, rl);
        }
        cl.sync();
      }
      {
        double e3 = 0.0, e4 = 0.0;
        if (on) {
          const float alf = (float)alp[l];
          if (conv[l]) {
            ROWS dv[i * R + rl] += alf * ph[i * R + rl];
          } else {
            ROWS {
              const int64_t q = i * R + rl;
              float sacc = 0.f;
              sacc = ell_row<float, float>(A.len, A.col, A.val32, A.ne, i, shv, R, rl);
              tv[q] = sacc;
              e3 += (double)(sacc * sv[q]);
              e4 += (double)(sacc * sacc);
            }
          }
        }
        const bool on2 = on && !conv[l];
        seg_add(e3, Rp, on2, part, l);
        seg_add(e4, Rp, on2, part2, l);
      }
      __syncthreads();
      multi_reduce(cl, part, slots, red1, Rl, phase);
      multi_reduce(cl, part2, slots2, red2, Rl, phase2);
      for (int m = threadIdx.x; m < Rl; m += blockDim.x) {
        if (conv[m]) act[m] = 0;
        if (act[m] && red2[m] == 0.0) act[m] = 0;
        if (act[m]) om[m] = red1[m] / red2[m];
      }
      __syncthreads();
      on = lane_on && act[l];
      {
        double e5 = 0.0, e6 = 0.0;
        if (on) {
          const float alf = (float)alp[l], omf = (float)om[l];
          ROWS {
            const int64_t q = i * R + rl;
            dv[q] += alf * ph[q] + omf * shv[q];
            const float ri = sv[q] - omf * tv[q];
            rv[q] = ri;
            e5 += (double)(ri * ri);
            e6 += (double)(rh[q] * ri);
          }
        }
        seg_add(e5, Rp, on, part, l);
        seg_add(e6, Rp, on, part2, l);
      }
      __syncthreads();
      multi_reduce(cl, part, slots, red1, Rl, phase);
      multi_reduce(cl, part2, slots2, red2, Rl, phase2);
      for (int m = threadIdx.x; m < Rl; m += blockDim.x) {
        if (!act[m]) continue;
        rho_old[m] = rho[m];
        rho[m] = red2[m];
        if (red1[m] <= kInner2 || om[m] == 0.0 || rho[m] == 0.0) act[m] = 0;
      }
      __syncthreads();
    }
    if (lane_on) {
      const double sc = sqrt(nr[l]);
      ROWS A.x[i * R + rl] += sc * (double)dv[i * R + rl];
    }
    cl.sync();
  }
  int nconv = 0;
  for (int m = 0; m < Rl; ++m) nconv += conv[m] ? 1 : 0;
  ROWS A.ring[(i * L + ((A.alpha - 1) & msk)) * R + rl] = A.x[i * R + rl];
#undef ROWS
  if (rk == 0 && threadIdx.x == 0) {
    atomicMax(&A.status[0], inner_total);
    atomicMax(&A.status[6], sweeps);
    if (nconv < Rl) atomicAdd(&A.status[4], 1);
    __threadfence();
    if (atomicAdd(&A.status[5], 1) == ncl - 1) {  // last cluster: publish the verdict
      __threadfence();
      int miss = atomicAdd(&A.status[4], 0);
      int it = atomicAdd(&A.status[0], 0);
      A.status[1] = miss == 0 ? 1 : 0;
      A.status[2] += miss == 0 ? 0 : 1;
      A.status[3] += it;
      A.status[7] += atomicAdd(&A.status[6], 0);
      A.status[4] = 0;
      A.status[5] = 0;
    }
  }
  cl.sync();
}

// CSR -> column-major ELL (padding entries are never read: len[i] bounds them)
__global__ void k_csr_to_ell(const int32_t* ptr, const int32_t* col, const double* val, int64_t ne, int32_t* len,
                             int32_t* ecol, double* eval, float* eval32) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= ne) return;
  const int b = ptr[i], n = ptr[i + 1] - b;
  len[i] = n;
  for (int k = 0; k < n; ++k) {
    ecol[(int64_t)k * ne + i] = col[b + k];
    eval[(int64_t)k * ne + i] = val[b + k];
    eval32[(int64_t)k * ne + i] = (float)val[b + k];
  }
}

__global__ void k_z0_f32(const double* z, const double* inv_diag, int64_t nnz, int64_t ne, float* z32, float* inv32) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < nnz) z32[i] = (float)z[i];
  if (i < ne) inv32[i] = (float)inv_diag[i];
}

}  // namespace tdbem

using namespace tdbem;

static int g_cluster = 0;

// Triangle-block (additive Schwarz) preconditioner: for every triangle the
// 3 x 3 block of Z0 among the RWG functions of its three sides is inverted,
// and P = sum over triangles of the inverses scattered to their rows and
// columns.  Row i of P couples edge i with the other sides of its two
// triangles (at most kPc entries).  A triangle whose block is singular adds
// its diagonal reciprocals instead.
static tdbem_status build_triangle_precond(tdbem_ctx* c, const std::vector<int32_t>& hp) {
  const int64_t ne = c->ne, nnz = hp[ne];
  std::vector<int32_t> hc(nnz);
  std::vector<double> hv(nnz);
  TDBEM_CUDA_TRY(c, cudaMemcpy(hc.data(), c->d_z0_col, nnz * sizeof(int32_t), cudaMemcpyDeviceToHost));
  TDBEM_CUDA_TRY(c, cudaMemcpy(hv.data(), c->d_z0_val, nnz * sizeof(double), cudaMemcpyDeviceToHost));
  auto z = [&](int32_t i, int32_t j) {
    for (int32_t k = hp[i]; k < hp[i + 1]; ++k)
      if (hc[k] == j) return hv[k];
    return 0.0;
  };
  std::vector<int32_t> pcol(kPc * ne, 0);
  std::vector<double> pval(kPc * ne, 0.0);
  std::vector<int> used(ne, 0);
  auto add = [&](int32_t i, int32_t j, double v) {
    for (int k = 0; k < used[i]; ++k)
      if (pcol[k * ne + i] == j) {
        pval[k * ne + i] += v;
        return true;
      }
    if (used[i] == kPc) return false;
    pcol[used[i] * ne + i] = j;
    pval[used[i] * ne + i] = v;
    ++used[i];
    return true;
  };
  for (int64_t t = 0; t < c->nt; ++t) {
    const int32_t e[3] = {c->te[3 * t], c->te[3 * t + 1], c->te[3 * t + 2]};
    double B[3][3];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) B[a][b] = z(e[a], e[b]);
    double C[3][3];  // cofactors
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) {
        const int a1 = (a + 1) % 3, a2 = (a + 2) % 3, b1 = (b + 1) % 3, b2 = (b + 2) % 3;
        C[a][b] = B[a1][b1] * B[a2][b2] - B[a1][b2] * B[a2][b1];
      }
    const double det = B[0][0] * C[0][0] + B[0][1] * C[0][1] + B[0][2] * C[0][2];
    double nb = 0.0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) nb = std::max(nb, std::fabs(B[a][b]));
    bool ok = std::fabs(det) > 1e-12 * nb * nb * nb;
    for (int a = 0; a < 3 && ok; ++a)
      for (int b = 0; b < 3 && ok; ++b) ok = add(e[a], e[b], C[b][a] / det);  // inverse = adjugate / det
    if (!ok)
      for (int a = 0; a < 3; ++a)
        if (B[a][a] != 0.0) add(e[a], e[a], 1.0 / B[a][a]);
  }
  std::vector<float> pv32(kPc * ne);
  for (int64_t k = 0; k < kPc * ne; ++k) pv32[k] = (float)pval[k];
  tdbem_status s;
  if ((s = c->dalloc(&c->d_pc_col, kPc * ne)) || (s = c->dalloc(&c->d_pc_val, kPc * ne))) return s;
  TDBEM_CUDA_TRY(c, cudaMemcpy(c->d_pc_col, pcol.data(), kPc * ne * sizeof(int32_t), cudaMemcpyHostToDevice));
  TDBEM_CUDA_TRY(c, cudaMemcpy(c->d_pc_val, pv32.data(), kPc * ne * sizeof(float), cudaMemcpyHostToDevice));
  return TDBEM_OK;
}

static tdbem_status tdbem_z0_f32(tdbem_ctx* c) {
  tdbem_status s;
  if ((s = c->dalloc(&c->d_z0_val32, c->z0_nnz)) || (s = c->dalloc(&c->d_z0_inv32, c->ne))) return s;
  int64_t n = std::max<int64_t>(c->z0_nnz, c->ne);
  k_z0_f32<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(c->d_z0_val, c->d_z0_inv_diag, c->z0_nnz, c->ne,
                                                               c->d_z0_val32, c->d_z0_inv32);
  TDBEM_CUDA_TRY(c, cudaGetLastError());
  // ELL width: the longest row
  std::vector<int32_t> hp(c->ne + 1);
  TDBEM_CUDA_TRY(c, cudaMemcpyAsync(hp.data(), c->d_z0_ptr, (c->ne + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost,
                                    c->stream));
  TDBEM_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  int32_t w = 1;
  for (int64_t i = 0; i < c->ne; ++i) w = std::max(w, hp[i + 1] - hp[i]);
  c->z0_ell_w = w;
  const int64_t ew = (int64_t)w * c->ne;
  if ((s = c->dalloc(&c->d_ell_len, c->ne)) || (s = c->dalloc(&c->d_ell_col, ew)) ||
      (s = c->dalloc(&c->d_ell_val, ew)) || (s = c->dalloc(&c->d_ell_val32, ew)))
    return s;
  k_csr_to_ell<<<(unsigned)((c->ne + 255) / 256), 256, 0, c->stream>>>(c->d_z0_ptr, c->d_z0_col, c->d_z0_val, c->ne,
                                                                       c->d_ell_len, c->d_ell_col, c->d_ell_val,
                                                                       c->d_ell_val32);
  TDBEM_CUDA_TRY(c, cudaGetLastError());
  TDBEM_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (c->p.precond == 1) return build_triangle_precond(c, hp);
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
  if ((s = c->dalloc(&c->d_work, 8 * ne * c->R)) || (s = c->dalloc(&c->d_status, 16)) || (s = c->dalloc(&c->d_dots, 4)))
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
  if ((s = c->dalloc(&c->d_work, 8 * ne * c->R)) || (s = c->dalloc(&c->d_status, 16)) || (s = c->dalloc(&c->d_dots, 4)))
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

// Meshes with at least this many RWG functions solve over a cooperative grid
// of every SM instead of one cluster: a 16-SM cluster spends about 1 ms per
// BiCGStab iteration at 120000 unknowns.
constexpr int64_t kGridSolveRows = 49152;
static int g_grid = 0;
static tdbem_status pick_grid(tdbem_ctx* c) {
  if (g_grid) return TDBEM_OK;
  int dev = 0, sms = 0, coop = 0, per = 0;
  TDBEM_CUDA_TRY(c, cudaGetDevice(&dev));
  TDBEM_CUDA_TRY(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  TDBEM_CUDA_TRY(c, cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  TDBEM_CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_bicgstab_grid, kSolveThreads, 0));
  if (!coop || per < 1) {
    c->set_error("solve: cooperative launch not available for the grid-wide solve");
    return TDBEM_ECUDA;
  }
  g_grid = sms * per;
  return TDBEM_OK;
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

static tdbem_status solve_multi(tdbem_ctx* c, int32_t alpha, int32_t warm) {
  tdbem_status s;
  if ((s = pick_multi(c))) return s;
  MultiArgs A;
  A.len = c->d_ell_len;
  A.col = c->d_ell_col;
  A.val = c->d_ell_val;
  A.val32 = c->d_ell_val32;
  A.inv_diag = c->d_z0_inv32;
  A.pc_col = c->d_pc_col;
  A.pc_val = c->d_pc_val;
  A.b = c->d_R;
  A.x = c->d_J;
  A.ring = c->d_Jring;
  A.L = c->L;
  A.alpha = alpha;
  A.warm = warm;
  A.R = c->R;
  A.w = c->d_work;
  A.ne = c->ne;
  A.tol = c->p.solve_tol;
  A.maxit = c->p.solve_maxit;
  A.jacobi = c->p.jacobi_sweeps;
  A.status = c->d_status;
  // every cluster must hold at most kMaxRhs right-hand sides
  int ncl = std::min(g_multi_ncl, c->R);
  if ((c->R + ncl - 1) / ncl > kMaxRhs) {
    c->set_error("solve: too many right-hand sides for the co-resident solver clusters");
    return TDBEM_EINVAL;
  }
  c->cluster = g_cluster;
  TDBEM_CUDA_TRY(c, cudaMemsetAsync(c->d_status, 0, sizeof(int32_t), c->stream));
  TDBEM_CUDA_TRY(c, cudaMemsetAsync(c->d_status + 6, 0, sizeof(int32_t), c->stream));
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

tdbem_status tdbem_solve_z0(tdbem_ctx* c, int32_t alpha, int32_t* iters, int32_t warm) {
  tdbem_status s;
  if (c->R > 1) {
    if ((s = solve_multi(c, alpha, warm))) return s;
  } else {
    const bool grid = c->p.solve_grid == 2 || (c->p.solve_grid == 0 && c->ne >= kGridSolveRows);
    if ((s = grid ? pick_grid(c) : pick_cluster(c))) return s;
    if (grid && !c->d_gslots && (s = c->dalloc(&c->d_gslots, (size_t)2 * g_grid * 4))) return s;
    SolveArgs A;
    A.len = c->d_ell_len;
    A.col = c->d_ell_col;
    A.val = c->d_ell_val;
    A.val32 = c->d_ell_val32;
    A.inv_diag = c->d_z0_inv32;
    A.pc_col = c->d_pc_col;
    A.pc_val = c->d_pc_val;
    A.b = c->d_R;
    A.x = c->d_J;
    A.ring = c->d_Jring;
    A.L = c->L;
    A.alpha = alpha;
    A.warm = warm;
    A.w = c->d_work;
    A.ne = c->ne;
    A.tol = c->p.solve_tol;
    A.maxit = c->p.solve_maxit;
    A.jacobi = c->p.jacobi_sweeps;
    A.status = c->d_status;
    A.resid = c->d_dots;
    A.gslots = c->d_gslots;
    if (grid) {
      c->cluster = g_grid;
      void* args[] = {&A};
      TDBEM_CUDA_TRY(c, cudaLaunchCooperativeKernel((void*)k_bicgstab_grid, dim3(g_grid), dim3(kSolveThreads), args,
                                                    0, c->stream));
    } else {
      // Default: the largest cluster, except in the pipelined direct march with
      // a history sum streaming at least 3 GB per step (about 0.5 ms).  There
      // the solve overlaps that sum on its own SMs, and a cluster of 4 leaves
      // 12 more SMs to it while the solve still hides behind it (7680-RWG
      // sphere, (hi, lo) store of 4.6 GB: 1145 steps/s against 1106 with 16).
      // A shorter sum (the FP32 store's 2.3 GB) leaves the solve on the
      // critical path, where 16 CTAs win (2160 steps/s against 1855 with 4).
      int cs = g_cluster;
      if (c->p.solve_cluster > 0)
        cs = std::min(c->p.solve_cluster, g_cluster);
      else if (c->p.mode == TDBEM_DIRECT && c->p.far_overlap && c->rt_bytes >= (3LL << 30))
        cs = std::min(4, g_cluster);
      c->cluster = cs;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(cs);
      cfg.blockDim = dim3(kSolveThreads);
      cfg.stream = c->stream;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = cs;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      TDBEM_CUDA_TRY(c, cudaLaunchKernelEx(&cfg, k_bicgstab, A));
    }
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
