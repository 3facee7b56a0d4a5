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

struct SolveArgs {
  const int32_t* ptr;
  const int32_t* col;
  const double* val;
  const double* inv_diag;
  const double* b;
  double* x;        // solution (also written to the ring)
  double* ring;     // [ne][L]
  int32_t L;
  int32_t alpha;    // solving J^{alpha-1}
  int32_t warm;     // 1: cubic extrapolation of J^{alpha-2..alpha-5}
  double* w;        // 8 work vectors [8][ne]: r, rh, p, v, s, t, ph, sh
  int64_t ne;
  double tol;
  int32_t maxit;
  int32_t* status;  // [0] iterations, [1] converged flag, [2] misses, [3] iteration total
  double* resid;    // [0] final relative residual
};

template <int NV>
__device__ __forceinline__ void block_sums(double (&v)[NV], double* sm) {
  // sm: [32][NV]
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

// Sum of per-CTA partials `mine` over the cluster: thread 0 of each CTA holds
// its block total; the totals are published in the CTA's shared slot, the
// cluster barrier orders them, and every thread reads all slots through DSMEM
// in rank order (identical result in every CTA).
template <int NV>
__device__ __forceinline__ void cluster_sums(cg::cluster_group& cl, double (&v)[NV], double* slot) {
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) slot[k] = v[k];
  cl.sync();
  unsigned nb = cl.num_blocks();
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = 0.0;
  for (unsigned r = 0; r < nb; ++r) {
    const double* rs = cl.map_shared_rank(slot, r);
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] += rs[k];
  }
}

__device__ __forceinline__ double spmv_row(const SolveArgs& A, int64_t i, const double* xin) {
  double s = 0.0;
  for (int k = A.ptr[i]; k < A.ptr[i + 1]; ++k) s += A.val[k] * xin[A.col[k]];
  return s;
}

__global__ void __launch_bounds__(kSolveThreads) k_bicgstab(SolveArgs A) {
  cg::cluster_group cl = cg::this_cluster();
  __shared__ double red[32 * 4];
  // one slot per reduction phase, so that a slot is rewritten only after a
  // further cluster barrier that every reader has passed
  __shared__ double slots[6][4];
  const int64_t ne = A.ne;
  const unsigned nb = cl.num_blocks(), rk = cl.block_rank();
  const int64_t rows = (ne + nb - 1) / nb;
  const int64_t r0 = rk * rows, r1 = min(ne, r0 + rows);
  double* r = A.w;
  double* rh = A.w + ne;
  double* p = A.w + 2 * ne;
  double* v = A.w + 3 * ne;
  double* s = A.w + 4 * ne;
  double* t = A.w + 5 * ne;
  double* ph = A.w + 6 * ne;
  double* sh = A.w + 7 * ne;
  const int L = A.L, msk = A.L - 1;
  // initial guess
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
  double d3[3];
  d3[0] = d3[1] = d3[2] = 0.0;
  for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
    double ri = A.b[i] - spmv_row(A, i, A.x);
    r[i] = ri;
    rh[i] = ri;
    p[i] = 0.0;
    v[i] = 0.0;
    d3[0] += ri * ri;
    d3[1] += A.b[i] * A.b[i];
  }
  block_sums<3>(d3, red);
  cluster_sums<3>(cl, d3, slots[0]);
  double rr = d3[0], bb = d3[1];
  double rho = rr, rho_old = 1.0, alp = 1.0, om = 1.0;
  const double tol2 = A.tol * A.tol * bb;
  int it = 0;
  bool conv = (rr <= tol2);
  while (!conv && it < A.maxit) {
    ++it;
    if (rho == 0.0) break;
    double beta = (rho / rho_old) * (alp / om);
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      double pi = r[i] + beta * (p[i] - om * v[i]);
      p[i] = pi;
      ph[i] = pi * A.inv_diag[i];
    }
    cl.sync();
    double d1[1] = {0.0};
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      double vi = spmv_row(A, i, ph);
      v[i] = vi;
      d1[0] += rh[i] * vi;
    }
    block_sums<1>(d1, red);
    cluster_sums<1>(cl, d1, slots[1]);
    if (d1[0] == 0.0) break;
    alp = rho / d1[0];
    double d1b[1] = {0.0};
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      double si = r[i] - alp * v[i];
      s[i] = si;
      sh[i] = si * A.inv_diag[i];
      d1b[0] += si * si;
    }
    block_sums<1>(d1b, red);
    cluster_sums<1>(cl, d1b, slots[2]);
    if (d1b[0] <= tol2) {
      for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
        A.x[i] += alp * ph[i];
        r[i] = s[i];
      }
      rr = d1b[0];
      conv = true;
      break;
    }
    double d2[2] = {0.0, 0.0};
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      double ti = spmv_row(A, i, sh);
      t[i] = ti;
      d2[0] += ti * s[i];
      d2[1] += ti * ti;
    }
    block_sums<2>(d2, red);
    cluster_sums<2>(cl, d2, slots[3]);
    if (d2[1] == 0.0) break;
    om = d2[0] / d2[1];
    double d2b[2] = {0.0, 0.0};
    for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
      A.x[i] += alp * ph[i] + om * sh[i];
      double ri = s[i] - om * t[i];
      r[i] = ri;
      d2b[0] += ri * ri;
      d2b[1] += rh[i] * ri;
    }
    block_sums<2>(d2b, red);
    cluster_sums<2>(cl, d2b, slots[4 + (it & 1)]);
    rr = d2b[0];
    rho_old = rho;
    rho = d2b[1];
    conv = (rr <= tol2);
    if (om == 0.0) break;
  }
  // publish J^{alpha-1}
  for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) A.ring[i * L + ((A.alpha - 1) & msk)] = A.x[i];
  if (rk == 0 && threadIdx.x == 0) {
    A.status[0] = it;
    A.status[1] = conv ? 1 : 0;
    A.status[2] += conv ? 0 : 1;  // solves that missed the tolerance since the last reset
    A.status[3] += it;            // iterations since the last reset
    A.resid[0] = bb > 0 ? sqrt(rr / bb) : 0.0;
  }
  cl.sync();  // keep every CTA's shared slots alive until all remote reads are done
}

}  // namespace tdbem

using namespace tdbem;

static int g_cluster = 0;

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
  if ((s = c->dalloc(&c->d_work, 8 * ne)) || (s = c->dalloc(&c->d_status, 4)) || (s = c->dalloc(&c->d_dots, 4)))
    return s;
  return TDBEM_OK;
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

tdbem_status tdbem_solve_z0(tdbem_ctx* c, int32_t alpha, int32_t* iters) {
  tdbem_status s;
  if ((s = pick_cluster(c))) return s;
  SolveArgs A;
  A.ptr = c->d_z0_ptr;
  A.col = c->d_z0_col;
  A.val = c->d_z0_val;
  A.inv_diag = c->d_z0_inv_diag;
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
