// fmm.cu -- fast mode: near field directly, far field by the space-time
// interpolation-based FMM (paper section 3).
//
// Clusters.  An adaptive octree over the triangle centroids (section 3.4.1,
// with triangles as the particles: each triangle carries the parts of its
// three RWG functions).  A cell is split while it holds more than n_leaf
// edges (1.5 per triangle) and while its children's time intervals can still
// hold d+1 = 3 steps (see below).  Cells at level l have size ds_l; the
// interpolation box of a cell is its cube enlarged by delta = max distance
// from a triangle centroid to its outer-rule points (the only points at which
// the far field samples a triangle), so that all of them lie inside:
// half-width H_l = ds_l/2 + delta.
//
// Time intervals (eq. Mt).  M_l steps per interval at level l, M_l = 2 M_{l+1}.
// Causality of one interval requires M_l c dt <= (smallest distance between
// two non-adjacent boxes) = ds_l - 2 delta, hence
//     M_lmax = floor((ds_lmax - 2 delta) / (c dt)),
// with EBREAKDOWN (Remark 1) when it is below d+1 (the window truncation below
// needs one interval to contain the d+1 first steps of a window).
//
// Far field (section 3.3).  With Jh^gamma = sum_k w^k J^{gamma-k} (eq. hat_J)
// the far interaction of a source cluster (S, J_k) with a target cluster
// (O, I_{k+q}) uses the truncated-power kernel U^2 of eq. U, interpolated in
// all eight variables on Chebyshev nodes (first kind):
//   K_phi = (c(t-s) - r)_+^2 / (r (c dt)^2)              (phi and P terms)
//   K_A   = d/dt K_phi = 2c (c(t-s) - r)_+ / (r (c dt)^2)  (A term, the second
//           time derivative goes on the target interpolant, eq. ddotA_fmm)
// Seven moment components: A (3, kernel K_A), phi (1) and mag (3) (kernel
// K_phi), eqs. ddotA_M, dotphi_fmm, P_fmm.
//
// Window truncation (exact; derived from Appendix A).  The far field of a
// target interval k' sums the sources of intervals k'-q_hi .. k'-1 only, with
// the Jh of the first 3 steps of interval k'-q_hi truncated at that interval's
// start: then sum_{gamma >= G} Jh_G^gamma U(...) = sum_{beta >= G} J^beta N(...)
// exactly, and every older current contributes N(tau) = 0 provided
// q_hi M_l >= 1 + r_max/(c dt).  Each source cluster therefore keeps a full and
// a truncated moment set; the truncated one serves q = q_hi of each pair.
//
// M2L operators are translation invariant and, since r depends only on |x-y|
// and the Chebyshev nodes are symmetric, invariant under the 48 symmetries of
// the cube: 16 canonical offsets (0 <= c1 <= c2 <= c3, c3 in {2, 3}) per level
// and lag q, applied to pairs through node-index maps.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>
#include <vector>

#include "internal.h"

namespace tdbem {

constexpr int kNC = 7;  // moment components: A x,y,z | phi | mag x,y,z

struct FmmLevel {
  int l = 0, ncell = 0, M = 0, Q = 0;
  double ds = 0, H = 0;
  std::vector<double> cen;        // host [ncell][3]
  std::vector<int> parent, leaf, tri_b, tri_e, icoord;  // icoord [ncell][3]
  std::vector<int> child;         // [ncell][8]
  // device
  double* d_cen = nullptr;
  int32_t* d_child = nullptr;     // [ncell][8]
  int32_t* d_leaf_cells = nullptr;  // leaf cell ids at this level
  int32_t* d_nonleaf_cells = nullptr;
  int nleaf = 0, nnonleaf = 0;
  int32_t* d_tri_b = nullptr;
  int32_t* d_tri_e = nullptr;
  float* mom = nullptr;           // [ncell][2 slot][2 var][kNC][P]
  float* loc = nullptr;           // [ncell][Q][kNC][P]
  // M2L
  int npairs = 0;
  int32_t* d_pO = nullptr;
  int32_t* d_pS = nullptr;
  int16_t* d_psym = nullptr;
  // distinct (source cell, symmetry) combinations of the pairs, in source
  // order, and each pair's combination (tensor-core M2L packing)
  int ncombo = 0;
  int32_t* d_pC = nullptr;
  int32_t* d_cS = nullptr;
  int16_t* d_csym = nullptr;
  float* ops = nullptr;           // [nop][2][P][P]
  uint4* ops_img = nullptr;       // the same in tensor-core shared-memory images (tensor-core M2L only)
  int nop = 0;
  int4* d_gemm = nullptr;         // {op index, pair base, npairs, kind | q << 8 | qhi << 16}
  int ngemm = 0;
  int4* d_tiles = nullptr;        // {gemm, row tile, col tile, 0}: 64 x 64 tiles (CUDA cores)
  int ntiles = 0;
  // tensor cores: {gemm, row-tile group, 128-column tile, 0} for groups of
  // mt = 1 or 2 128-row operator tiles per CTA; tc_mt is the shape the setup
  // autotuner measured faster for this level
  int4* d_tiles_tc[2] = {nullptr, nullptr};
  int ntiles_tc[2] = {0, 0};
  // every tile list holds first the tiles of lag q = 1 (their local
  // coefficients are read in the event that fires them), then those of
  // q >= 2 (read one interval later or after), which may be deferred
  int ntiles_urgent = 0;
  int ntiles_tc_urgent[2] = {0, 0};
  float* d_pack = nullptr;          // packed moments of this level's event (tensor-core M2L)
  float* d_pkinv = nullptr;         // their inverse row scales (FP16 form)
  float* d_opinv = nullptr;         // inverse operator scales (FP16 form)
  // FP16 form with P <= 256: the resident-operator kernel k_m2l_res, its work
  // units {gemm, 128-row tile, first 128-column tile, column tiles} (lag-1
  // units first) and its packed FP16 hi/lo moments
  bool res_ok = false;  // eligible (FP16 form, P <= 256)
  bool res = false;     // chosen by the autotuner
  float res_ms = 0.f;   // autotuner: mean time of one M2L event of the resident kernel
  int4* d_units = nullptr;
  int nunits = 0, nunits_urgent = 0;
  __half* d_pk16 = nullptr;
  cudaEvent_t ev_defer = nullptr;   // recorded on the side stream after a deferred M2L
  bool defer_pending = false;       // host: a deferred M2L not yet waited for
  int tc_mt = 1;
  float tc_ms[2] = {0.f, 0.f};     // autotuner: mean time of one M2L event per shape
  double flops_event = 0;         // M2L flops of one gating event
  // time tables: source/target factors for offsets i = 0..M-1
  float* d_tsrc = nullptr;        // [M][pt]  l_n(s_i)
  float* d_ttgt = nullptr;        // [M][3][pt]  l_m, l_m'/h_t, chi l_m'/h_t + zeta l_m
};

struct FmmPlan {
  int p = 4, pt = 4, PS = 64, P = 256;
  int lmax = 0, lfar = 2;  // far field at levels lfar..lmax
  double delta = 0, root[3] = {0, 0, 0}, D = 0;
  std::vector<FmmLevel> lev;
  int32_t* d_perm = nullptr;      // triangles in cell order
  float* d_W = nullptr;           // [nt][3][kNC][PS] P2M tables
  float* d_T = nullptr;           // [nt][3][kNC][PS] L2P tables
  int16_t* d_smap = nullptr;      // [48][PS] inverse node maps
  float* d_Sx = nullptr;          // per level pair (l -> l+1): [lev][2][p][p]
  float* d_St = nullptr;          // [2][pt][pt] (the same at every level)
  // near field (CSR over test edges)
  int64_t* d_row_ptr = nullptr;
  int32_t* d_col = nullptr;
  int16_t* d_mlo = nullptr;
  uint8_t* d_nlag = nullptr;
  int64_t* d_off = nullptr;
  double* d_val64 = nullptr;
  float* d_val32 = nullptr;
  // the near history flattened per test edge: for row i, entries hrow[i] ..
  // hrow[i+1]-1 hold a coefficient (FP32) and (column << 8) | lag, lags >= 2
  int64_t* d_hrow = nullptr;
  float* d_hval = nullptr;
  int32_t* d_hmeta = nullptr;
  // the same entries split by lag for the pipelined single-RHS march: the
  // lags >= 3 of step alpha + 2 need the currents up to J^{alpha-1} only, so
  // they are summed on the near stream while step alpha's solve runs; the
  // lag-2 entries (and the far field) are added once J^{alpha} is known
  int64_t* d_hrow2 = nullptr;
  float* d_hval2 = nullptr;
  int32_t* d_hmeta2 = nullptr;
  int64_t* d_hrow3 = nullptr;
  float* d_hval3 = nullptr;
  int32_t* d_hmeta3 = nullptr;
  double* d_Rp = nullptr;          // [2][ne] -(lags >= 3) of the step alpha in buffer alpha & 1
  // the lags >= 3 tiled by column blocks (k_near_tile): columns in Morton
  // order of their edges' midpoints, blocks of kNB consecutive ones; a
  // segment is one row's entries within one block (FP32 coefficient, and the
  // column's place in the block << 8 | lag as 16 bits), the segments block
  // by block; tasks (block, first and end segment) of at most kNTaskEntries
  // entries; per row its segments (ascending) for the fixed-order reduce
  int32_t* d_corder = nullptr;     // [ne] edge at sorted position k
  int64_t* d_seg_ptr = nullptr;    // [nseg + 1]
  float* d_cval = nullptr;         // [entries]
  uint16_t* d_cmeta = nullptr;     // [entries]
  int4* d_ntasks = nullptr;        // [ntask] {block, s0, s1, 0}
  int64_t* d_rseg_ptr = nullptr;   // [ne + 1]
  int32_t* d_rseg = nullptr;       // [nseg]
  double* d_spart = nullptr;       // [nseg] segment sums
  int64_t nseg = 0;
  int32_t ntask = 0;
  cudaStream_t nstream = nullptr;  // near stream (null: no pipelining)
  cudaEvent_t ev_solved = nullptr; // context stream: a solve has been enqueued
  cudaEvent_t ev_near[2] = {nullptr, nullptr};  // near stream: buffer b is written
  int32_t ahead[2] = {0, 0};       // step whose partial sum is in buffer b, launched ahead (0: none)
  int64_t nnz = 0, nval = 0, n_near_tri_pairs = 0;
  // far right-hand sides (targets ahead of the current step)
  int Lr = 0;
  double* d_Rfar = nullptr;       // [Lr][ne]
  int32_t* d_err = nullptr;       // bounded-wait timeouts of the tensor-core M2L
  // second stream for the deferred (q >= 2) M2L products, and the event that
  // orders it after the context's stream
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr;
  // second far state for history_eval
  std::vector<float*> mom_eval, loc_eval;
  double* d_Rfar_eval = nullptr;
  int32_t max_near_lag = 0;
};

// ---------------------------------------------------------------------------
// Lagrange polynomials on Chebyshev nodes of the first kind
__host__ __device__ inline double cheb_node(int a, int p) { return cos((2.0 * a + 1.0) * 3.14159265358979323846 / (2.0 * p)); }

__host__ __device__ inline void lagrange(int p, double x, double* l, double* dl) {
  double w[8];
  for (int a = 0; a < p; ++a) w[a] = cheb_node(a, p);
  for (int a = 0; a < p; ++a) {
    double v = 1.0, dv = 0.0;
    for (int b = 0; b < p; ++b) {
      if (b == a) continue;
      double f = 1.0 / (w[a] - w[b]);
      dv = dv * (x - w[b]) * f + v * f;
      v *= (x - w[b]) * f;
    }
    l[a] = v;
    if (dl) dl[a] = dv;
  }
}

// The paper's CHI (section 3.2), read as piecewise cubic Hermite interpolation
// on n >= 2 uniformly spaced nodes of [-1, 1] (the interval's ends included),
// the node derivatives being finite differences of the node values: central
// inside, second-order one-sided at the ends (first-order when n = 2).  It is
// linear in the node values and reproduces polynomials of degree 2.  l[j] is
// the interpolant of the node data e_j at x, dl and d2l its first two
// derivatives (either may be null).
__host__ __device__ inline double chi_node(int a, int n) { return -1.0 + 2.0 * a / (n - 1); }

// h times the finite-difference derivative at node q of the node data e_j
__host__ __device__ inline double chi_fd(int q, int j, int n) {
  auto f = [j](int r) { return r == j ? 1.0 : 0.0; };
  if (n == 2) return f(1) - f(0);
  if (q == 0) return 0.5 * (-3.0 * f(0) + 4.0 * f(1) - f(2));
  if (q == n - 1) return 0.5 * (3.0 * f(n - 1) - 4.0 * f(n - 2) + f(n - 3));
  return 0.5 * (f(q + 1) - f(q - 1));
}

__host__ __device__ inline void chi_basis(int n, double x, double* l, double* dl, double* d2l) {
  const double h = 2.0 / (n - 1);
  int k = (int)floor((x + 1.0) / h);
  k = k < 0 ? 0 : (k > n - 2 ? n - 2 : k);
  const double t = (x + 1.0) / h - k;
  // Hermite cubics on [0, 1]: values h00 h10 h01 h11, first (g) and second (s) derivatives in t
  const double h00 = 2 * t * t * t - 3 * t * t + 1, h10 = t * t * t - 2 * t * t + t;
  const double h01 = -2 * t * t * t + 3 * t * t, h11 = t * t * t - t * t;
  const double g00 = 6 * t * t - 6 * t, g10 = 3 * t * t - 4 * t + 1, g01 = -6 * t * t + 6 * t, g11 = 3 * t * t - 2 * t;
  const double s00 = 12 * t - 6, s10 = 6 * t - 4, s01 = -12 * t + 6, s11 = 6 * t - 2;
  for (int j = 0; j < n; ++j) {
    const double f0 = k == j ? 1.0 : 0.0, f1 = k + 1 == j ? 1.0 : 0.0;
    const double m0 = chi_fd(k, j, n), m1 = chi_fd(k + 1, j, n);
    l[j] = h00 * f0 + h10 * m0 + h01 * f1 + h11 * m1;
    if (dl) dl[j] = (g00 * f0 + g10 * m0 + g01 * f1 + g11 * m1) / h;
    if (d2l) d2l[j] = (s00 * f0 + s10 * m0 + s01 * f1 + s11 * m1) / (h * h);
  }
}

// Interpolation in space (tdbem_params.s_interp) and in time (t_interp):
// 0 Lagrange polynomials on the Chebyshev nodes above (degree n - 1), 1 CHI.
__host__ __device__ inline double interp_node(int a, int n, int interp) {
  return interp == 1 ? chi_node(a, n) : cheb_node(a, n);
}

__host__ __device__ inline void space_basis(int p, int interp, double x, double* l, double* dl) {
  if (interp == 1)
    chi_basis(p, x, l, dl, nullptr);
  else
    lagrange(p, x, l, dl);
}

// The vector potential's second time derivative (tdbem_params.a_deriv): how
// many of the two the interpolated kernel K_A carries, and which time factor
// of the L2P table the target takes (0 l, 1 l'/h_t, 3 l''/h_t^2).
inline int a_kernel_derivs(int a_deriv) { return a_deriv == 0 ? 1 : (a_deriv == 1 ? 0 : 2); }
inline int a_target_kind(int a_deriv) { return a_deriv == 0 ? 1 : (a_deriv == 1 ? 3 : 0); }

// l[a], l'[a], l''[a] of the time basis at x (any of dl, d2l may be null).
inline void time_basis(int pt, int interp, double x, double* l, double* dl, double* d2l) {
  if (interp == 1) {
    chi_basis(pt, x, l, dl, d2l);
    return;
  }
  // Lagrange: monomial coefficients of each cardinal polynomial, then Horner
  double w[8];
  for (int a = 0; a < pt; ++a) w[a] = cheb_node(a, pt);
  for (int a = 0; a < pt; ++a) {
    double cf[9] = {1.0};  // cf[k]: coefficient of x^k, degree grows to pt - 1
    int deg = 0;
    double den = 1.0;
    for (int b = 0; b < pt; ++b) {
      if (b == a) continue;
      for (int k = deg + 1; k >= 1; --k) cf[k] = cf[k - 1] - w[b] * cf[k];
      cf[0] = -w[b] * cf[0];
      ++deg;
      den *= w[a] - w[b];
    }
    double v = 0, d1 = 0, d2 = 0;
    for (int k = deg; k >= 0; --k) {
      d2 = d2 * x + 2.0 * d1;
      d1 = d1 * x + v;
      v = v * x + cf[k];
    }
    l[a] = v / den;
    if (dl) dl[a] = d1 / den;
    if (d2l) d2l[a] = d2 / den;
  }
}

// ---------------------------------------------------------------------------
// Setup kernels

// P2M table W[t][k][c][b] (exact collapsed-Gauss source rule, nq points) and
// L2P table T[t][k][c][a] (the 7-point outer rule), relative to the leaf box
// of each triangle.
__global__ void k_far_tables(TriGeom g, Phys ph, int p, int sint, int nt, const double* box /*[nt][4] centre, H*/,
                             const double* qu, const double* qwt, int nq1, float* W, float* T) {
  int t = blockIdx.x;
  if (t >= nt) return;
  const int PS = p * p * p;
  const double* v = g.v + 9 * t;
  const double cx = box[4 * t], cy = box[4 * t + 1], cz = box[4 * t + 2], H = box[4 * t + 3];
  const double A = g.area[t];
  const double PI = 3.14159265358979323846;
  double nin[3] = {-g.nrm[3 * t], -g.nrm[3 * t + 1], -g.nrm[3 * t + 2]};
  for (int e = threadIdx.x; e < 3 * PS; e += blockDim.x) {
    int k = e / PS, b = e % PS;
    int b1 = b / (p * p), b2 = (b / p) % p, b3 = b % p;
    double sg = g.sgn[3 * t + k], l = g.elen[3 * t + k];
    double cf = sg * l / (2 * A), dv = sg * l / A;
    const double* o = g.opp + 9 * t + 3 * k;
    double w[kNC] = {0, 0, 0, 0, 0, 0, 0};
    // source side: exact integral of f_j l_b, div f_j l_b, f_j x grad l_b
    for (int iu = 0; iu < nq1; ++iu)
      for (int iv = 0; iv < nq1; ++iv) {
        double u = qu[iu], vv = qu[iv];
        double l0 = u, l1 = (1 - u) * vv, l2 = (1 - u) * (1 - vv);
        double wt = 2 * A * (1 - u) * qwt[iu] * qwt[iv];
        double y[3];
        for (int q = 0; q < 3; ++q) y[q] = l0 * v[q] + l1 * v[3 + q] + l2 * v[6 + q];
        double L1[8], D1[8], L2[8], D2[8], L3[8], D3[8];
        space_basis(p, sint, (y[0] - cx) / H, L1, D1);
        space_basis(p, sint, (y[1] - cy) / H, L2, D2);
        space_basis(p, sint, (y[2] - cz) / H, L3, D3);
        double lb = L1[b1] * L2[b2] * L3[b3];
        double gr[3] = {D1[b1] * L2[b2] * L3[b3] / H, L1[b1] * D2[b2] * L3[b3] / H, L1[b1] * L2[b2] * D3[b3] / H};
        double f[3] = {cf * (y[0] - o[0]), cf * (y[1] - o[1]), cf * (y[2] - o[2])};
        w[0] += wt * f[0] * lb;
        w[1] += wt * f[1] * lb;
        w[2] += wt * f[2] * lb;
        w[3] += wt * dv * lb;
        w[4] += wt * (f[1] * gr[2] - f[2] * gr[1]);
        w[5] += wt * (f[2] * gr[0] - f[0] * gr[2]);
        w[6] += wt * (f[0] * gr[1] - f[1] * gr[0]);
      }
    // target side: 7-point rule, constants of eq. z_ij folded in
    double tv[kNC] = {0, 0, 0, 0, 0, 0, 0};
    const double kA = ph.mu / (4 * PI), kphi = 1.0 / (4 * PI * ph.eps), kP = ph.theta * ph.eta / (4 * PI);
    for (int q = 0; q < kNq; ++q) {
      double x[3];
      for (int u = 0; u < 3; ++u) x[u] = ph.qb[q][0] * v[u] + ph.qb[q][1] * v[3 + u] + ph.qb[q][2] * v[6 + u];
      double wq = ph.qw[q] * A;
      double L1[8], L2[8], L3[8];
      space_basis(p, sint, (x[0] - cx) / H, L1, nullptr);
      space_basis(p, sint, (x[1] - cy) / H, L2, nullptr);
      space_basis(p, sint, (x[2] - cz) / H, L3, nullptr);
      double la = L1[b1] * L2[b2] * L3[b3];
      double f[3] = {cf * (x[0] - o[0]), cf * (x[1] - o[1]), cf * (x[2] - o[2])};
      double fxn[3] = {f[1] * nin[2] - f[2] * nin[1], f[2] * nin[0] - f[0] * nin[2], f[0] * nin[1] - f[1] * nin[0]};
      tv[0] += wq * kA * f[0] * la;
      tv[1] += wq * kA * f[1] * la;
      tv[2] += wq * kA * f[2] * la;
      tv[3] += wq * kphi * dv * la;
      tv[4] += wq * kP * fxn[0] * la;
      tv[5] += wq * kP * fxn[1] * la;
      tv[6] += wq * kP * fxn[2] * la;
    }
    for (int c = 0; c < kNC; ++c) {
      W[(((int64_t)t * 3 + k) * kNC + c) * PS + b] = (float)w[c];
      T[(((int64_t)t * 3 + k) * kNC + c) * PS + b] = (float)tv[c];
    }
  }
}

// M2L operators of one level: for canonical offset cv[op] and lag qv[op],
// ops[op][kind][(a,m)][(b,n)], kind 0 = the vector potential's kernel K_A,
// 1 = K_phi.  kern selects the kernel pair (tdbem_params.far_kernel): 0 the
// truncated powers of the method, 1 the polynomial check kernel K_phi =
// (1 + r^2) T3(tau/(64 dt) - 1), 2 zero, 3 the check kernel with T2 for T3.  adeg is the number of time
// derivatives K_A carries (tdbem_params.a_deriv): 1 (the paper's split, the
// other on the target factor), 0 (both on the target factor) or 2 (both on the
// kernel).  interp places the time nodes (tdbem_params.t_interp).
__global__ void k_m2l_ops(int p, int pt, double ds, double H, double ht, int M, double dt, double cc, double a,
                          const int4* opdesc /* {c1,c2,c3,q} */, int nop, int kern, int adeg, int sint, int interp,
                          float* ops) {
  const int PS = p * p * p, P = PS * pt;
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t total = (int64_t)nop * P * P;
  if (e >= total) return;
  int op = (int)(e / ((int64_t)P * P));
  int rc = (int)(e % ((int64_t)P * P));
  int row = rc / P, col = rc % P;
  int4 d = opdesc[op];
  int aa = row / pt, m = row % pt, bb = col / pt, n = col % pt;
  int ai[3] = {aa / (p * p), (aa / p) % p, aa % p}, bi[3] = {bb / (p * p), (bb / p) % p, bb % p};
  int cv[3] = {d.x, d.y, d.z};
  double r2 = 0.0;
  for (int k = 0; k < 3; ++k) {
    double dx = cv[k] * ds + H * (interp_node(ai[k], p, sint) - interp_node(bi[k], p, sint));
    r2 += dx * dx;
  }
  double r = sqrt(r2);
  double tau = (d.w * M + 1) * dt + ht * (interp_node(m, pt, interp) - interp_node(n, pt, interp));
  double u = cc * tau - r;
  double kphi = 0.0, kA = 0.0;
  if (kern == 1) {
    // (1 + r^2) T3(tau/ts - 1), T3(x) = 4x^3 - 3x, ts = 64 dt, and its time derivatives
    const double g = 1.0 + r2, ts = 64.0 * dt, x = tau / ts - 1.0;
    kphi = g * (4.0 * x * x * x - 3.0 * x);
    kA = adeg == 0 ? kphi : (adeg == 1 ? g * (12.0 * x * x - 3.0) / ts : g * 24.0 * x / (ts * ts));
  } else if (kern == 3) {
    // (1 + r^2) T2(tau/ts - 1), T2(x) = 2x^2 - 1: degree 2 in every variable
    const double g = 1.0 + r2, ts = 64.0 * dt, x = tau / ts - 1.0;
    kphi = g * (2.0 * x * x - 1.0);
    kA = adeg == 0 ? kphi : (adeg == 1 ? g * 4.0 * x / ts : g * 4.0 / (ts * ts));
  } else if (kern == 0 && u > 0.0) {
    kphi = u * u / (r * a * a);
    kA = adeg == 0 ? kphi : (adeg == 1 ? 2.0 * cc * u / (r * a * a) : 2.0 * cc * cc / (r * a * a));
  }
  ops[((int64_t)op * 2 + 0) * P * P + rc] = (float)kA;
  ops[((int64_t)op * 2 + 1) * P * P + rc] = (float)kphi;
}

// ---------------------------------------------------------------------------
// Event kernels

// P2M at the leaves of one level for source interval k: one block per leaf.
// jh over the interval's M steps (full and truncated at the interval start),
// contracted with the time factors, then with the W table.
__global__ void k_p2m(const int32_t* leaf_cells, const int32_t* tri_b, const int32_t* tri_e, const int32_t* perm,
                      const TriGeom g, const float* W, const float* tsrc, const double* ring, int L, int p, int pt,
                      int M, int k, float* mom, int R) {
  extern __shared__ float sm[];
  const int PS = p * p * p, P = PS * pt;
  const int rhs = blockIdx.y;  // right-hand side of this block
  int cell = leaf_cells[blockIdx.x];
  int tb = tri_b[cell], te_ = tri_e[cell];
  int ntk = 3 * (te_ - tb);
  float* jt = sm;  // [ntk][2][pt]
  const double w4[4] = {0.5, -1.5, 1.5, -0.5};
  const int G = k * M;
  for (int e = threadIdx.x; e < ntk; e += blockDim.x) {
    int t = perm[tb + e / 3], kk = e % 3;
    int j = g.edge[3 * t + kk];
    const double* Jr = ring + (int64_t)j * L * R + rhs;
    double acc[2][8];
    for (int v = 0; v < 2; ++v)
      for (int n = 0; n < pt; ++n) acc[v][n] = 0.0;
    for (int i = 0; i < M; ++i) {
      int gam = G + i;
      double full = 0.0, trunc = 0.0;
      for (int kap = 0; kap <= 3; ++kap) {
        int b = gam - kap;
        if (b < 0) continue;
        double jv = w4[kap] * Jr[(int64_t)(b & (L - 1)) * R];
        full += jv;
        if (kap <= i) trunc += jv;
      }
      for (int n = 0; n < pt; ++n) {
        acc[0][n] += full * tsrc[i * pt + n];
        acc[1][n] += trunc * tsrc[i * pt + n];
      }
    }
    for (int v = 0; v < 2; ++v)
      for (int n = 0; n < pt; ++n) jt[(e * 2 + v) * pt + n] = (float)acc[v][n];
  }
  __syncthreads();
  float* out = mom + (((int64_t)cell * 2 + (k & 1)) * 2 * R + rhs) * kNC * P;  // variant stride R kNC P
  const int64_t vstr = (int64_t)R * kNC * P;
  // the grid's z dimension splits a cell's (component, node) outputs over
  // several blocks (each recomputes the cheap time moments above)
  for (int e = blockIdx.z * blockDim.x + threadIdx.x; e < kNC * PS; e += gridDim.z * blockDim.x) {
    int c = e / PS, b = e % PS;
    float a0[8], a1[8];
    for (int n = 0; n < pt; ++n) a0[n] = a1[n] = 0.f;
    for (int q = 0; q < ntk; ++q) {
      int t = perm[tb + q / 3], kk = q % 3;
      float wv = W[(((int64_t)t * 3 + kk) * kNC + c) * PS + b];
      for (int n = 0; n < pt; ++n) {
        a0[n] += wv * jt[(q * 2 + 0) * pt + n];
        a1[n] += wv * jt[(q * 2 + 1) * pt + n];
      }
    }
    for (int n = 0; n < pt; ++n) {
      out[(int64_t)c * P + b * pt + n] = a0[n];
      out[vstr + (int64_t)c * P + b * pt + n] = a1[n];
    }
  }
}

// M2M: parent moments of source interval k from the children's intervals 2k
// (slot 0) and 2k+1 (slot 1); the truncated parent set takes the truncated
// set of child interval 2k and the full set of 2k+1.
__global__ void k_m2m(const int32_t* cells, const int32_t* child, const float* Sx /*[2][p][p]*/, const float* St,
                      int p, int pt, int k, const float* cmom, float* pmom, int R) {
  const int PS = p * p * p, P = PS * pt;
  const int rhs = blockIdx.y;
  int cell = cells[blockIdx.x];
  float* out = pmom + ((int64_t)cell * 2 + (k & 1)) * 2 * R * kNC * P;
  for (int e = threadIdx.x; e < 2 * kNC * P; e += blockDim.x) {
    int var = e / (kNC * P), r = e % (kNC * P);
    int c = r / P, bn = r % P;
    int b = bn / pt, n = bn % pt;
    int b1 = b / (p * p), b2 = (b / p) % p, b3 = b % p;
    float s = 0.f;
    for (int o = 0; o < 8; ++o) {
      int ch = child[cell * 8 + o];
      if (ch < 0) continue;
      int sx = (o >> 2) & 1, sy = (o >> 1) & 1, sz = o & 1;
      for (int h = 0; h < 2; ++h) {
        int cvar = (var == 1 && h == 0) ? 1 : 0;
        const float* src = cmom + ((((int64_t)ch * 2 + h) * 2 + cvar) * R + rhs) * kNC * P + (int64_t)c * P;
        for (int n2 = 0; n2 < pt; ++n2) {
          float tt = St[(h * pt + n) * pt + n2];
          if (tt == 0.f) continue;
          for (int c1 = 0; c1 < p; ++c1) {
            float f1 = Sx[(sx * p + b1) * p + c1] * tt;
            for (int c2 = 0; c2 < p; ++c2) {
              float f2 = f1 * Sx[(sy * p + b2) * p + c2];
              const float* s3 = src + ((c1 * p + c2) * p) * pt + n2;
              for (int c3 = 0; c3 < p; ++c3) s += f2 * Sx[(sz * p + b3) * p + c3] * s3[c3 * pt];
            }
          }
        }
      }
    }
    out[((int64_t)var * R + rhs) * kNC * P + c * P + bn] = s;
  }
}

// One 1-D contraction of nch tensors [p][p][p][pt] (channel stride P) along
// `axis` (0..2 space, 3 time): out[.., j, ..] = sum_i M(j, i) in[.., i, ..]
// with M(j, i) = mat[j*n + i] (trans = 0) or mat[i*n + j] (trans = 1).
__device__ __forceinline__ void contract_axis(const float* in, float* out, const float* mat, bool trans, int axis,
                                              int p, int pt, int nch) {
  const int PS = p * p * p, P = PS * pt;
  const int n = axis == 3 ? pt : p;
  const int stride = axis == 3 ? 1 : (axis == 2 ? pt : (axis == 1 ? p * pt : p * p * pt));
  for (int e = threadIdx.x; e < nch * P; e += blockDim.x) {
    int ch = e / P, r = e % P;
    int j = (r / stride) % n;
    const float* src = in + (int64_t)ch * P + (r - j * stride);
    float acc = 0.f;
    for (int i = 0; i < n; ++i) acc += (trans ? mat[i * n + j] : mat[j * n + i]) * src[i * stride];
    out[e] = acc;
  }
  __syncthreads();
}

// M2M, factorised: for each child and half-interval, the 14 channels (7
// components x full/truncated) are interpolated one axis at a time and
// accumulated into the parent moments of source interval k.  The grid's z
// dimension splits the channels over blocks (per = ceil(14 / gridDim.z)
// channels each; shared memory 3 per P floats).
__global__ void k_m2m_fact(const int32_t* cells, const int32_t* child, const float* Sx, const float* St, int p, int pt,
                           int k, const float* cmom, float* pmom, int R) {
  extern __shared__ float sm[];
  const int PS = p * p * p, P = PS * pt, nct = 2 * kNC;
  const int per = (nct + gridDim.z - 1) / gridDim.z, c0 = blockIdx.z * per, nch = min(per, nct - c0);
  if (nch <= 0) return;
  const int rhs = blockIdx.y;
  const int64_t vstr = (int64_t)R * kNC * P;  // stride of the full/truncated variant
  float* b0 = sm;
  float* b1 = sm + nch * P;
  float* acc = sm + 2 * nch * P;
  int cell = cells[blockIdx.x];
  for (int e = threadIdx.x; e < nch * P; e += blockDim.x) acc[e] = 0.f;
  for (int o = 0; o < 8; ++o) {
    int ch = child[cell * 8 + o];
    if (ch < 0) continue;
    int sx = (o >> 2) & 1, sy = (o >> 1) & 1, sz = o & 1;
    for (int h = 0; h < 2; ++h) {
      const float* src = cmom + ((int64_t)ch * 2 + h) * 2 * vstr + (int64_t)rhs * kNC * P;
      __syncthreads();
      for (int e = threadIdx.x; e < nch * P; e += blockDim.x) {
        const int gc = c0 + e / P;  // channel: variant * kNC + component
        int var = gc / kNC, r = (gc % kNC) * P + e % P;
        int cvar = (var == 1 && h == 0) ? 1 : 0;  // truncated parent = truncated first half + full second half
        b0[e] = src[(int64_t)cvar * vstr + r];
      }
      __syncthreads();
      contract_axis(b0, b1, St + h * pt * pt, false, 3, p, pt, nch);
      contract_axis(b1, b0, Sx + sz * p * p, false, 2, p, pt, nch);
      contract_axis(b0, b1, Sx + sy * p * p, false, 1, p, pt, nch);
      contract_axis(b1, b0, Sx + sx * p * p, false, 0, p, pt, nch);
      for (int e = threadIdx.x; e < nch * P; e += blockDim.x) acc[e] += b0[e];
    }
  }
  __syncthreads();
  float* out = pmom + ((int64_t)cell * 2 + (k & 1)) * 2 * vstr + (int64_t)rhs * kNC * P;
  for (int e = threadIdx.x; e < nch * P; e += blockDim.x) {
    const int gc = c0 + e / P;
    int var = gc / kNC, r = (gc % kNC) * P + e % P;
    out[(int64_t)var * vstr + r] = acc[e];
  }
}

// L2L, factorised (transposed interpolation): the parent's local coefficients
// of interval k+1 are evaluated at each child's nodes for the child intervals
// 2(k+1) and 2(k+1)+1 and added there; the parent slot is then cleared.
__global__ void k_l2l_fact(const int32_t* cells, const int32_t* child, const float* Sx, const float* St, int p, int pt,
                           int k, float* ploc, int Qp, float* cloc, int Qc, int R) {
  extern __shared__ float sm[];
  const int PS = p * p * p, P = PS * pt;
  // components c0 .. c0 + nch - 1 (the grid's z dimension splits the 7)
  const int per = (kNC + gridDim.z - 1) / gridDim.z, c0 = blockIdx.z * per, nch = min(per, kNC - c0);
  if (nch <= 0) return;
  const int rhs = blockIdx.y;
  float* b0 = sm;
  float* b1 = sm + nch * P;
  float* par = sm + 2 * nch * P;
  int cell = cells[blockIdx.x];
  float* src = ploc + (((int64_t)cell * Qp + ((k + 1) % Qp)) * R + rhs) * kNC * P + (int64_t)c0 * P;
  for (int e = threadIdx.x; e < nch * P; e += blockDim.x) par[e] = src[e];
  for (int o = 0; o < 8; ++o) {
    int ch = child[cell * 8 + o];
    if (ch < 0) continue;
    int sx = (o >> 2) & 1, sy = (o >> 1) & 1, sz = o & 1;
    for (int h = 0; h < 2; ++h) {
      __syncthreads();
      contract_axis(par, b0, St + h * pt * pt, true, 3, p, pt, nch);
      contract_axis(b0, b1, Sx + sz * p * p, true, 2, p, pt, nch);
      contract_axis(b1, b0, Sx + sy * p * p, true, 1, p, pt, nch);
      contract_axis(b0, b1, Sx + sx * p * p, true, 0, p, pt, nch);
      int slot = (2 * (k + 1) + h) % Qc;
      float* dst = cloc + (((int64_t)ch * Qc + slot) * R + rhs) * kNC * P + (int64_t)c0 * P;
      for (int e = threadIdx.x; e < nch * P; e += blockDim.x) dst[e] += b1[e];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nch * P; e += blockDim.x) src[e] = 0.f;
}

// M2L as a batch of dense GEMMs on CUDA cores (FP32): for every (canonical
// offset, lag q, kernel kind) the operator (P x P) multiplies the gathered
// moments of all pairs of that offset class; results are added to the target
// local coefficients of interval k+q.  Tile 64 x 64, 256 threads, 4 x 4 each.
__global__ void __launch_bounds__(256) k_m2l_fp32(const int4* gemm, const int4* tiles, const float* ops, int P, int pt,
                                                  int PS, const int32_t* pO, const int32_t* pS, const int16_t* psym,
                                                  const int16_t* smap, const float* mom, int k, float* loc, int Q,
                                                  int R) {
  __shared__ float As[16][64 + 4];
  __shared__ float Bs[16][64 + 4];
  int4 tl = tiles[blockIdx.x];
  int4 gd = gemm[tl.x];
  const int kind = gd.w & 0xff, q = (gd.w >> 8) & 0xff, qhi = (gd.w >> 16) & 0xff;
  const int nk = kind == 0 ? 3 : 4, c0 = kind == 0 ? 0 : 3;
  const int var = (q == qhi) ? 1 : 0;
  const float* A = ops + ((int64_t)gd.x * 2 + (kind == 0 ? 0 : 1)) * P * P;
  const int row0 = tl.y * 64, col0 = tl.z * 64;
  const int ncol = gd.z * nk * R;  // columns (pair, right-hand side, component)
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float acc[4][4] = {};
  // column descriptors of this thread's B loads (column = threadIdx.x & 63)
  int lc = threadIdx.x & 63;
  int gcol = col0 + lc;
  const float* bsrc = nullptr;
  const int16_t* bmap = nullptr;
  if (gcol < ncol) {
    int pr = gd.y + gcol / (nk * R), rem = gcol % (nk * R), rhs = rem / nk, c = c0 + rem % nk;
    bsrc = mom + (((((int64_t)pS[pr] * 2 + (k & 1)) * 2 + var) * R + rhs) * kNC + c) * P;
    bmap = smap + (int64_t)psym[pr] * PS;
  }
  for (int k0 = 0; k0 < P; k0 += 16) {
    for (int e = threadIdx.x; e < 64 * 16; e += 256) {
      int rr = e / 16, kk = e % 16;
      As[kk][rr] = (row0 + rr < P && k0 + kk < P) ? A[(int64_t)(row0 + rr) * P + k0 + kk] : 0.f;
    }
    for (int kk = threadIdx.x >> 6; kk < 16; kk += 4) {
      float v = 0.f;
      if (bsrc && k0 + kk < P) {
        int kidx = k0 + kk;
        int bp = kidx / pt, n = kidx % pt;
        v = bsrc[bmap[bp] * pt + n];
      }
      Bs[kk][lc] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
  }
  for (int j = 0; j < 4; ++j) {
    int gc = col0 + tx * 4 + j;
    if (gc >= ncol) continue;
    int pr = gd.y + gc / (nk * R), rem = gc % (nk * R), rhs = rem / nk, c = c0 + rem % nk;
    const int16_t* map = smap + (int64_t)psym[pr] * PS;
    float* dst = loc + ((((int64_t)pO[pr] * Q + ((k + q) % Q)) * R + rhs) * kNC + c) * P;
    for (int i = 0; i < 4; ++i) {
      int row = row0 + ty * 4 + i;
      if (row >= P) continue;
      int ap = row / pt, m = row % pt;
      atomicAdd(dst + map[ap] * pt + m, acc[i][j]);
    }
  }
}

// L2L: children's local coefficients of intervals 2(k+1), 2(k+1)+1 from the
// parent's (interval k+1); then the parent slot is cleared.
__global__ void k_l2l(const int32_t* cells, const int32_t* child, const float* Sx, const float* St, int p, int pt,
                      int k, float* ploc, int Qp, float* cloc, int Qc, int R) {
  const int PS = p * p * p, P = PS * pt;
  const int rhs = blockIdx.y;
  int cell = cells[blockIdx.x];
  float* src = ploc + (((int64_t)cell * Qp + ((k + 1) % Qp)) * R + rhs) * kNC * P;
  for (int o = 0; o < 8; ++o) {
    int ch = child[cell * 8 + o];
    if (ch < 0) continue;
    int sx = (o >> 2) & 1, sy = (o >> 1) & 1, sz = o & 1;
    for (int e = threadIdx.x; e < 2 * kNC * P; e += blockDim.x) {
      int h = e / (kNC * P), r = e % (kNC * P);
      int c = r / P, an = r % P;
      int a = an / pt, m2 = an % pt;
      int a1 = a / (p * p), a2 = (a / p) % p, a3 = a % p;
      const float* s = src + (int64_t)c * P;
      float acc = 0.f;
      for (int m = 0; m < pt; ++m) {
        float tt = St[(h * pt + m) * pt + m2];
        if (tt == 0.f) continue;
        for (int c1 = 0; c1 < p; ++c1) {
          float f1 = Sx[(sx * p + c1) * p + a1] * tt;
          for (int c2 = 0; c2 < p; ++c2) {
            float f2 = f1 * Sx[(sy * p + c2) * p + a2];
            const float* s3 = s + ((c1 * p + c2) * p) * pt + m;
            for (int c3 = 0; c3 < p; ++c3) acc += f2 * Sx[(sz * p + c3) * p + a3] * s3[c3 * pt];
          }
        }
      }
      int slot = (2 * (k + 1) + h) % Qc;
      cloc[(((int64_t)ch * Qc + slot) * R + rhs) * kNC * P + (int64_t)c * P + an] += acc;
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < kNC * P; e += blockDim.x) src[e] = 0.f;
}

// L2P at the leaves of one level for target interval k+1: every target step
// rho of the interval receives -(far history) in the far right-hand side ring;
// the local-coefficient slot is cleared afterwards.
__global__ void k_l2p(const int32_t* leaf_cells, const int32_t* tri_b, const int32_t* tri_e, const int32_t* perm,
                      const TriGeom g, const float* T, const float* ttgt, int p, int pt, int M, int k, float* loc,
                      int Q, double* Rfar, int Lr, int64_t ne, int R, int s0, int ns, int clear, int akind) {
  extern __shared__ float sm[];
  const int PS = p * p * p, P = PS * pt;
  const int rhs = blockIdx.y;
  int cell = leaf_cells[blockIdx.x];
  float* L = loc + (((int64_t)cell * Q + ((k + 1) % Q)) * R + rhs) * kNC * P;
  // steps s0 .. s0 + ns - 1 of the interval (several launches when the
  // interval's evaluated coefficients exceed shared memory); the last clears
  // the consumed local coefficients
  float* Le = sm;  // [ns][kNC][PS]
  for (int e = threadIdx.x; e < ns * kNC * PS; e += blockDim.x) {
    int i = s0 + e / (kNC * PS), r = e % (kNC * PS);
    int c = r / PS, a = r % PS;
    // A: l' (or l'' / l by the placement of its time derivatives), phi: l, mag: chi l' + zeta l
    int kind = (c < 3) ? akind : (c == 3 ? 0 : 2);
    float s = 0.f;
    for (int m = 0; m < pt; ++m) s += L[(int64_t)c * P + a * pt + m] * ttgt[(i * 4 + kind) * pt + m];
    Le[e] = s;
  }
  __syncthreads();
  int tb = tri_b[cell], te_ = tri_e[cell];
  int ntk = 3 * (te_ - tb);
  // one warp per (triangle, side): the lanes stride the row of T (coalesced,
  // read once per 8 steps) and the rows of Le (consecutive words, no bank
  // conflicts); the 8 partial dot products are then summed across the warp
  constexpr int kSt = 8;
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int nr = kNC * PS;
  for (int q = threadIdx.x >> 5; q < ntk; q += nw) {
    const int t = perm[tb + q / 3], kk = q % 3;
    const float* Tt = T + ((int64_t)t * 3 + kk) * nr;
    const int64_t edge = g.edge[3 * t + kk];
    for (int i0 = 0; i0 < ns; i0 += kSt) {
      float acc[kSt];
#pragma unroll
      for (int u = 0; u < kSt; ++u) acc[u] = 0.f;
      for (int r = lane; r < nr; r += 32) {
        const float tv = __ldg(Tt + r);
#pragma unroll
        for (int u = 0; u < kSt; ++u)
          if (i0 + u < ns) acc[u] += tv * Le[(int64_t)(i0 + u) * nr + r];
      }
#pragma unroll
      for (int u = 0; u < kSt; ++u)
        for (int o = 16; o > 0; o >>= 1) acc[u] += __shfl_xor_sync(0xffffffffu, acc[u], o);
      if (lane < kSt && i0 + lane < ns) {
        float sv = acc[0];
#pragma unroll
        for (int u = 1; u < kSt; ++u)
          if (lane == u) sv = acc[u];
        const int rho = (k + 1) * M + s0 + i0 + lane;
        atomicAdd(Rfar + ((int64_t)(rho & (Lr - 1)) * ne + edge) * R + rhs, -(double)sv);
      }
    }
  }
  if (!clear) return;
  __syncthreads();
  for (int e = threadIdx.x; e < kNC * P; e += blockDim.x) L[e] = 0.f;
}

// Near field, flattened form: a warp streams its row's (coefficient,
// column << 8 | lag) entries with coalesced loads; every lane does the same
// work, and the lags of one column are neighbours in the history ring.
// R_i = V_i + V2_i + Rfar_i - sum over the row's entries of z J_col^{alpha-m}
// (V, V2 and Rfar may be null).
__global__ void __launch_bounds__(256) k_near_history_flat(const int64_t* hrow, const float* hval, const int32_t* hmeta,
                                                          int64_t ne, const double* ring, int L, int alpha,
                                                          const double* V, const double* V2, double* Rfar_slot,
                                                          double* R) {
  int64_t i = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
  int lane = threadIdx.x & 31;
  if (i >= ne) return;
  const int64_t e0 = hrow[i], e1 = hrow[i + 1];
  float s0 = 0.f, s1 = 0.f;
  int64_t e = e0 + lane;
  for (; e + 32 < e1; e += 64) {
    const float z0 = __ldg(hval + e), z1 = __ldg(hval + e + 32);
    const int q0 = __ldg(hmeta + e), q1 = __ldg(hmeta + e + 32);
    const int b0 = alpha - (q0 & 0xff), b1 = alpha - (q1 & 0xff);
    if (b0 >= 0) s0 += z0 * (float)ring[(int64_t)(q0 >> 8) * L + (b0 & (L - 1))];
    if (b1 >= 0) s1 += z1 * (float)ring[(int64_t)(q1 >> 8) * L + (b1 & (L - 1))];
  }
  if (e < e1) {
    const int q0 = __ldg(hmeta + e);
    const int b0 = alpha - (q0 & 0xff);
    if (b0 >= 0) s0 += __ldg(hval + e) * (float)ring[(int64_t)(q0 >> 8) * L + (b0 & (L - 1))];
  }
  double d = (double)s0 + (double)s1;
  for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
  if (lane == 0) {
    double far = Rfar_slot ? Rfar_slot[i] : 0.0;
    R[i] = (V ? V[i] : 0.0) + (V2 ? V2[i] : 0.0) + far - d;
    if (Rfar_slot) Rfar_slot[i] = 0.0;
  }
}

// ---------------------------------------------------------------------------
// Near field, lags >= 3, tiled by column blocks.  One CTA per task: it stages
// the block's history for the lags the entries use (up to the largest stored
// near-field lag), hist[m][c] = J^{alpha-m} of the block's column c (FP32:
// the products are FP32, as in the flat kernel), zero for m < m_min or m >
// alpha; then each warp takes one segment (one row's entries within the
// block) at a time, its lanes striding the entries with the history read
// from shared memory, and writes the segment's sum.  k_near_seg_reduce adds
// each row's segment sums in a fixed order: R_i = -sum.
constexpr int kNB = 128;              // columns per block
constexpr int kNBS = kNB + 1;         // row stride of the staged block (no bank conflicts when staging)
constexpr int kNTaskEntries = 16384;  // entries per task (about)

__global__ void __launch_bounds__(256) k_near_tile(const int4* tasks, const int32_t* corder, const int64_t* seg_ptr,
                                                   const float* cval, const uint16_t* cmeta, int64_t ne,
                                                   const double* ring, int L, int nlag, int alpha, int m_min,
                                                   double* spart) {
  extern __shared__ float nh[];  // [nlag][kNBS]: the lags 0 .. nlag - 1 the entries use
  const int4 tk = tasks[blockIdx.x];
  const int64_t p0 = (int64_t)tk.x * kNB;
  for (int k = threadIdx.x; k < kNB * nlag; k += blockDim.x) {
    const int cb = k / nlag, m = k - cb * nlag;  // consecutive threads: one column's ring row
    float v = 0.f;
    if (p0 + cb < ne && m >= m_min && m <= alpha)
      v = (float)ring[(int64_t)corder[p0 + cb] * L + ((alpha - m) & (L - 1))];
    nh[m * kNBS + cb] = v;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int sg = tk.y + warp; sg < tk.z; sg += nw) {
    const int64_t e1 = seg_ptr[sg + 1];
    float a0 = 0.f, a1 = 0.f;
    int64_t e = seg_ptr[sg] + lane;
    for (; e + 32 < e1; e += 64) {
      const uint32_t q0 = cmeta[e], q1 = cmeta[e + 32];
      a0 += __ldg(cval + e) * nh[(q0 & 0xff) * kNBS + (q0 >> 8)];
      a1 += __ldg(cval + e + 32) * nh[(q1 & 0xff) * kNBS + (q1 >> 8)];
    }
    if (e < e1) {
      const uint32_t q0 = cmeta[e];
      a0 += __ldg(cval + e) * nh[(q0 & 0xff) * kNBS + (q0 >> 8)];
    }
    double d = (double)a0 + (double)a1;
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    if (lane == 0) spart[sg] = d;
  }
}

// R_i = -(the sums of row i's segments), eight lanes per row, fixed order
__global__ void k_near_seg_reduce(const int64_t* rseg_ptr, const int32_t* rseg, const double* spart, int64_t ne,
                                  double* R) {
  const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 8;
  const int sub = threadIdx.x % 8;
  double t = 0.0;
  if (i < ne)
    for (int64_t k = rseg_ptr[i] + sub; k < rseg_ptr[i + 1]; k += 8) t += spart[rseg[k]];
#pragma unroll
  for (int d = 4; d > 0; d >>= 1) t += __shfl_xor_sync(0xffffffffu, t, d);
  if (i < ne && sub == 0) R[i] = -t;
}

// Batched near field on the flattened entries: one block per row; thread t
// takes right-hand side r0 + t mod RL (RL = R rounded up to a power of two,
// at most 32) and the row's entries sub, sub + nsub, ... (sub = t / RL), so
// each entry's coefficient is read once per lane group and its history
// R-vector contiguously; partial sums meet in shared memory.
__global__ void __launch_bounds__(256) k_near_history_flat_multi(const int64_t* hrow, const float* hval,
                                                                const int32_t* hmeta, int64_t ne, const double* ring,
                                                                int L, int alpha, int R, int RL, const double* V,
                                                                double* Rfar_slot, double* Rout) {
  __shared__ double red[8][32];
  const int64_t i = blockIdx.x;
  const int rr = threadIdx.x % RL, sub = threadIdx.x / RL, nsub = blockDim.x / RL;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t e0 = hrow[i], e1 = hrow[i + 1];
  for (int r0 = 0; r0 < R; r0 += RL) {
    const int r = r0 + rr;
    float s = 0.f;
    if (r < R) {
      for (int64_t e = e0 + sub; e < e1; e += nsub) {
        const int q = __ldg(hmeta + e);
        const int b = alpha - (q & 0xff);
        if (b >= 0) s += __ldg(hval + e) * (float)ring[((int64_t)(q >> 8) * L + (b & (L - 1))) * R + r];
      }
    }
    double d = s;
    for (int o = 16; o >= RL; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    if (lane < RL) red[warp][lane] = d;
    __syncthreads();
    if (threadIdx.x < RL && r0 + (int)threadIdx.x < R) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w][threadIdx.x];
      const int64_t q = i * R + r0 + threadIdx.x;
      const double far = Rfar_slot ? Rfar_slot[q] : 0.0;
      Rout[q] = (V ? V[q] : 0.0) + far - t;
      if (Rfar_slot) Rfar_slot[q] = 0.0;
    }
    __syncthreads();
  }
}

__global__ void k_f64_to_f32(const double* a, float* b, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

}  // namespace tdbem

using namespace tdbem;

// ---------------------------------------------------------------------------
// Host planner

namespace {

struct TreeBuild {
  const std::vector<double>* cen;
  std::vector<int>* perm;
  std::vector<FmmLevel>* lev;
  double root[3];
  double D;
  int lcap;
  int n_leaf;
};

void build_cell(TreeBuild& tb, int l, int ix, int iy, int iz, int b, int e, int parent) {
  std::vector<FmmLevel>& lev = *tb.lev;
  if ((int)lev.size() <= l) lev.resize(l + 1);
  FmmLevel& L = lev[l];
  int id = L.ncell++;
  double ds = tb.D / (1 << l);
  L.cen.push_back(tb.root[0] + (ix + 0.5) * ds);
  L.cen.push_back(tb.root[1] + (iy + 0.5) * ds);
  L.cen.push_back(tb.root[2] + (iz + 0.5) * ds);
  L.icoord.push_back(ix);
  L.icoord.push_back(iy);
  L.icoord.push_back(iz);
  L.parent.push_back(parent);
  L.tri_b.push_back(b);
  L.tri_e.push_back(e);
  for (int o = 0; o < 8; ++o) L.child.push_back(-1);
  bool split = 1.5 * (e - b) > tb.n_leaf && l < tb.lcap;
  L.leaf.push_back(split ? 0 : 1);
  if (!split) return;
  // partition [b, e) into octants
  std::vector<int>& P = *tb.perm;
  const std::vector<double>& C = *tb.cen;
  double mid[3] = {tb.root[0] + (ix + 0.5) * ds, tb.root[1] + (iy + 0.5) * ds, tb.root[2] + (iz + 0.5) * ds};
  std::vector<int> bucket[8];
  for (int q = b; q < e; ++q) {
    int t = P[q];
    int o = ((C[3 * t] >= mid[0]) << 2) | ((C[3 * t + 1] >= mid[1]) << 1) | (C[3 * t + 2] >= mid[2]);
    bucket[o].push_back(t);
  }
  int pos = b;
  int starts[8];
  for (int o = 0; o < 8; ++o) {
    starts[o] = pos;
    for (int t : bucket[o]) P[pos++] = t;
  }
  for (int o = 0; o < 8; ++o) {
    if (bucket[o].empty()) continue;
    int cid = (int)((int)lev.size() > l + 1 ? lev[l + 1].ncell : 0);
    lev[l].child[8 * id + o] = cid;
    build_cell(tb, l + 1, 2 * ix + ((o >> 2) & 1), 2 * iy + ((o >> 1) & 1), 2 * iz + (o & 1), starts[o],
               starts[o] + (int)bucket[o].size(), id);
  }
}

void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w) {
  x.resize(n);
  w.resize(n);
  const double PI = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double z = cos(PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      double dp = n * (z * p1 - p0) / (z * z - 1);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    double p0 = 1, p1 = z;
    for (int k = 2; k <= n; ++k) {
      double p2 = ((2.0 * k - 1) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    double dp = n * (z * p1 - p0) / (z * z - 1);
    x[i] = 0.5 * (z + 1);
    w[i] = 1.0 / ((1 - z * z) * dp * dp);  // (2/((1-z^2)P'^2)) / 2
  }
}

}  // namespace

tdbem_status tdbem_build_fast(tdbem_ctx* c) {
  FmmPlan* F = new (std::nothrow) FmmPlan();
  if (!F) return TDBEM_ENOMEM;
  c->fmm = F;
  const int p = c->p.p_s, pt = c->p.p_t;
  F->p = p;
  F->pt = pt;
  F->PS = p * p * p;
  F->P = F->PS * pt;
  const int PS = F->PS, P = F->P;
  const int64_t nt = c->nt, ne = c->ne;
  const double a = c->phys.a;
  // centroids, delta, root cube
  std::vector<double> cen(3 * nt);
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t v = 0; v < c->nv; ++v)
    for (int q = 0; q < 3; ++q) {
      lo[q] = std::min(lo[q], c->V[3 * v + q]);
      hi[q] = std::max(hi[q], c->V[3 * v + q]);
    }
  for (int64_t t = 0; t < nt; ++t)
    for (int q = 0; q < 3; ++q)
      cen[3 * t + q] = (c->V[3 * c->T[3 * t] + q] + c->V[3 * c->T[3 * t + 1] + q] + c->V[3 * c->T[3 * t + 2] + q]) / 3.0;
  F->delta = c->max_quad_rad;
  double D = std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2])) * (1 + 1e-9);
  F->D = D;
  for (int q = 0; q < 3; ++q) F->root[q] = lo[q];
  // deepest level whose intervals still hold d+1 steps
  int lcap = 0;
  for (int l = 0; l < 30; ++l) {
    double ds = D / (1 << l);
    if (std::floor((ds - 2 * F->delta) / a) >= 3) lcap = l;
  }
  std::vector<int> perm(nt);
  std::iota(perm.begin(), perm.end(), 0);
  TreeBuild tb{&cen, &perm, &F->lev, {lo[0], lo[1], lo[2]}, D, lcap, c->p.n_leaf};
  build_cell(tb, 0, 0, 0, 0, 0, (int)nt, -1);
  F->lmax = (int)F->lev.size() - 1;
  const int lmax = F->lmax;
  for (int l = 0; l <= lmax; ++l) {
    F->lev[l].l = l;
    F->lev[l].ds = D / (1 << l);
    F->lev[l].H = F->lev[l].ds / 2 + F->delta;
  }
  bool far = lmax >= 2;
  int Mlmax = far ? (int)std::floor((F->lev[lmax].ds - 2 * F->delta) / a) : 0;
  if (far && Mlmax < 3) {
    c->set_error("fast: time interval of the finest level holds fewer than d+1 steps");
    return TDBEM_EBREAKDOWN;
  }
  for (int l = 0; l <= lmax; ++l) F->lev[l].M = far ? Mlmax << (lmax - l) : 0;
  // ---- near triangle pairs and interaction lists
  std::vector<int2> near;
  int64_t far_count = 0;
  std::vector<std::vector<int>> il_pairs(lmax + 1);  // flat (O, S, ox, oy, oz)
  for (int l = 0; l <= lmax; ++l) {
    FmmLevel& L = F->lev[l];
    // hash of cells by integer coordinates
    std::vector<std::pair<long long, int>> key(L.ncell);
    auto K = [](int x, int y, int z) { return ((long long)x << 42) | ((long long)y << 21) | (long long)z; };
    for (int i = 0; i < L.ncell; ++i) key[i] = {K(L.icoord[3 * i], L.icoord[3 * i + 1], L.icoord[3 * i + 2]), i};
    std::sort(key.begin(), key.end());
    auto find = [&](int x, int y, int z) -> int {
      if (x < 0 || y < 0 || z < 0) return -1;
      auto it = std::lower_bound(key.begin(), key.end(), std::make_pair(K(x, y, z), -1));
      if (it != key.end() && it->first == K(x, y, z)) return it->second;
      return -1;
    };
    for (int O = 0; O < L.ncell; ++O) {
      int ox = L.icoord[3 * O], oy = L.icoord[3 * O + 1], oz = L.icoord[3 * O + 2];
      for (int dx = -1; dx <= 1; ++dx)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dz = -1; dz <= 1; ++dz) {
            int S = find(ox + dx, oy + dy, oz + dz);
            if (S < 0 || !(L.leaf[O] || L.leaf[S])) continue;
            for (int u = L.tri_b[O]; u < L.tri_e[O]; ++u)
              for (int w = L.tri_b[S]; w < L.tri_e[S]; ++w) near.push_back(make_int2(perm[u], perm[w]));
          }
      if (l < 2 || !far) continue;
      // interaction list: children of the parent's neighbours, not adjacent to O
      const FmmLevel& Lp = F->lev[l - 1];
      int par = L.parent[O];
      int px = Lp.icoord[3 * par], py = Lp.icoord[3 * par + 1], pz = Lp.icoord[3 * par + 2];
      for (int dx = -1; dx <= 1; ++dx)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dz = -1; dz <= 1; ++dz) {
            int PN = -1;
            // parent-level lookup
            {
              int x = px + dx, y = py + dy, z = pz + dz;
              for (int i = 0; i < Lp.ncell; ++i)
                if (Lp.icoord[3 * i] == x && Lp.icoord[3 * i + 1] == y && Lp.icoord[3 * i + 2] == z) {
                  PN = i;
                  break;
                }
            }
            if (PN < 0) continue;
            for (int o = 0; o < 8; ++o) {
              int S = Lp.child[8 * PN + o];
              if (S < 0) continue;
              int sx = L.icoord[3 * S] - ox, sy = L.icoord[3 * S + 1] - oy, sz = L.icoord[3 * S + 2] - oz;
              if (std::abs(sx) <= 1 && std::abs(sy) <= 1 && std::abs(sz) <= 1) continue;
              il_pairs[l].insert(il_pairs[l].end(), {O, S, sx, sy, sz});
              far_count += (int64_t)(L.tri_e[O] - L.tri_b[O]) * (L.tri_e[S] - L.tri_b[S]);
            }
          }
    }
  }
  if ((int64_t)near.size() + far_count != nt * nt) {
    c->set_error("fast: near and far triangle pairs do not partition all pairs");
    return TDBEM_EINVAL;
  }
  F->n_near_tri_pairs = (int64_t)near.size();
  // ---- near edge pairs (CSR over test edges)
  {
    std::vector<std::vector<int32_t>> rows(ne);
    for (const int2& q : near)
      for (int u = 0; u < 3; ++u)
        for (int w = 0; w < 3; ++w) rows[c->te[3 * q.x + u]].push_back(c->te[3 * q.y + w]);
    std::vector<int64_t> rp(ne + 1, 0);
    for (int64_t i = 0; i < ne; ++i) {
      std::sort(rows[i].begin(), rows[i].end());
      rows[i].erase(std::unique(rows[i].begin(), rows[i].end()), rows[i].end());
      rp[i + 1] = rp[i] + (int64_t)rows[i].size();
    }
    F->nnz = rp[ne];
    std::vector<int32_t> col(F->nnz);
    for (int64_t i = 0; i < ne; ++i) std::copy(rows[i].begin(), rows[i].end(), col.begin() + rp[i]);
    tdbem_status s;
    int2* d_near = nullptr;
    if ((s = c->dalloc(&F->d_row_ptr, ne + 1)) || (s = c->dalloc(&F->d_col, F->nnz)) ||
        (s = c->dalloc(&d_near, near.size())))
      return s;
    TDBEM_CUDA_TRY(c, cudaMemcpy(F->d_row_ptr, rp.data(), (ne + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
    TDBEM_CUDA_TRY(c, cudaMemcpy(F->d_col, col.data(), F->nnz * sizeof(int32_t), cudaMemcpyHostToDevice));
    TDBEM_CUDA_TRY(c, cudaMemcpy(d_near, near.data(), near.size() * sizeof(int2), cudaMemcpyHostToDevice));
    s = tdbem_assemble_csr(c, d_near, (int64_t)near.size(), F->d_row_ptr, F->d_col, F->nnz, &F->d_mlo, &F->d_nlag,
                           &F->d_off, &F->d_val64, &F->nval);
    if (s) return s;
    if ((s = c->dalloc(&F->d_val32, F->nval))) return s;
    k_f64_to_f32<<<(unsigned)((F->nval + 255) / 256), 256, 0, c->stream>>>(F->d_val64, F->d_val32, F->nval);
    TDBEM_CUDA_TRY(c, cudaGetLastError());
    // the blocking copies below run on the legacy stream, which does not wait
    // for the context's (non-blocking) stream
    TDBEM_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    // largest near lag (ring length)
    std::vector<int16_t> ml(F->nnz);
    std::vector<uint8_t> nl(F->nnz);
    TDBEM_CUDA_TRY(c, cudaMemcpy(ml.data(), F->d_mlo, F->nnz * sizeof(int16_t), cudaMemcpyDeviceToHost));
    TDBEM_CUDA_TRY(c, cudaMemcpy(nl.data(), F->d_nlag, F->nnz, cudaMemcpyDeviceToHost));
    int32_t mx = 0;
    for (int64_t q = 0; q < F->nnz; ++q) mx = std::max<int32_t>(mx, ml[q] + nl[q] - 1);
    F->max_near_lag = mx;
    // flattened history entries (lags >= 2) per test edge
    if (mx > 255 || ne >= ((int64_t)1 << 23)) {
      c->set_error("fast: near window or edge count beyond the flattened near-field encoding");
      return TDBEM_EINVAL;
    }
    {
      std::vector<int64_t> off(F->nnz);
      std::vector<float> v32(F->nval);
      TDBEM_CUDA_TRY(c, cudaMemcpy(off.data(), F->d_off, F->nnz * sizeof(int64_t), cudaMemcpyDeviceToHost));
      TDBEM_CUDA_TRY(c, cudaMemcpy(v32.data(), F->d_val32, F->nval * sizeof(float), cudaMemcpyDeviceToHost));
      std::vector<int64_t> hrow(ne + 1, 0);
      std::vector<float> hval;
      std::vector<int32_t> hmeta;
      hval.reserve(F->nval);
      hmeta.reserve(F->nval);
      for (int64_t i = 0; i < ne; ++i) {
        hrow[i] = (int64_t)hval.size();
        for (int64_t q = rp[i]; q < rp[i + 1]; ++q)
          for (int w = 0; w < nl[q]; ++w) {
            const int m = ml[q] + w;
            if (m < 2) continue;
            hval.push_back(v32[off[q] + w]);
            hmeta.push_back((col[q] << 8) | m);
          }
      }
      hrow[ne] = (int64_t)hval.size();
      // one right-hand side with far_overlap keeps only the lag-split copy
      // below (the history evaluation sums its two parts in turn); otherwise
      // the flat entries go to the device as they are
      if (c->R != 1) {
        if ((s = c->dalloc(&F->d_hrow, ne + 1)) || (s = c->dalloc(&F->d_hval, hval.size())) ||
            (s = c->dalloc(&F->d_hmeta, hmeta.size())))
          return s;
        TDBEM_CUDA_TRY(c, cudaMemcpy(F->d_hrow, hrow.data(), (ne + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
        TDBEM_CUDA_TRY(c, cudaMemcpy(F->d_hval, hval.data(), hval.size() * sizeof(float), cudaMemcpyHostToDevice));
        TDBEM_CUDA_TRY(c,
                       cudaMemcpy(F->d_hmeta, hmeta.data(), hmeta.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
      }
      if (c->R == 1) {
        // lag 2 / lags >= 3 (see FmmPlan), each row's entries in the same order
        std::vector<int64_t> r2(ne + 1, 0), r3(ne + 1, 0);
        std::vector<float> v2, v3;
        std::vector<int32_t> m2, m3;
        for (int64_t i = 0; i < ne; ++i) {
          r2[i] = (int64_t)v2.size();
          r3[i] = (int64_t)v3.size();
          for (int64_t e = hrow[i]; e < hrow[i + 1]; ++e) {
            const bool two = (hmeta[e] & 0xff) == 2;
            (two ? v2 : v3).push_back(hval[e]);
            (two ? m2 : m3).push_back(hmeta[e]);
          }
        }
        r2[ne] = (int64_t)v2.size();
        r3[ne] = (int64_t)v3.size();
        if ((s = c->dalloc(&F->d_hrow2, ne + 1)) || (s = c->dalloc(&F->d_hval2, v2.size())) ||
            (s = c->dalloc(&F->d_hmeta2, m2.size())) || (s = c->dalloc(&F->d_hrow3, ne + 1)) ||
            (s = c->dalloc(&F->d_hval3, v3.size())) || (s = c->dalloc(&F->d_hmeta3, m3.size())) ||
            (s = c->dalloc(&F->d_Rp, 2 * ne)))
          return s;
        TDBEM_CUDA_TRY(c, cudaMemcpy(F->d_hrow2, r2.data(), (ne + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
        TDBEM_CUDA_TRY(c, cudaMemcpy(F->d_hrow3, r3.data(), (ne + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
        if (!v2.empty()) {
          TDBEM_CUDA_TRY(c, cudaMemcpy(F->d_hval2, v2.data(), v2.size() * sizeof(float), cudaMemcpyHostToDevice));
          TDBEM_CUDA_TRY(c, cudaMemcpy(F->d_hmeta2, m2.data(), m2.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
        }
        if (!v3.empty()) {
          TDBEM_CUDA_TRY(c, cudaMemcpy(F->d_hval3, v3.data(), v3.size() * sizeof(float), cudaMemcpyHostToDevice));
          TDBEM_CUDA_TRY(c, cudaMemcpy(F->d_hmeta3, m3.data(), m3.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
        }
        // the lags >= 3 tiled by column blocks (k_near_tile) for the pipelined
        // march, when the entry indices fit 32 bits.  Measured on the 7680-RWG
        // sphere: the pipelined march gains 9% (the block's history comes from
        // shared memory, not from L2 gathers that compete with the
        // overlapped M2L), while alone the flat kernel is the faster one
        // A task stages L x kNB history values before its entries: the tiling
        // pays only where a block holds many entries per staged value (long
        // lag windows over few columns, as with a small step, do not)
        // Measured in the pipelined march: on the 7680-RWG sphere (4.0 k
        // entries per row) the tiled form gains 9%; on the paper's case 2
        // (4320 RWG, dt = h/7, 32 k entries per row) the flat kernel's long
        // rows stream well and the tiled form loses 30%.  Rows of at most 16 k
        // entries are tiled.
        const int64_t nlag = F->max_near_lag + 1;  // lags staged per block
        const int64_t nblk_est = (ne + kNB - 1) / kNB;
        const bool tile_pays = (int64_t)v3.size() >= 8 * nblk_est * kNB * nlag && (int64_t)v3.size() <= 16384 * ne;
        if (c->p.far_overlap && tile_pays && !v3.empty() && (int64_t)v3.size() < ((int64_t)1 << 31)) {
          // Morton order of the edges' midpoints (mean of the two triangles' centroids)
          std::vector<double> mid(3 * ne);
          double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
          for (int64_t e = 0; e < ne; ++e)
            for (int d = 0; d < 3; ++d) {
              double x = 0.0;
              for (int side = 0; side < 2; ++side) {
                const int32_t t = c->et[2 * e + side];
                for (int q = 0; q < 3; ++q) x += c->V[3 * c->T[3 * t + q] + d];
              }
              mid[3 * e + d] = x / 6.0;
              lo[d] = std::min(lo[d], x / 6.0);
              hi[d] = std::max(hi[d], x / 6.0);
            }
          std::vector<uint64_t> key(ne);
          for (int64_t e = 0; e < ne; ++e) {
            uint64_t code = 0;
            for (int d = 0; d < 3; ++d) {
              const double u = (mid[3 * e + d] - lo[d]) / std::max(hi[d] - lo[d], 1e-300);
              const uint64_t qd = (uint64_t)std::min(1023.0, std::max(0.0, std::floor(u * 1024.0)));
              for (int bit = 0; bit < 10; ++bit) code |= ((qd >> bit) & 1ull) << (3 * bit + d);
            }
            key[e] = (code << 24) | (uint64_t)e;  // ties by edge index
          }
          std::sort(key.begin(), key.end());
          std::vector<int32_t> corder(ne), cpos(ne);
          for (int64_t k = 0; k < ne; ++k) {
            corder[k] = (int32_t)(key[k] & 0xffffff);
            cpos[corder[k]] = (int32_t)k;
          }
          // entries grouped by block (counting sort), rows in order within a block
          const int64_t nblk = (ne + kNB - 1) / kNB, nent = (int64_t)v3.size();
          std::vector<int64_t> bstart(nblk + 1, 0);
          for (int64_t e = 0; e < nent; ++e) ++bstart[cpos[m3[e] >> 8] / kNB + 1];
          for (int64_t b = 0; b < nblk; ++b) bstart[b + 1] += bstart[b];
          std::vector<int64_t> fill(bstart.begin(), bstart.end() - 1);
          std::vector<float> cval(nent);
          std::vector<uint16_t> cmeta(nent);
          std::vector<int32_t> erow(nent);
          for (int64_t i = 0; i < ne; ++i)
            for (int64_t e = r3[i]; e < r3[i + 1]; ++e) {
              const int32_t pos = cpos[m3[e] >> 8];
              const int64_t k = fill[pos / kNB]++;
              cval[k] = v3[e];
              cmeta[k] = (uint16_t)(((pos % kNB) << 8) | (m3[e] & 0xff));
              erow[k] = (int32_t)i;
            }
          // segments, tasks and each row's segment list
          std::vector<int64_t> seg_ptr;
          std::vector<int32_t> seg_row;
          std::vector<int4> tasks;
          // at least four entries per staged value in a task
          const int64_t task_entries = std::max<int64_t>(kNTaskEntries, 4 * kNB * nlag);
          for (int64_t b = 0; b < nblk; ++b) {
            int64_t t0 = (int64_t)seg_row.size(), tent = 0;
            for (int64_t k = bstart[b]; k < bstart[b + 1];) {
              int64_t k1 = k;
              while (k1 < bstart[b + 1] && erow[k1] == erow[k]) ++k1;
              if (tent > 0 && tent + (k1 - k) > task_entries) {
                tasks.push_back(make_int4((int)b, (int)t0, (int)seg_row.size(), 0));
                t0 = (int64_t)seg_row.size();
                tent = 0;
              }
              seg_ptr.push_back(k);
              seg_row.push_back(erow[k]);
              tent += k1 - k;
              k = k1;
            }
            if ((int64_t)seg_row.size() > t0) tasks.push_back(make_int4((int)b, (int)t0, (int)seg_row.size(), 0));
          }
          seg_ptr.push_back(nent);
          const int64_t nseg = (int64_t)seg_row.size();
          std::vector<int64_t> rptr(ne + 1, 0);
          for (int64_t g = 0; g < nseg; ++g) ++rptr[seg_row[g] + 1];
          for (int64_t i = 0; i < ne; ++i) rptr[i + 1] += rptr[i];
          std::vector<int32_t> rseg(std::max<int64_t>(1, nseg));
          {
            std::vector<int64_t> rf(rptr.begin(), rptr.end() - 1);
            for (int64_t g = 0; g < nseg; ++g) rseg[rf[seg_row[g]]++] = (int32_t)g;  // ascending per row
          }
          if (nseg >= INT32_MAX) {
            c->set_error("fast: too many near-field segments");
            return TDBEM_EINVAL;
          }
          F->nseg = nseg;
          F->ntask = (int32_t)tasks.size();
          if ((s = c->dalloc(&F->d_corder, ne)) || (s = c->dalloc(&F->d_seg_ptr, nseg + 1)) ||
              (s = c->dalloc(&F->d_cval, nent)) || (s = c->dalloc(&F->d_cmeta, nent)) ||
              (s = c->dalloc(&F->d_ntasks, std::max<int64_t>(1, F->ntask))) || (s = c->dalloc(&F->d_rseg_ptr, ne + 1)) ||
              (s = c->dalloc(&F->d_rseg, std::max<int64_t>(1, nseg))) ||
              (s = c->dalloc(&F->d_spart, std::max<int64_t>(1, nseg))))
            return s;
          TDBEM_CUDA_TRY(c, cudaMemcpy(F->d_corder, corder.data(), ne * sizeof(int32_t), cudaMemcpyHostToDevice));
          TDBEM_CUDA_TRY(c, cudaMemcpy(F->d_seg_ptr, seg_ptr.data(), (nseg + 1) * sizeof(int64_t),
                                       cudaMemcpyHostToDevice));
          TDBEM_CUDA_TRY(c, cudaMemcpy(F->d_cval, cval.data(), nent * sizeof(float), cudaMemcpyHostToDevice));
          TDBEM_CUDA_TRY(c, cudaMemcpy(F->d_cmeta, cmeta.data(), nent * sizeof(uint16_t), cudaMemcpyHostToDevice));
          if (F->ntask)
            TDBEM_CUDA_TRY(c, cudaMemcpy(F->d_ntasks, tasks.data(), F->ntask * sizeof(int4), cudaMemcpyHostToDevice));
          TDBEM_CUDA_TRY(c, cudaMemcpy(F->d_rseg_ptr, rptr.data(), (ne + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
          if (nseg)
            TDBEM_CUDA_TRY(c, cudaMemcpy(F->d_rseg, rseg.data(), nseg * sizeof(int32_t), cudaMemcpyHostToDevice));
        }
        if (c->p.far_overlap) {
          // between the deferred M2L's lowest priority and the steps' highest:
          // the next solve's cluster, which needs whole SMs, is dispatched ahead
          // of this stream's remaining CTAs
          int prio_lo = 0, prio_hi = 0;
          TDBEM_CUDA_TRY(c, cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
          TDBEM_CUDA_TRY(c,
                         cudaStreamCreateWithPriority(&F->nstream, cudaStreamNonBlocking, (prio_lo + prio_hi) / 2));
          TDBEM_CUDA_TRY(c, cudaEventCreateWithFlags(&F->ev_solved, cudaEventDisableTiming));
          for (int b = 0; b < 2; ++b)
            TDBEM_CUDA_TRY(c, cudaEventCreateWithFlags(&F->ev_near[b], cudaEventDisableTiming));
        }
      }
    }
  }
  c->max_lag = std::max(F->max_near_lag, far ? F->lev[2].M + 4 : 0);
  tdbem_status s;
  if ((s = c->dalloc(&F->d_perm, nt))) return s;
  TDBEM_CUDA_TRY(c, cudaMemcpy(F->d_perm, perm.data(), nt * sizeof(int32_t), cudaMemcpyHostToDevice));
  if (!far) return TDBEM_OK;
  // ---- per-level device data, time tables, M2L operators and work lists
  const double dt = c->dt, cc = c->phys.c;
  TDBEM_CUDA_TRY(c, cudaFuncSetAttribute(k_l2p, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  TDBEM_CUDA_TRY(c, cudaFuncSetAttribute(k_p2m, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  TDBEM_CUDA_TRY(c, cudaFuncSetAttribute(k_m2m_fact, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
  TDBEM_CUDA_TRY(c, cudaFuncSetAttribute(k_l2l_fact, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));

  std::vector<double> tbox(4 * nt);
  for (int l = 0; l <= lmax; ++l) {
    FmmLevel& L = F->lev[l];
    std::vector<int> lc, nlc;
    for (int i = 0; i < L.ncell; ++i) (L.leaf[i] ? lc : nlc).push_back(i);
    L.nleaf = (int)lc.size();
    L.nnonleaf = (int)nlc.size();
    for (int i : lc)
      for (int u = L.tri_b[i]; u < L.tri_e[i]; ++u) {
        int t = perm[u];
        tbox[4 * t] = L.cen[3 * i];
        tbox[4 * t + 1] = L.cen[3 * i + 1];
        tbox[4 * t + 2] = L.cen[3 * i + 2];
        tbox[4 * t + 3] = L.H;
      }
    if (l < 2) continue;
    if ((s = c->dalloc(&L.d_child, 8 * (int64_t)L.ncell)) || (s = c->dalloc(&L.d_tri_b, L.ncell)) ||
        (s = c->dalloc(&L.d_tri_e, L.ncell)) || (s = c->dalloc(&L.d_leaf_cells, L.nleaf)) ||
        (s = c->dalloc(&L.d_nonleaf_cells, L.nnonleaf)))
      return s;
    TDBEM_CUDA_TRY(c, cudaMemcpy(L.d_child, L.child.data(), 8 * L.ncell * sizeof(int32_t), cudaMemcpyHostToDevice));
    TDBEM_CUDA_TRY(c, cudaMemcpy(L.d_tri_b, L.tri_b.data(), L.ncell * sizeof(int32_t), cudaMemcpyHostToDevice));
    TDBEM_CUDA_TRY(c, cudaMemcpy(L.d_tri_e, L.tri_e.data(), L.ncell * sizeof(int32_t), cudaMemcpyHostToDevice));
    if (L.nleaf)
      TDBEM_CUDA_TRY(c, cudaMemcpy(L.d_leaf_cells, lc.data(), L.nleaf * sizeof(int32_t), cudaMemcpyHostToDevice));
    if (L.nnonleaf)
      TDBEM_CUDA_TRY(
          c, cudaMemcpy(L.d_nonleaf_cells, nlc.data(), L.nnonleaf * sizeof(int32_t), cudaMemcpyHostToDevice));
    // time tables: source factors, and per target step the factors of the
    // four kinds l, l'/h_t, chi l'/h_t + zeta l, l''/h_t^2
    std::vector<float> ts(L.M * pt), tt(L.M * 4 * pt);
    const double ht = 0.5 * L.M * dt;
    for (int i = 0; i < L.M; ++i) {
      double xi = (i - 0.5 * (L.M - 1)) / (0.5 * L.M);
      double lv[8], dv[8], d2v[8];
      time_basis(pt, c->p.t_interp, xi, lv, dv, d2v);
      for (int n = 0; n < pt; ++n) {
        ts[i * pt + n] = (float)lv[n];
        tt[(i * 4 + 0) * pt + n] = (float)lv[n];
        tt[(i * 4 + 1) * pt + n] = (float)(dv[n] / ht);
        tt[(i * 4 + 2) * pt + n] = (float)(c->p.chi * dv[n] / ht + c->p.zeta * lv[n]);
        tt[(i * 4 + 3) * pt + n] = (float)(d2v[n] / (ht * ht));
      }
    }
    if ((s = c->dalloc(&L.d_tsrc, ts.size())) || (s = c->dalloc(&L.d_ttgt, tt.size()))) return s;
    TDBEM_CUDA_TRY(c, cudaMemcpy(L.d_tsrc, ts.data(), ts.size() * sizeof(float), cudaMemcpyHostToDevice));
    TDBEM_CUDA_TRY(c, cudaMemcpy(L.d_ttgt, tt.data(), tt.size() * sizeof(float), cudaMemcpyHostToDevice));
    // interaction pairs grouped by canonical offset
    struct PairRec {
      int O, S, canon, sym;
    };
    std::vector<PairRec> pr;
    std::vector<std::array<int, 3>> canons;
    const std::vector<int>& ip = il_pairs[l];
    for (size_t q = 0; q < ip.size(); q += 5) {
      // x - y = (c_O - c_S) + H (w_a - w_b): the symmetry is taken on O - S
      int o[3] = {-ip[q + 2], -ip[q + 3], -ip[q + 4]};
      int ab[3] = {std::abs(o[0]), std::abs(o[1]), std::abs(o[2])};
      int ax[3] = {0, 1, 2};
      std::sort(ax, ax + 3, [&](int u, int w) { return ab[u] != ab[w] ? ab[u] < ab[w] : u < w; });
      std::array<int, 3> cv = {ab[ax[0]], ab[ax[1]], ab[ax[2]]};
      int ci = -1;
      for (size_t z = 0; z < canons.size(); ++z)
        if (canons[z] == cv) ci = (int)z;
      if (ci < 0) {
        canons.push_back(cv);
        ci = (int)canons.size() - 1;
      }
      // symmetry id: permutation (index of ax among the 6) and signs
      static const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
      int pi = 0;
      for (int z = 0; z < 6; ++z)
        if (perms[z][0] == ax[0] && perms[z][1] == ax[1] && perms[z][2] == ax[2]) pi = z;
      int sg = (o[0] < 0 ? 4 : 0) | (o[1] < 0 ? 2 : 0) | (o[2] < 0 ? 1 : 0);
      pr.push_back({ip[q], ip[q + 1], ci, pi * 8 + sg});
    }
    std::stable_sort(pr.begin(), pr.end(), [](const PairRec& x, const PairRec& y) { return x.canon < y.canon; });
    L.npairs = (int)pr.size();
    std::vector<int32_t> hO(L.npairs), hS(L.npairs);
    std::vector<int16_t> hsym(L.npairs);
    for (int q = 0; q < L.npairs; ++q) {
      hO[q] = pr[q].O;
      hS[q] = pr[q].S;
      hsym[q] = (int16_t)pr[q].sym;
    }
    if ((s = c->dalloc(&L.d_pO, L.npairs)) || (s = c->dalloc(&L.d_pS, L.npairs)) ||
        (s = c->dalloc(&L.d_psym, L.npairs)))
      return s;
    if (L.npairs) {
      TDBEM_CUDA_TRY(c, cudaMemcpy(L.d_pO, hO.data(), L.npairs * sizeof(int32_t), cudaMemcpyHostToDevice));
      TDBEM_CUDA_TRY(c, cudaMemcpy(L.d_pS, hS.data(), L.npairs * sizeof(int32_t), cudaMemcpyHostToDevice));
      TDBEM_CUDA_TRY(c, cudaMemcpy(L.d_psym, hsym.data(), L.npairs * sizeof(int16_t), cudaMemcpyHostToDevice));
    }
    // (source cell, symmetry) combinations: the tensor-core M2L permutes each
    // source moment once per symmetry in use instead of once per pair and lag
    {
      std::map<std::pair<int, int>, int> cid;
      for (int q = 0; q < L.npairs; ++q) cid.emplace(std::make_pair(pr[q].S, pr[q].sym), 0);
      std::vector<int32_t> cS, hC(L.npairs);
      std::vector<int16_t> csym;
      for (auto& e : cid) {
        e.second = (int)cS.size();
        cS.push_back(e.first.first);
        csym.push_back((int16_t)e.first.second);
      }
      for (int q = 0; q < L.npairs; ++q) hC[q] = cid[std::make_pair(pr[q].S, pr[q].sym)];
      L.ncombo = (int)cS.size();
      if ((s = c->dalloc(&L.d_pC, std::max(1, L.npairs))) || (s = c->dalloc(&L.d_cS, std::max(1, L.ncombo))) ||
          (s = c->dalloc(&L.d_csym, std::max(1, L.ncombo))))
        return s;
      if (L.npairs) {
        TDBEM_CUDA_TRY(c, cudaMemcpy(L.d_pC, hC.data(), L.npairs * sizeof(int32_t), cudaMemcpyHostToDevice));
        TDBEM_CUDA_TRY(c, cudaMemcpy(L.d_cS, cS.data(), L.ncombo * sizeof(int32_t), cudaMemcpyHostToDevice));
        TDBEM_CUDA_TRY(c, cudaMemcpy(L.d_csym, csym.data(), L.ncombo * sizeof(int16_t), cudaMemcpyHostToDevice));
      }
    }
    // lag ranges per canonical offset; operators; GEMM and tile lists
    std::vector<int4> opdesc, gemm, tiles, tiles_tc, tiles_tc2;
    int qmax = 1;
    for (size_t ci = 0; ci < canons.size(); ++ci) {
      int base = -1, cnt = 0;
      for (int q = 0; q < L.npairs; ++q)
        if (pr[q].canon == (int)ci) {
          if (base < 0) base = q;
          ++cnt;
        }
      const std::array<int, 3>& cv = canons[ci];
      double rmin2 = 0, rmax2 = 0;
      for (int k = 0; k < 3; ++k) {
        double g = std::max(0.0, cv[k] * L.ds - 2 * L.H);
        rmin2 += g * g;
        double h = cv[k] * L.ds + 2 * L.H;
        rmax2 += h * h;
      }
      double rmin = std::sqrt(rmin2), rmax = std::sqrt(rmax2);
      int qlo = std::max(1, (int)std::floor(rmin / (L.M * a)));
      int qhi = (int)std::ceil((1.0 + rmax / a) / L.M);
      qmax = std::max(qmax, qhi);
      for (int q = qlo; q <= qhi; ++q) {
        int op = (int)opdesc.size();
        opdesc.push_back(make_int4(cv[0], cv[1], cv[2], q));
        for (int kind = 0; kind < 2; ++kind) {
          int g = (int)gemm.size();
          gemm.push_back(make_int4(op, base, cnt, kind | (q << 8) | (qhi << 16)));
          int ncol = cnt * (kind == 0 ? 3 : 4) * c->R;  // columns (pair, right-hand side, component)
          for (int rt = 0; rt < (P + 63) / 64; ++rt)
            for (int ct = 0; ct < (ncol + 63) / 64; ++ct) tiles.push_back(make_int4(g, rt, ct, 0));
          for (int rt = 0; rt < (P + 127) / 128; ++rt)  // single 128-row tiles
            for (int ct = 0; ct < (ncol + 127) / 128; ++ct) tiles_tc.push_back(make_int4(g, rt, ct, 0));
          for (int rt = 0; rt < (P + 255) / 256; ++rt)  // pairs of 128-row tiles
            for (int ct = 0; ct < (ncol + 127) / 128; ++ct) tiles_tc2.push_back(make_int4(g, rt, ct, 0));
          L.flops_event += 2.0 * P * P * ncol;
        }
      }
    }
    // lag-1 tiles first in every list (see FmmLevel): only they feed the
    // interval the event's own L2L and L2P read
    auto lag1_first = [&](std::vector<int4>& tl) {
      auto it = std::stable_partition(tl.begin(), tl.end(),
                                      [&](const int4& t) { return ((gemm[t.x].w >> 8) & 0xff) == 1; });
      return (int)(it - tl.begin());
    };
    L.ntiles_urgent = lag1_first(tiles);
    L.ntiles_tc_urgent[0] = lag1_first(tiles_tc);
    L.ntiles_tc_urgent[1] = lag1_first(tiles_tc2);
    // resident-operator units: runs of up to 8 column tiles per (GEMM, row
    // tile), the run length chosen so that each list still has about four
    // units per SM
    L.res_ok = c->p.m2l_prec == TDBEM_P_F16X3 && P <= 256;
    if (L.res_ok && !gemm.empty()) {
      int nsm = 0;
      TDBEM_CUDA_TRY(c, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device));
      const int nrt = (P + 127) / 128;
      std::vector<int4> units;
      for (int urgent = 1; urgent >= 0; --urgent) {
        int64_t tot = 0;
        for (size_t g = 0; g < gemm.size(); ++g)
          if ((((gemm[g].w >> 8) & 0xff) == 1) == (urgent == 1)) {
            const int nk = (gemm[g].w & 0xff) == 0 ? 3 : 4;
            tot += (int64_t)nrt * ((gemm[g].z * nk * c->R + 127) / 128);
          }
        const int run = (int)std::max<int64_t>(1, std::min<int64_t>(8, (tot + 4 * nsm - 1) / (4 * nsm)));
        for (size_t g = 0; g < gemm.size(); ++g) {
          if ((((gemm[g].w >> 8) & 0xff) == 1) != (urgent == 1)) continue;
          const int nk = (gemm[g].w & 0xff) == 0 ? 3 : 4;
          const int nct = (gemm[g].z * nk * c->R + 127) / 128;
          for (int rt = 0; rt < nrt; ++rt)
            for (int c0 = 0; c0 < nct; c0 += run) units.push_back(make_int4((int)g, rt, c0, std::min(run, nct - c0)));
        }
        if (urgent) L.nunits_urgent = (int)units.size();
      }
      L.nunits = (int)units.size();
      if ((s = c->dalloc(&L.d_units, std::max(1, L.nunits)))) return s;
      if (L.nunits)
        TDBEM_CUDA_TRY(c, cudaMemcpy(L.d_units, units.data(), L.nunits * sizeof(int4), cudaMemcpyHostToDevice));
    }
    if (qmax >= 255) {
      c->set_error("fast: too many time intervals per interaction");
      return TDBEM_EINVAL;
    }
    L.Q = qmax + 1;
    L.nop = (int)opdesc.size();
    L.ngemm = (int)gemm.size();
    L.ntiles = (int)tiles.size();
    for (int v = 0; v < 2; ++v) {
      const std::vector<int4>& tl = v == 0 ? tiles_tc : tiles_tc2;
      L.ntiles_tc[v] = (int)tl.size();
      if ((s = c->dalloc(&L.d_tiles_tc[v], std::max(1, L.ntiles_tc[v])))) return s;
      if (L.ntiles_tc[v])
        TDBEM_CUDA_TRY(c, cudaMemcpy(L.d_tiles_tc[v], tl.data(), L.ntiles_tc[v] * sizeof(int4), cudaMemcpyHostToDevice));
    }
    int4* d_opdesc = nullptr;
    if ((s = c->dalloc(&d_opdesc, std::max(1, L.nop))) || (s = c->dalloc(&L.ops, (int64_t)L.nop * 2 * P * P)) ||
        (s = c->dalloc(&L.d_gemm, std::max(1, L.ngemm))) || (s = c->dalloc(&L.d_tiles, std::max(1, L.ntiles))))
      return s;
    if (L.nop) {
      TDBEM_CUDA_TRY(c, cudaMemcpy(d_opdesc, opdesc.data(), L.nop * sizeof(int4), cudaMemcpyHostToDevice));
      TDBEM_CUDA_TRY(c, cudaMemcpy(L.d_gemm, gemm.data(), L.ngemm * sizeof(int4), cudaMemcpyHostToDevice));
      TDBEM_CUDA_TRY(c, cudaMemcpy(L.d_tiles, tiles.data(), L.ntiles * sizeof(int4), cudaMemcpyHostToDevice));
      int64_t tot = (int64_t)L.nop * P * P;
      k_m2l_ops<<<(unsigned)((tot + 255) / 256), 256, 0, c->stream>>>(p, pt, L.ds, L.H, 0.5 * L.M * dt, L.M, dt, cc, a,
                                                                      d_opdesc, L.nop, c->p.far_kernel,
                                                                      a_kernel_derivs(c->p.a_deriv), c->p.s_interp,
                                                                      c->p.t_interp, L.ops);
      TDBEM_CUDA_TRY(c, cudaGetLastError());
      if (c->p.m2l_prec != TDBEM_P_FP32 && (s = tdbem_m2l_tc_images(c, L.ops, L.nop, P, c->p.m2l_prec, &L.ops_img, &L.d_opinv)))
        return s;
    }
    // moment and local-coefficient storage (march state and history_eval state)
    const int64_t RP = (int64_t)c->R * kNC * P;  // one cluster's coefficients of all right-hand sides
    if ((s = c->dalloc(&L.mom, (int64_t)L.ncell * 4 * RP)) || (s = c->dalloc(&L.loc, (int64_t)L.ncell * L.Q * RP)))
      return s;
    TDBEM_CUDA_TRY(c, cudaMemset(L.mom, 0, (int64_t)L.ncell * 4 * RP * sizeof(float)));
    TDBEM_CUDA_TRY(c, cudaMemset(L.loc, 0, (int64_t)L.ncell * L.Q * RP * sizeof(float)));
    float *me = nullptr, *le = nullptr;
    if ((s = c->dalloc(&me, (int64_t)L.ncell * 4 * RP)) || (s = c->dalloc(&le, (int64_t)L.ncell * L.Q * RP)))
      return s;
    F->mom_eval.push_back(me);
    F->loc_eval.push_back(le);
  }
  // interpolation matrices between levels (space: child node -> parent
  // polynomial, per octant sign; time: the same at every level)
  {
    std::vector<float> Sx((lmax + 1) * 2 * p * p, 0.f), St(2 * pt * pt);
    for (int l = 0; l < lmax; ++l) {
      double Hp = F->lev[l].H, Hc = F->lev[l + 1].H, dsp = F->lev[l].ds;
      for (int sgn = 0; sgn < 2; ++sgn)
        for (int cb = 0; cb < p; ++cb) {
          double xi = ((sgn ? 0.25 : -0.25) * dsp + Hc * interp_node(cb, p, c->p.s_interp)) / Hp;
          double lv[8];
          space_basis(p, c->p.s_interp, xi, lv, nullptr);
          for (int b = 0; b < p; ++b) Sx[((l * 2 + sgn) * p + b) * p + cb] = (float)lv[b];
        }
    }
    for (int h = 0; h < 2; ++h)
      for (int cn = 0; cn < pt; ++cn) {
        double xi = 0.5 * interp_node(cn, pt, c->p.t_interp) + (h ? 0.5 : -0.5);
        double lv[8];
        time_basis(pt, c->p.t_interp, xi, lv, nullptr, nullptr);
        for (int n = 0; n < pt; ++n) St[(h * pt + n) * pt + cn] = (float)lv[n];
      }
    if ((s = c->dalloc(&F->d_Sx, Sx.size())) || (s = c->dalloc(&F->d_St, St.size()))) return s;
    TDBEM_CUDA_TRY(c, cudaMemcpy(F->d_Sx, Sx.data(), Sx.size() * sizeof(float), cudaMemcpyHostToDevice));
    TDBEM_CUDA_TRY(c, cudaMemcpy(F->d_St, St.data(), St.size() * sizeof(float), cudaMemcpyHostToDevice));
  }
  // symmetry maps: for symmetry (perm pi, signs sg), canonical node index a'
  // -> original node index a (a'_k = a~_{i_k}, a~_i = a_i or p-1-a_i)
  {
    static const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    std::vector<int16_t> sm(48 * PS);
    for (int pi = 0; pi < 6; ++pi)
      for (int sg = 0; sg < 8; ++sg)
        for (int ap = 0; ap < PS; ++ap) {
          int acan[3] = {ap / (p * p), (ap / p) % p, ap % p};
          int aorig[3];
          for (int k = 0; k < 3; ++k) {
            int i = perms[pi][k];
            int v = acan[k];
            bool flip = (sg >> (2 - i)) & 1;
            aorig[i] = flip ? p - 1 - v : v;
          }
          sm[(pi * 8 + sg) * PS + ap] = (int16_t)((aorig[0] * p + aorig[1]) * p + aorig[2]);
        }
    if ((s = c->dalloc(&F->d_smap, sm.size()))) return s;
    TDBEM_CUDA_TRY(c, cudaMemcpy(F->d_smap, sm.data(), sm.size() * sizeof(int16_t), cudaMemcpyHostToDevice));
  }
  // P2M / L2P tables
  {
    int nq1 = std::max(6, (3 * p + 1) / 2 + 1);
    std::vector<double> qx, qw;
    gauss_legendre01(nq1, qx, qw);
    double *d_box = nullptr, *d_qx = nullptr, *d_qw = nullptr;
    if ((s = c->dalloc(&d_box, 4 * nt)) || (s = c->dalloc(&d_qx, nq1)) || (s = c->dalloc(&d_qw, nq1)) ||
        (s = c->dalloc(&F->d_W, nt * 3 * kNC * PS)) || (s = c->dalloc(&F->d_T, nt * 3 * kNC * PS)))
      return s;
    TDBEM_CUDA_TRY(c, cudaMemcpy(d_box, tbox.data(), 4 * nt * sizeof(double), cudaMemcpyHostToDevice));
    TDBEM_CUDA_TRY(c, cudaMemcpy(d_qx, qx.data(), nq1 * sizeof(double), cudaMemcpyHostToDevice));
    TDBEM_CUDA_TRY(c, cudaMemcpy(d_qw, qw.data(), nq1 * sizeof(double), cudaMemcpyHostToDevice));
    k_far_tables<<<(unsigned)nt, 256, 0, c->stream>>>(c->tg, c->phys, p, c->p.s_interp, (int)nt, d_box, d_qx, d_qw, nq1, F->d_W,
                                                       F->d_T);
    TDBEM_CUDA_TRY(c, cudaGetLastError());
  }
  // far right-hand-side rings
  int Mmax = F->lev[2].M;
  int Lr = 8;
  while (Lr < 2 * Mmax) Lr <<= 1;
  F->Lr = Lr;
  const int64_t nrf = (int64_t)Lr * ne * c->R;  // [Lr][ne][R]
  if ((s = c->dalloc(&F->d_Rfar, nrf)) || (s = c->dalloc(&F->d_Rfar_eval, nrf)) || (s = c->dalloc(&F->d_err, 1)))
    return s;
  TDBEM_CUDA_TRY(c, cudaMemset(F->d_err, 0, sizeof(int32_t)));
  TDBEM_CUDA_TRY(c, cudaMemset(F->d_Rfar, 0, nrf * sizeof(double)));
  if (c->p.m2l_prec != TDBEM_P_FP32) {
    // packed moments of each level's event (one buffer per level: a deferred
    // M2L of one level may still read its buffer while another level packs),
    // zeroed so that the autotuner's trial launches below add nothing
    for (int l = 2; l <= F->lmax; ++l) {
      const int64_t npk = std::max<int64_t>(1, (int64_t)F->lev[l].ncombo * 2 * c->R * kNC * P);
      if ((s = c->dalloc(&F->lev[l].d_pack, npk))) return s;
      TDBEM_CUDA_TRY(c, cudaMemset(F->lev[l].d_pack, 0, npk * sizeof(float)));
      if (c->p.m2l_prec == TDBEM_P_F16X3) {
        const int64_t nrow = std::max<int64_t>(1, (int64_t)F->lev[l].ncombo * 2 * c->R * kNC);
        if ((s = c->dalloc(&F->lev[l].d_pkinv, nrow))) return s;
        TDBEM_CUDA_TRY(c, cudaMemset(F->lev[l].d_pkinv, 0, nrow * sizeof(float)));
        if (F->lev[l].res_ok) {
          const int64_t n16 = nrow * 2 * ((P + 63) / 64 * 64);
          if ((s = c->dalloc(&F->lev[l].d_pk16, n16))) return s;
          TDBEM_CUDA_TRY(c, cudaMemset(F->lev[l].d_pk16, 0, n16 * sizeof(__half)));
        }
      }
    }
  }
  if (c->p.far_overlap) {
    int prio_lo = 0, prio_hi = 0;
    TDBEM_CUDA_TRY(c, cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
    TDBEM_CUDA_TRY(c, cudaStreamCreateWithPriority(&F->side, cudaStreamNonBlocking, prio_lo));

    TDBEM_CUDA_TRY(c, cudaEventCreateWithFlags(&F->ev_fork, cudaEventDisableTiming));
    for (int l = 2; l <= F->lmax; ++l)
      TDBEM_CUDA_TRY(c, cudaEventCreateWithFlags(&F->lev[l].ev_defer, cudaEventDisableTiming));
  }
  TDBEM_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  // M2L autotuner: time one gating event of each level with every kernel
  // shape that applies -- the tiled kernel with one or two 128-row operator
  // tiles per CTA, and for the FP16 form with P <= 256 the resident-operator
  // kernel -- on this context's own operators, pairs and right-hand sides,
  // and keep the fastest.  The packed moments are still zero, so the trial
  // launches add nothing to the local coefficients.
  if (c->p.m2l_prec != TDBEM_P_FP32 && c->p.m2l_tile_rows != 0) {
    for (int l = 2; l <= F->lmax; ++l) {
      F->lev[l].tc_mt = c->p.m2l_tile_rows == 256 ? 2 : 1;
      F->lev[l].res = c->p.m2l_tile_rows == 1 && F->lev[l].res_ok;
    }
  } else if (c->p.m2l_prec != TDBEM_P_FP32) {
    cudaEvent_t e0, e1;
    TDBEM_CUDA_TRY(c, cudaEventCreate(&e0));
    TDBEM_CUDA_TRY(c, cudaEventCreate(&e1));
    for (int l = 2; l <= F->lmax; ++l) {
      FmmLevel& L = F->lev[l];
      if (!L.ntiles_tc[0]) continue;
      for (int v = 0; v < (L.res_ok ? 3 : 2); ++v) {
        const int reps = 3;
        for (int it = -1; it < reps; ++it) {  // one untimed launch first
          if (it == 0) TDBEM_CUDA_TRY(c, cudaEventRecord(e0, c->stream));
          if (v < 2)
            s = tdbem_m2l_tc(c, v + 1, L.d_gemm, L.d_tiles_tc[v], L.ntiles_tc[v], L.ops_img, P, pt, PS, L.d_pO,
                             L.d_pC, L.d_psym, F->d_smap, L.d_pack, 0, L.loc, L.Q, c->R, c->p.m2l_prec, L.d_opinv,
                             L.d_pkinv, F->d_err);
          else
            s = tdbem_m2l_res(c, L.d_gemm, L.d_units, 0, L.nunits, L.ops_img, P, pt, PS, L.d_pO, L.d_pC, L.d_psym,
                              F->d_smap, L.d_pk16, 0, L.loc, L.Q, c->R, L.d_opinv, L.d_pkinv, F->d_err, 0);
          if (s) return s;
        }
        TDBEM_CUDA_TRY(c, cudaEventRecord(e1, c->stream));
        TDBEM_CUDA_TRY(c, cudaEventSynchronize(e1));
        float ms = 0.f;
        TDBEM_CUDA_TRY(c, cudaEventElapsedTime(&ms, e0, e1));
        (v < 2 ? L.tc_ms[v] : L.res_ms) = ms / reps;
      }
      L.tc_mt = L.tc_ms[1] < L.tc_ms[0] ? 2 : 1;
      L.res = L.res_ok && L.res_ms < std::min(L.tc_ms[0], L.tc_ms[1]);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if ((s = tdbem_fast_check(c))) return s;
  }
  return TDBEM_OK;
}

// ---------------------------------------------------------------------------
// Step pieces

static tdbem_status far_events(tdbem_ctx* c, int32_t alpha, const double* ring, bool eval) {
  FmmPlan* F = c->fmm;
  if (!F || F->lmax < 2) return TDBEM_OK;
  const int p = F->p, pt = F->pt, PS = F->PS, P = F->P, lmax = F->lmax, R = c->R;
  auto MOM = [&](int l) { return eval ? F->mom_eval[l - 2] : F->lev[l].mom; };
  auto LOC = [&](int l) { return eval ? F->loc_eval[l - 2] : F->lev[l].loc; };
  double* Rfar = eval ? F->d_Rfar_eval : F->d_Rfar;
  // The deferred M2L of a level's previous event adds to local coefficients
  // that this event reads (and reads the packed moments it rewrites): order it
  // before any work of a level that fires now.  History evaluation packs into
  // the same buffers, so it waits for every level.
  for (int l = 2; l <= lmax; ++l) {
    FmmLevel& L = F->lev[l];
    if (L.defer_pending && (eval || alpha % L.M == 0)) {
      TDBEM_CUDA_TRY(c, cudaStreamWaitEvent(c->stream, L.ev_defer, 0));
      L.defer_pending = false;
    }
  }
  // upward pass
  for (int l = lmax; l >= 2; --l) {
    FmmLevel& L = F->lev[l];
    if (alpha % L.M) continue;
    int k = alpha / L.M - 1;
    if (L.nleaf) {
      int maxtri = 0;
      for (int i = 0; i < L.ncell; ++i)
        if (L.leaf[i]) maxtri = std::max(maxtri, L.tri_e[i] - L.tri_b[i]);
      size_t smem = (size_t)3 * maxtri * 2 * pt * sizeof(float);
      cudaEvent_t e = c->prof_begin(3);
      k_p2m<<<dim3(L.nleaf, R, 2), 256, smem, c->stream>>>(L.d_leaf_cells, L.d_tri_b, L.d_tri_e, F->d_perm, c->tg,
                                                         F->d_W, L.d_tsrc, ring, c->L, p, pt, L.M, k, MOM(l), R);
      c->prof_end(3, e);
      TDBEM_CUDA_TRY(c, cudaGetLastError());
    }
    if (L.nnonleaf && l < lmax) {
      cudaEvent_t e = c->prof_begin(4);
      constexpr int kZ = 7;  // blocks per cell, 2 of the 14 channels each
      size_t smem = (size_t)3 * ((2 * kNC + kZ - 1) / kZ) * P * sizeof(float);
      if (smem <= 227 * 1024)
        k_m2m_fact<<<dim3(L.nnonleaf, R, kZ), 512, smem, c->stream>>>(
            L.d_nonleaf_cells, L.d_child, F->d_Sx + (size_t)l * 2 * p * p, F->d_St, p, pt, k, MOM(l + 1), MOM(l), R);
      else  // large p: direct tensor-product sums from global memory
        k_m2m<<<dim3(L.nnonleaf, R), 256, 0, c->stream>>>(L.d_nonleaf_cells, L.d_child,
                                                           F->d_Sx + (size_t)l * 2 * p * p, F->d_St, p, pt, k,
                                                           MOM(l + 1), MOM(l), R);
      c->prof_end(4, e);
      TDBEM_CUDA_TRY(c, cudaGetLastError());
    }
  }
  // downward pass
  for (int l = 2; l <= lmax; ++l) {
    FmmLevel& L = F->lev[l];
    if (alpha % L.M) continue;
    int k = alpha / L.M - 1;
    if (L.ntiles) {
      const bool tc = c->p.m2l_prec != TDBEM_P_FP32;
      const int v = L.tc_mt - 1;
      if (tc) {
        cudaEvent_t e = c->prof_begin(8);
        tdbem_status s = L.res ? tdbem_m2l_pack_f16(c, L.d_cS, L.d_csym, L.ncombo, F->d_smap, MOM(l), k, R, PS, pt,
                                                    L.d_pk16, L.d_pkinv)
                               : tdbem_m2l_pack(c, L.d_cS, L.d_csym, L.ncombo, F->d_smap, MOM(l), k, R, PS, pt,
                                                L.d_pack, L.d_pkinv);
        if (s) return s;
        c->prof_end(8, e);
      }
      // tiles [t0, t0 + n) of this level's list, on c->stream
      auto m2l_range = [&](int t0, int n) -> tdbem_status {
        if (n <= 0) return TDBEM_OK;
        cudaEvent_t e = c->prof_begin(5);
        if (!tc) {
          k_m2l_fp32<<<n, 256, 0, c->stream>>>(L.d_gemm, L.d_tiles + t0, L.ops, P, pt, PS, L.d_pO, L.d_pS, L.d_psym,
                                               F->d_smap, MOM(l), k, LOC(l), L.Q, R);
          TDBEM_CUDA_TRY(c, cudaGetLastError());
        } else if (L.res) {
          // the deferred launch on the side stream runs one CTA per unit, so
          // that the hardware interleaves it with the steps it overlaps
          tdbem_status s = tdbem_m2l_res(c, L.d_gemm, L.d_units, t0, n, L.ops_img, P, pt, PS, L.d_pO, L.d_pC,
                                         L.d_psym, F->d_smap, L.d_pk16, k, LOC(l), L.Q, R, L.d_opinv, L.d_pkinv,
                                         F->d_err, (F->side && c->stream == F->side) ? -1 : 0);
          if (s) return s;
        } else {
          tdbem_status s = tdbem_m2l_tc(c, L.tc_mt, L.d_gemm, L.d_tiles_tc[v] + t0, n, L.ops_img, P, pt, PS, L.d_pO,
                                        L.d_pC, L.d_psym, F->d_smap, L.d_pack, k, LOC(l), L.Q, R, c->p.m2l_prec,
                                        L.d_opinv, L.d_pkinv, F->d_err);
          if (s) return s;
        }
        c->prof_end(5, e);
        return TDBEM_OK;
      };
      const int nall = L.res ? L.nunits : tc ? L.ntiles_tc[v] : L.ntiles;
      const int nu = L.res ? L.nunits_urgent : tc ? L.ntiles_tc_urgent[v] : L.ntiles_urgent;
      tdbem_status s;
      if (!F->side || eval) {
        if ((s = m2l_range(0, nall))) return s;
      } else {
        // lag 1 now; lags >= 2 on the side stream, overlapping the next
        // steps, waited for when this level fires again
        if ((s = m2l_range(0, nu))) return s;
        if (nall > nu) {
          TDBEM_CUDA_TRY(c, cudaEventRecord(F->ev_fork, c->stream));
          TDBEM_CUDA_TRY(c, cudaStreamWaitEvent(F->side, F->ev_fork, 0));
          cudaStream_t main = c->stream;
          c->stream = F->side;
          s = m2l_range(nu, nall - nu);
          c->stream = main;
          if (s) return s;
          TDBEM_CUDA_TRY(c, cudaEventRecord(L.ev_defer, F->side));
          L.defer_pending = true;
        }
      }
    }
    if (L.nnonleaf && l < lmax) {
      cudaEvent_t e = c->prof_begin(6);
      constexpr int kZ = 7;  // blocks per cell, one component each
      size_t smem = (size_t)3 * ((kNC + kZ - 1) / kZ) * P * sizeof(float);
      if (smem <= 227 * 1024)
        k_l2l_fact<<<dim3(L.nnonleaf, R, kZ), 512, smem, c->stream>>>(L.d_nonleaf_cells, L.d_child,
                                                                   F->d_Sx + (size_t)l * 2 * p * p, F->d_St, p, pt, k,
                                                                   LOC(l), L.Q, LOC(l + 1), F->lev[l + 1].Q, R);
      else
        k_l2l<<<dim3(L.nnonleaf, R), 256, 0, c->stream>>>(L.d_nonleaf_cells, L.d_child,
                                                           F->d_Sx + (size_t)l * 2 * p * p, F->d_St, p, pt, k, LOC(l),
                                                           L.Q, LOC(l + 1), F->lev[l + 1].Q, R);
      c->prof_end(6, e);
      TDBEM_CUDA_TRY(c, cudaGetLastError());
    }
    if (L.nleaf) {
      // steps per launch: as many of the interval's evaluated coefficients as
      // fit the 200 KB of shared memory the kernel is set up for
      const int per = std::max(1, (int)((200 * 1024) / (kNC * PS * sizeof(float))));
      cudaEvent_t e = c->prof_begin(7);
      for (int s0 = 0; s0 < L.M; s0 += per) {
        const int ns = std::min(per, L.M - s0);
        const size_t smem = (size_t)ns * kNC * PS * sizeof(float);
        k_l2p<<<dim3(L.nleaf, R), 256, smem, c->stream>>>(L.d_leaf_cells, L.d_tri_b, L.d_tri_e, F->d_perm, c->tg,
                                                           F->d_T, L.d_ttgt, p, pt, L.M, k, LOC(l), L.Q, Rfar, F->Lr,
                                                           c->ne, R, s0, ns, s0 + ns >= L.M ? 1 : 0,
                                                           a_target_kind(c->p.a_deriv));
        TDBEM_CUDA_TRY(c, cudaGetLastError());
      }
      c->prof_end(7, e);
      TDBEM_CUDA_TRY(c, cudaGetLastError());
    }
  }
  return TDBEM_OK;
}

static tdbem_status near_lags3(tdbem_ctx* c, const double* ring, int32_t alpha, double* out, cudaStream_t st);

tdbem_status tdbem_fast_history(tdbem_ctx* c, int32_t alpha, const double* ring, const double* V, bool eval) {
  FmmPlan* F = c->fmm;
  double* slot = nullptr;
  if (F->lmax >= 2)
    slot = (eval ? F->d_Rfar_eval : F->d_Rfar) + (int64_t)((alpha - 1) & (F->Lr - 1)) * c->ne * c->R;
  if (!eval && F->nstream) {
    // pipelined march: -(lags >= 3) was summed ahead on the near stream
    // (it depends on the history only); otherwise it is summed now
    const int b = alpha & 1;
    double* Rp = F->d_Rp + (int64_t)b * c->ne;
    const unsigned grid = (unsigned)((c->ne + 7) / 8);
    if (F->ahead[b]) TDBEM_CUDA_TRY(c, cudaStreamWaitEvent(c->stream, F->ev_near[b], 0));
    const bool have = F->ahead[b] == alpha;
    F->ahead[b] = 0;
    cudaEvent_t e = c->prof_begin(1);
    if (!have) {
      tdbem_status s = near_lags3(c, ring, alpha, Rp, c->stream);
      if (s) return s;
    }
    // V, lag 2 (the currents of the step just solved) and the far field
    k_near_history_flat<<<grid, 256, 0, c->stream>>>(F->d_hrow2, F->d_hval2, F->d_hmeta2, c->ne, ring, c->L, alpha,
                                                     V, Rp, slot, c->d_R);
    c->prof_end(1, e);
    TDBEM_CUDA_TRY(c, cudaGetLastError());
    return TDBEM_OK;
  }
  cudaEvent_t e = c->prof_begin(1);
  if (c->R == 1 && F->d_hrow3) {
    // history evaluation with only the lag-split entries: R = -(lags >= 3),
    // then V + lag 2 + far field added in place (V is an incident row here)
    const unsigned grid = (unsigned)((c->ne + 7) / 8);
    tdbem_status s = near_lags3(c, ring, alpha, c->d_R, c->stream);
    if (s) return s;
    k_near_history_flat<<<grid, 256, 0, c->stream>>>(F->d_hrow2, F->d_hval2, F->d_hmeta2, c->ne, ring, c->L, alpha,
                                                     V, c->d_R, slot, c->d_R);
  } else if (c->R == 1) {
    k_near_history_flat<<<(unsigned)((c->ne + 7) / 8), 256, 0, c->stream>>>(F->d_hrow, F->d_hval, F->d_hmeta, c->ne,
                                                                             ring, c->L, alpha, V, nullptr, slot,
                                                                             c->d_R);
  } else {
    int RL = 1;
    while (RL < c->R && RL < 32) RL <<= 1;
    k_near_history_flat_multi<<<(unsigned)c->ne, 256, 0, c->stream>>>(F->d_hrow, F->d_hval, F->d_hmeta, c->ne, ring,
                                                                        c->L, alpha, c->R, RL, V, slot, c->d_R);
  }
  c->prof_end(1, e);
  TDBEM_CUDA_TRY(c, cudaGetLastError());
  return TDBEM_OK;
}

// -(lags >= 3) of step alpha into out[ne] on stream st: the tiled kernel
// where it was built, else the flat one
static tdbem_status near_lags3(tdbem_ctx* c, const double* ring, int32_t alpha, double* out, cudaStream_t st) {
  FmmPlan* F = c->fmm;
  // the staged block holds the lags 0 .. max_near_lag of kNB columns
  const int nlag = F->max_near_lag + 1;
  const int smem = (int)(kNBS * nlag * sizeof(float));
  if (F->d_seg_ptr && smem <= 160 * 1024) {
    static int smem_set = 0;
    if (smem > smem_set) {
      TDBEM_CUDA_TRY(c, cudaFuncSetAttribute(k_near_tile, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
      smem_set = smem;
    }
    if (F->ntask)
      k_near_tile<<<(unsigned)F->ntask, 256, smem, st>>>(
          F->d_ntasks, F->d_corder, F->d_seg_ptr, F->d_cval, F->d_cmeta, c->ne, ring, c->L, nlag, alpha, 3,
          F->d_spart);
    k_near_seg_reduce<<<(unsigned)((c->ne * 8 + 255) / 256), 256, 0, st>>>(F->d_rseg_ptr, F->d_rseg, F->d_spart,
                                                                          c->ne, out);
  } else {
    k_near_history_flat<<<(unsigned)((c->ne + 7) / 8), 256, 0, st>>>(F->d_hrow3, F->d_hval3, F->d_hmeta3, c->ne, ring,
                                                                     c->L, alpha, nullptr, nullptr, nullptr, out);
  }
  TDBEM_CUDA_TRY(c, cudaGetLastError());
  return TDBEM_OK;
}

tdbem_status tdbem_fast_after_solve(tdbem_ctx* c, int32_t alpha) {
  FmmPlan* F = c->fmm;
  if (F->nstream && alpha + 2 <= c->Nt - 1) {
    // -(lags >= 3) of step alpha + 2 needs the currents up to J^{alpha-1},
    // which this solve completes; its buffer was last read by the lag-2 pass
    // of step alpha, before the solve.  It runs on the near stream while the
    // far field of this step and the next step proceed.
    const int32_t a2 = alpha + 2;
    const int b = a2 & 1;
    TDBEM_CUDA_TRY(c, cudaEventRecord(F->ev_solved, c->stream));
    TDBEM_CUDA_TRY(c, cudaStreamWaitEvent(F->nstream, F->ev_solved, 0));
    cudaStream_t main = c->stream;
    c->stream = F->nstream;
    cudaEvent_t e = c->prof_begin(1);
    tdbem_status s = near_lags3(c, c->d_Jring, a2, F->d_Rp + (int64_t)b * c->ne, F->nstream);
    c->prof_end(1, e);
    c->stream = main;
    if (s) return s;
    TDBEM_CUDA_TRY(c, cudaEventRecord(F->ev_near[b], F->nstream));
    F->ahead[b] = a2;
  }
  return far_events(c, alpha, c->d_Jring, false);
}

// Evaluation state for history_eval: cleared, then the far events of steps
// 1 .. alpha-1 are replayed on the supplied history.
tdbem_status tdbem_fast_eval_reset(tdbem_ctx* c) {
  FmmPlan* F = c->fmm;
  if (!F || F->lmax < 2) return TDBEM_OK;
  for (int l = 2; l <= F->lmax; ++l) {
    FmmLevel& L = F->lev[l];
    const int64_t RP = (int64_t)c->R * kNC * F->P;
    TDBEM_CUDA_TRY(c, cudaMemsetAsync(F->mom_eval[l - 2], 0, (int64_t)L.ncell * 4 * RP * sizeof(float), c->stream));
    TDBEM_CUDA_TRY(c, cudaMemsetAsync(F->loc_eval[l - 2], 0, (int64_t)L.ncell * L.Q * RP * sizeof(float), c->stream));
  }
  TDBEM_CUDA_TRY(c, cudaMemsetAsync(F->d_Rfar_eval, 0, (int64_t)F->Lr * c->ne * c->R * sizeof(double), c->stream));
  return TDBEM_OK;
}

tdbem_status tdbem_fast_consume_eval_slot(tdbem_ctx* c, int32_t alpha) {
  FmmPlan* F = c->fmm;
  if (!F || F->lmax < 2) return TDBEM_OK;
  TDBEM_CUDA_TRY(c, cudaMemsetAsync(F->d_Rfar_eval + (int64_t)((alpha - 1) & (F->Lr - 1)) * c->ne * c->R, 0,
                                    c->ne * c->R * sizeof(double), c->stream));
  return TDBEM_OK;
}

tdbem_status tdbem_fast_replay_step(tdbem_ctx* c, int32_t alpha, const double* ring) {
  return far_events(c, alpha, ring, true);
}

tdbem_status tdbem_fast_reset(tdbem_ctx* c) {
  FmmPlan* F = c->fmm;
  if (!F) return TDBEM_OK;
  tdbem_status s0 = tdbem_fast_invalidate(c);
  if (s0 || F->lmax < 2) return s0;
  for (int l = 2; l <= F->lmax; ++l) {
    FmmLevel& L = F->lev[l];
    const int64_t RP = (int64_t)c->R * kNC * F->P;
    TDBEM_CUDA_TRY(c, cudaMemsetAsync(L.mom, 0, (int64_t)L.ncell * 4 * RP * sizeof(float), c->stream));
    TDBEM_CUDA_TRY(c, cudaMemsetAsync(L.loc, 0, (int64_t)L.ncell * L.Q * RP * sizeof(float), c->stream));
  }
  TDBEM_CUDA_TRY(c, cudaMemsetAsync(F->d_Rfar, 0, (int64_t)F->Lr * c->ne * c->R * sizeof(double), c->stream));
  return TDBEM_OK;
}

// The context's stream waits for every deferred M2L and every near-field
// sum launched ahead that is still in flight (the sums stay usable).
tdbem_status tdbem_fast_join(tdbem_ctx* c) {
  FmmPlan* F = c->fmm;
  if (!F) return TDBEM_OK;
  for (int b = 0; b < 2; ++b)
    if (F->ahead[b]) TDBEM_CUDA_TRY(c, cudaStreamWaitEvent(c->stream, F->ev_near[b], 0));
  for (int l = 2; l <= F->lmax; ++l) {
    FmmLevel& L = F->lev[l];
    if (L.defer_pending) {
      TDBEM_CUDA_TRY(c, cudaStreamWaitEvent(c->stream, L.ev_defer, 0));
      L.defer_pending = false;
    }
  }
  return TDBEM_OK;
}

// As tdbem_fast_join, and the sums launched ahead are discarded (the march
// state is about to change).
tdbem_status tdbem_fast_invalidate(tdbem_ctx* c) {
  FmmPlan* F = c->fmm;
  if (!F) return TDBEM_OK;
  tdbem_status s = tdbem_fast_join(c);
  F->ahead[0] = F->ahead[1] = 0;
  return s;
}

// Device buffers of the fast mode's march state, in a fixed order: per far
// level its moments and local coefficients, then the far right-hand-side
// ring (the evaluation state of history_eval and the near-field sums launched
// ahead are not part of it: the former is rebuilt per call, the latter are
// recomputed by the same kernel when absent).
void tdbem_fast_state(tdbem_ctx* c, std::vector<std::pair<void*, size_t>>* bufs) {
  FmmPlan* F = c->fmm;
  if (!F || F->lmax < 2) return;
  const int64_t RP = (int64_t)c->R * kNC * F->P;
  for (int l = 2; l <= F->lmax; ++l) {
    FmmLevel& L = F->lev[l];
    bufs->push_back({L.mom, (size_t)L.ncell * 4 * RP * sizeof(float)});
    bufs->push_back({L.loc, (size_t)L.ncell * L.Q * RP * sizeof(float)});
  }
  bufs->push_back({F->d_Rfar, (size_t)F->Lr * c->ne * c->R * sizeof(double)});
}

void tdbem_fast_free(tdbem_ctx* c) {
  FmmPlan* F = c->fmm;
  if (F) {
    if (F->nstream) cudaStreamSynchronize(F->nstream);
    for (int b = 0; b < 2; ++b)
      if (F->ev_near[b]) cudaEventDestroy(F->ev_near[b]);
    if (F->ev_solved) cudaEventDestroy(F->ev_solved);
    if (F->nstream) cudaStreamDestroy(F->nstream);
    if (F->side) cudaStreamSynchronize(F->side);
    for (size_t l = 2; l < F->lev.size(); ++l)
      if (F->lev[l].ev_defer) cudaEventDestroy(F->lev[l].ev_defer);
    if (F->ev_fork) cudaEventDestroy(F->ev_fork);
    if (F->side) cudaStreamDestroy(F->side);
  }
  delete c->fmm;
  c->fmm = nullptr;
}

void tdbem_fast_info(const tdbem_ctx* c, tdbem_info* info) {
  const FmmPlan* F = c->fmm;
  if (!F) return;
  info->lmax = F->lmax;
  info->n_levels = F->lmax + 1;
  info->mt_leaf = F->lmax >= 2 ? F->lev[F->lmax].M : 0;
  info->n_near_pairs = F->nnz;
  info->near_coef_bytes = F->nval * (int64_t)sizeof(float);
  int64_t il = 0;
  double fl = 0;
  for (int l = 2; l <= F->lmax; ++l) {
    il += F->lev[l].npairs;
    if (F->lev[l].M) fl += F->lev[l].flops_event / F->lev[l].M;
  }
  info->n_far_pairs = il;
  info->m2l_flops_per_step = fl;
  for (int l = 2; l <= F->lmax && l < 8; ++l) {
    info->m2l_tile_rows[l] = (c->p.m2l_prec != TDBEM_P_FP32 && F->lev[l].ntiles_tc[0])
                                 ? (F->lev[l].res ? 128 : 128 * F->lev[l].tc_mt)
                                 : 0;
    if (F->lev[l].res) info->m2l_resident |= 1 << l;
  }
}

// CSR of Z0 from the near store
tdbem_status tdbem_fast_z0_source(const tdbem_ctx* c, const int64_t** row_ptr, const int32_t** col,
                                  const int16_t** m_lo, const uint8_t** nlag, const int64_t** off, const double** val) {
  const FmmPlan* F = c->fmm;
  *row_ptr = F->d_row_ptr;
  *col = F->d_col;
  *m_lo = F->d_mlo;
  *nlag = F->d_nlag;
  *off = F->d_off;
  *val = F->d_val64;
  return TDBEM_OK;
}

// timeouts recorded by bounded device waits (0: none)
tdbem_status tdbem_fast_check(tdbem_ctx* c) {
  FmmPlan* F = c->fmm;
  if (!F || !F->d_err) return TDBEM_OK;
  int32_t h = 0;
  TDBEM_CUDA_TRY(c, cudaMemcpyAsync(&h, F->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
  TDBEM_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (h) {
    c->set_error("fast: a bounded wait of the tensor-core M2L expired");
    return TDBEM_ETIMEOUT;
  }
  return TDBEM_OK;
}
