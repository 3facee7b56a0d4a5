// direct.cu -- interaction coefficients of every time lag for a set of edge
// pairs (paper section 2.4, eq. z_ij), the incident right-hand side (eq. v_i)
// and the direct FP64 history sum of eq. R.
//
// The coefficient of J_j^beta in the tested equation at t_alpha depends on the
// lag m = alpha - beta only (eq. layer_disc_tmp with the B-spline of eq. J):
//   Zt^(m)_ij = sum over the triangles S_i^rho of i and S_j^sigma of j of
//     sum_q w_q A_i^rho [ mu/(4 pi dt^2) f_i(x_q) . int f_j Nddot(tau)/r dS
//                       + 1/(4 pi eps) div f_i div f_j int N(tau)/r dS
//                       + theta eta/(4 pi) f_i(x_q) . (n x int f_j x grad_y g dS) ]
// plus the MFIE identity term s_jump theta eta/2 (f_i, f_j) (chi Ndot(m)/dt + zeta N(m)).
// The outer integral uses the 7-point degree-5 rule; the inner integral is
// exact (integrals.cuh).  One thread owns one (test triangle, source triangle)
// pair, accumulates its 3x3 local edge pairs over the 7 points and adds them to
// the edge-pair store with FP64 atomics (each edge pair receives the 4
// triangle pairs of its two supports).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <type_traits>
#include <vector>

#include "integrals.cuh"
#include "internal.h"
#include "tc.cuh"

namespace tdbem {

__device__ __forceinline__ double dist3(const double* a, const double* b) {
  double x = a[0] - b[0], y = a[1] - b[1], z = a[2] - b[2];
  return sqrt(x * x + y * y + z * z);
}

// Conservative lag window [m_lo, m_lo + n) of an edge pair from the bounding
// spheres (centroid, max centroid-vertex distance) of its four triangle pairs.
__device__ __forceinline__ void edge_pair_window(const TriGeom& g, const int32_t* et, int i, int j, double a,
                                                 int* m_lo, int* n) {
  double rlo = 1e300, rhi = 0.0;
  for (int u = 0; u < 2; ++u)
    for (int w = 0; w < 2; ++w) {
      int t = et[2 * i + u], s = et[2 * j + w];
      double dc = dist3(g.cen + 3 * t, g.cen + 3 * s);
      double rr = g.rad[t] + g.rad[s];
      rlo = fmin(rlo, fmax(dc - rr, 0.0));
      rhi = fmax(rhi, dc + rr);
    }
  lag_window(rlo, rhi, a, m_lo, n);
}

__global__ void k_direct_windows(TriGeom g, const int32_t* et, int64_t ne, double a, int16_t* m_lo, uint8_t* nlag,
                                 int32_t* err) {
  int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= ne * ne) return;
  int i = (int)(p / ne), j = (int)(p % ne);
  int lo, n;
  edge_pair_window(g, et, i, j, a, &lo, &n);
  if (n > 255 || lo > 32767) {
    atomicExch(err, 1);
    n = 0;
  }
  m_lo[p] = (int16_t)lo;
  nlag[p] = (uint8_t)n;
}

// largest stored lag m_lo + nlag - 1 over all pairs (atomic maximum into *mx)
__global__ void k_max_lag(const int16_t* m_lo, const uint8_t* nlag, int64_t n, int32_t* mx) {
  int v = 0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
    if (nlag[p]) v = max(v, (int)m_lo[p] + (int)nlag[p] - 1);
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) atomicMax(mx, v);
}

// per-row sums of nlag
__global__ void k_row_totals(const uint8_t* nlag, int64_t ne, int64_t* tot) {
  int64_t i = blockIdx.x;
  int64_t s = 0;
  for (int64_t j = threadIdx.x; j < ne; j += blockDim.x) s += nlag[i * ne + j];
  __shared__ int64_t red[32];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) tot[i] = s;
  }
}

// per-row exclusive scan of nlag into off (row base from the host scan)
__global__ void k_row_offsets(const uint8_t* nlag, int64_t ne, const int64_t* rowbase, int64_t* off) {
  int64_t i = blockIdx.x;
  __shared__ int64_t wsum[32];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = rowbase[i];
  __syncthreads();
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t j0 = 0; j0 < ne; j0 += blockDim.x) {
    int64_t j = j0 + threadIdx.x;
    int64_t v = (j < ne) ? nlag[i * ne + j] : 0;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
      int64_t w = (lane < nw) ? wsum[lane] : 0;
      for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, w, o);
        if (lane >= o) w += y;
      }
      if (lane < nw) wsum[lane] = w;
    }
    __syncthreads();
    int64_t excl = x - v + (wid > 0 ? wsum[wid - 1] : 0) + carry;
    if (j < ne) off[i * ne + j] = excl;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = excl + v;
    __syncthreads();
  }
}

// Sink of the direct store: every (i, j) of the mesh.  An edge pair receives
// one contribution from each of the four triangle pairs of its two supports,
// class k = 2 (test triangle is i's "-" triangle) + (source triangle is j's
// "-" triangle).  With val4 set, contribution k goes to its own slot
// val4[4 (off + w) + k] with a plain store, and k_sum4 adds the four in a
// fixed order afterwards, so the stored coefficients do not depend on the
// order in which threads finish; without it the contributions are added to
// val with FP64 atomics.
struct DirectSink {
  const int16_t* m_lo;
  const uint8_t* nlag;
  const int64_t* off;
  double* val;
  int64_t ne;
  double* val4;
  __device__ __forceinline__ bool add(int i, int j, int m, int k, double v) const {
    int64_t p = (int64_t)i * ne + j;
    int w = m - m_lo[p];
    if (w < 0 || w >= nlag[p]) return false;
    if (val4)
      val4[4 * (off[p] + w) + k] = v;
    else
      atomicAdd(val + off[p] + w, v);
    return true;
  }
};

// val[e] = ((v4[4e] + v4[4e+1]) + v4[4e+2]) + v4[4e+3]
__global__ void k_sum4(const double* v4, int64_t n, double* val) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n) return;
  const double* q = v4 + 4 * e;
  val[e] = ((q[0] + q[1]) + q[2]) + q[3];
}

// One thread per (test triangle t, source triangle s) listed in `pairs` (or
// all pairs when pairs == nullptr).
template <class Sink>
__global__ void __launch_bounds__(128) k_assemble(TriGeom g, Phys ph, int64_t nt, const int2* pairs, int64_t npairs,
                                                  Sink sink, int32_t* err) {
  int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= npairs) return;
  int t, s;
  if (pairs) {
    int2 q = pairs[idx];
    t = q.x;
    s = q.y;
  } else {
    t = (int)(idx / nt);
    s = (int)(idx % nt);
  }
  const double a = ph.a;
  // union lag window of the triangle pair
  double dc = dist3(g.cen + 3 * t, g.cen + 3 * s);
  int M0, NM;
  lag_window(fmax(dc - g.rad[t] - g.rad[s], 0.0), dc + g.rad[t] + g.rad[s], a, &M0, &NM);
  if (NM > kMaxWin) {
    atomicExch(err, 2);
    return;
  }
  double acc[3][3][kMaxWin];
  for (int u = 0; u < 3; ++u)
    for (int w = 0; w < 3; ++w)
      for (int k = 0; k < NM; ++k) acc[u][w][k] = 0.0;
  double vt[9], vs[9], ns[3], nin[3];
  for (int k = 0; k < 9; ++k) {
    vt[k] = g.v[9 * t + k];
    vs[k] = g.v[9 * s + k];
  }
  for (int k = 0; k < 3; ++k) {
    ns[k] = g.nrm[3 * s + k];
    nin[k] = -g.nrm[3 * t + k];  // n points into the conductor (paper section 2.1)
  }
  const double At = g.area[t], As = g.area[s];
  double ci[3], divi[3], oi[3][3], cj[3], divj[3], oj[3][3];
  for (int k = 0; k < 3; ++k) {
    double sg = g.sgn[3 * t + k], l = g.elen[3 * t + k];
    ci[k] = sg * l / (2 * At);
    divi[k] = sg * l / At;
    for (int q = 0; q < 3; ++q) oi[k][q] = g.opp[9 * t + 3 * k + q];
    double sg2 = g.sgn[3 * s + k], l2 = g.elen[3 * s + k];
    cj[k] = sg2 * l2 / (2 * As);
    divj[k] = sg2 * l2 / As;
    for (int q = 0; q < 3; ++q) oj[k][q] = g.opp[9 * s + 3 * k + q];
  }
  const double PI = 3.14159265358979323846;
  const double kA = ph.mu / (4 * PI * ph.dt * ph.dt), kphi = 1.0 / (4 * PI * ph.eps), kP = ph.theta * ph.eta / (4 * PI);
  InnerOut io;
  for (int q = 0; q < kNq; ++q) {
    double x[3];
    for (int k = 0; k < 3; ++k) x[k] = ph.qb[q][0] * vt[k] + ph.qb[q][1] * vt[3 + k] + ph.qb[q][2] * vt[6 + k];
    double wq = ph.qw[q] * At;
    double rhi = fmax(fmax(dist3(x, vs), dist3(x, vs + 3)), dist3(x, vs + 6));
    double rlo = fmax(dist3(x, g.cen + 3 * s) - g.rad[s], 0.0);
    int m0, nm;
    lag_window(rlo, rhi, a, &m0, &nm);
    if (m0 < M0 || m0 + nm > M0 + NM || nm > kMaxWin) {
      atomicExch(err, 3);
      return;
    }
    if (!inner_integrals(x, vs, ns, g.lmax[s], a, ph.chi / ph.dt, ph.zeta, m0, nm, io)) {
      atomicExch(err, 4);
      return;
    }
    double fi[3][3], xo[3][3];
    for (int k = 0; k < 3; ++k)
      for (int u = 0; u < 3; ++u) {
        fi[k][u] = ci[k] * (x[u] - oi[k][u]);
        xo[k][u] = x[u] - oj[k][u];
      }
    const double h = io.h;
    for (int im = 0; im < nm; ++im) {
      double A1[3], P1[3];
      for (int u = 0; u < 3; ++u) {
        A1[u] = io.EA[im][u] - h * ns[u] * io.A0[im];
        P1[u] = io.EP[im][u] - h * ns[u] * io.Sn[im];
      }
      for (int ks = 0; ks < 3; ++ks) {
        double IA[3], IP[3], nIP[3];
        for (int u = 0; u < 3; ++u) IA[u] = cj[ks] * (A1[u] + xo[ks][u] * io.A0[im]);
        IP[0] = cj[ks] * (xo[ks][1] * P1[2] - xo[ks][2] * P1[1]);
        IP[1] = cj[ks] * (xo[ks][2] * P1[0] - xo[ks][0] * P1[2]);
        IP[2] = cj[ks] * (xo[ks][0] * P1[1] - xo[ks][1] * P1[0]);
        nIP[0] = nin[1] * IP[2] - nin[2] * IP[1];
        nIP[1] = nin[2] * IP[0] - nin[0] * IP[2];
        nIP[2] = nin[0] * IP[1] - nin[1] * IP[0];
        for (int kt = 0; kt < 3; ++kt) {
          double val = kA * (fi[kt][0] * IA[0] + fi[kt][1] * IA[1] + fi[kt][2] * IA[2]) +
                       kphi * divi[kt] * divj[ks] * io.phi[im] +
                       kP * (fi[kt][0] * nIP[0] + fi[kt][1] * nIP[1] + fi[kt][2] * nIP[2]);
          acc[kt][ks][m0 - M0 + im] += wq * val;
        }
      }
    }
    // MFIE identity term on the test triangle itself (lags 1 and 2)
    if (s == t && ph.s_jump != 0.0) {
      const double c1 = ph.chi / ph.dt + 0.5 * ph.zeta, c2 = -ph.chi / ph.dt + 0.5 * ph.zeta;
      for (int kt = 0; kt < 3; ++kt)
        for (int ks = 0; ks < 3; ++ks) {
          double fj[3];
          for (int u = 0; u < 3; ++u) fj[u] = cj[ks] * xo[ks][u];
          double G = wq * (fi[kt][0] * fj[0] + fi[kt][1] * fj[1] + fi[kt][2] * fj[2]);
          double sc = ph.s_jump * ph.theta * ph.eta * 0.5 * G;
          if (1 - M0 >= 0 && 1 - M0 < NM) acc[kt][ks][1 - M0] += sc * c1;
          if (2 - M0 >= 0 && 2 - M0 < NM) acc[kt][ks][2 - M0] += sc * c2;
        }
    }
  }
  for (int kt = 0; kt < 3; ++kt) {
    int i = g.edge[3 * t + kt];
    for (int ks = 0; ks < 3; ++ks) {
      int j = g.edge[3 * s + ks];
      for (int k = 0; k < NM; ++k) {
        double v = acc[kt][ks][k];
        if (v == 0.0) continue;
        const int cls = (g.sgn[3 * t + kt] < 0 ? 2 : 0) + (g.sgn[3 * s + ks] < 0 ? 1 : 0);
        if (!sink.add(i, j, M0 + k, cls, v)) atomicExch(err, 5);
      }
    }
  }
}

template __global__ void k_assemble<DirectSink>(TriGeom, Phys, int64_t, const int2*, int64_t, DirectSink, int32_t*);

// Sink of a sparse edge-pair store: CSR over test edges i, sorted source edges j.
struct CsrSink {
  const int64_t* row_ptr;
  const int32_t* col;
  const int16_t* m_lo;
  const uint8_t* nlag;
  const int64_t* off;
  double* val;
  __device__ __forceinline__ bool add(int i, int j, int m, int /*k*/, double v) const {
    int64_t lo = row_ptr[i], hi = row_ptr[i + 1] - 1;
    while (lo <= hi) {
      int64_t mid = (lo + hi) >> 1;
      int c = col[mid];
      if (c == j) {
        int w = m - m_lo[mid];
        if (w < 0 || w >= nlag[mid]) return false;
        atomicAdd(val + off[mid] + w, v);
        return true;
      }
      if (c < j) lo = mid + 1; else hi = mid - 1;
    }
    return false;
  }
};

template __global__ void k_assemble<CsrSink>(TriGeom, Phys, int64_t, const int2*, int64_t, CsrSink, int32_t*);

// windows of the listed edge pairs (CSR entries)
__global__ void k_csr_windows(TriGeom g, const int32_t* et, const int64_t* row_ptr, const int32_t* col, int64_t ne,
                              double a, int16_t* m_lo, uint8_t* nlag, int32_t* err) {
  int64_t i = blockIdx.x;
  if (i >= ne) return;
  for (int64_t p = row_ptr[i] + threadIdx.x; p < row_ptr[i + 1]; p += blockDim.x) {
    int lo, n;
    edge_pair_window(g, et, (int)i, col[p], a, &lo, &n);
    if (n > 255 || lo > 32767) {
      atomicExch(err, 1);
      n = 0;
    }
    m_lo[p] = (int16_t)lo;
    nlag[p] = (uint8_t)n;
  }
}

// ---------------------------------------------------------------------------
// Incident right-hand side V_i^{alpha-1} (eq. v_i) for a plane wave (a
// modulated Gaussian, or the Sin^2 pulse of section 4.1 when sigma < 0); one
// thread per edge, 2 triangles x 7 points, FP64.
// grid: (edge blocks, steps); right-hand side r of R:
// V[((alpha-alpha0)*ne + i)*R + r] for alpha = alpha0 .. alpha0+gridDim.y-1
__global__ void k_rhs_plane(TriGeom g, Phys ph, const int32_t* et, int64_t ne, const double* pulse, int32_t alpha0,
                            int32_t R, int32_t r, double* V) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= ne) return;
  const int32_t alpha = alpha0 + blockIdx.y;
  double* Rv = V + (int64_t)(alpha - alpha0) * ne * R;
  const double PI = 3.14159265358979323846;
  double kv[3] = {pulse[0], pulse[1], pulse[2]}, pol[3] = {pulse[3], pulse[4], pulse[5]};
  double f0 = pulse[6], sg = pulse[7], t0 = pulse[8], zmin = pulse[9];
  double kxp[3] = {kv[1] * pol[2] - kv[2] * pol[1], kv[2] * pol[0] - kv[0] * pol[2], kv[0] * pol[1] - kv[1] * pol[0]};
  double t = alpha * ph.dt;
  double sum = 0.0;
  for (int rho = 0; rho < 2; ++rho) {
    int tri = et[2 * i + rho];
    int side = 0;
    for (int k = 0; k < 3; ++k)
      if (g.edge[3 * tri + k] == (int)i) side = k;
    double sgn = g.sgn[3 * tri + side], A = g.area[tri];
    double ci = sgn * g.elen[3 * tri + side] / (2 * A);
    const double* o = g.opp + 9 * tri + 3 * side;
    const double* v = g.v + 9 * tri;
    double nin[3] = {-g.nrm[3 * tri], -g.nrm[3 * tri + 1], -g.nrm[3 * tri + 2]};
    for (int q = 0; q < kNq; ++q) {
      double x[3];
      for (int u = 0; u < 3; ++u) x[u] = ph.qb[q][0] * v[u] + ph.qb[q][1] * v[3 + u] + ph.qb[q][2] * v[6 + u];
      double u_ = t - (kv[0] * x[0] + kv[1] * x[1] + kv[2] * x[2] - zmin) / ph.c;
      double vv = u_ - t0;
      double gg, gd;
      if (sg > 0) {
        double e = exp(-vv * vv / (2 * sg * sg));
        double sw, cw;
        sincos(2 * PI * f0 * vv, &sw, &cw);
        gg = cw * e;
        gd = (-2 * PI * f0 * sw - vv / (sg * sg) * cw) * e;
      } else {  // Sin^2 pulse: length f0, amplitude -sg
        const double w = 2 * PI * ph.c / f0, ph_ = w * vv;
        gg = gd = 0.0;
        if (ph_ >= 0.0 && ph_ <= 2 * PI) {
          double sw, cw;
          sincos(ph_, &sw, &cw);
          gg = -sg * sw * sw;
          gd = -sg * 2.0 * sw * cw * w;
        }
      }
      // -Edot + theta eta n x (chi Hdot + zeta H), E = pol g, H = k x pol g / eta
      double Hm[3], nH[3];
      for (int u = 0; u < 3; ++u) Hm[u] = kxp[u] * (ph.chi * gd + ph.zeta * gg) / ph.eta;
      nH[0] = nin[1] * Hm[2] - nin[2] * Hm[1];
      nH[1] = nin[2] * Hm[0] - nin[0] * Hm[2];
      nH[2] = nin[0] * Hm[1] - nin[1] * Hm[0];
      double val = 0.0;
      for (int u = 0; u < 3; ++u) val += ci * (x[u] - o[u]) * (-pol[u] * gd + ph.theta * ph.eta * nH[u]);
      sum += ph.qw[q] * A * val;
    }
  }
  Rv[i * R + r] = sum;
}

// The single-right-hand-side history sum runs on the FP32 pipes in
// double-float arithmetic (each FP64 operand held as an unevaluated sum of two
// FP32 numbers, hi + lo with |lo| <= ulp(hi)/2): GB300 issues FP64 FMAs at
// 1/64 of its FP32 rate, which bounded the plain FP64 loop well below the HBM
// roofline.  The product of two split numbers keeps hi*hi exactly (an FMA
// recovers its rounding error) and the two cross terms; the dropped lo*lo and
// the splits themselves are below 2^-47 of the product, so a term carries 46
// significant bits against FP64's 53 while the sum stays compensated (TwoSum
// into a hi/lo accumulator).  Operands must lie inside FP32's normal range.
__device__ __forceinline__ float2 df_split(double v) {
  const float h = __double2float_rn(v);
  return make_float2(h, __double2float_rn(v - (double)h));
}

__device__ __forceinline__ void df_fma_acc(float& sh, float& sl, float2 z, float2 x) {
  const float p = __fmul_rn(z.x, x.x);
  float e = __fmaf_rn(z.x, x.x, -p);
  e = __fmaf_rn(z.x, x.y, e);
  e = __fmaf_rn(z.y, x.x, e);
  const float s = __fadd_rn(sh, p);  // TwoSum(sh, p)
  const float bb = __fsub_rn(s, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(err, e));
}

// (sh, sl) += (bh, bl), both double-float: TwoSum of the high parts, the low
// parts and the rounding error added to the low part.
__device__ __forceinline__ void df_add(float& sh, float& sl, float bh, float bl) {
  const float s = __fadd_rn(sh, bh);
  const float bb = __fsub_rn(s, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(bh, bb));
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(err, bl));
}

// Stored coefficients split in place, double -> (hi, lo) pair of the same 8 bytes.
__global__ void k_split_values(double* val, int64_t n) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const float2 s = df_split(val[t]);
  reinterpret_cast<float2*>(val)[t] = s;
}

// ring2[slot*ne + j] = split(ring[j*L + slot]): the history of one right-hand
// side transposed, so that the columns of a warp at one lag read contiguously.
__global__ void k_ring_split(const double* ring, int64_t ne, int32_t L, float2* ring2) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= ne * L) return;
  const int64_t j = t / L;
  const int32_t slot = (int32_t)(t - j * L);
  ring2[(int64_t)slot * ne + j] = df_split(ring[t]);
}

constexpr int kDhThreads = 256;  // column pairs per chunk (one per thread)
constexpr int kDhCap = 3072;     // coefficients staged per chunk buffer (24 KB; four blocks per SM)

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(a), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(a), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

struct DhChunk {
  int lo = 0, n = 0;
  int64_t o = 0, start = 0, cnt = 0;
};

// Metadata of the chunk starting at column j0 (thread t takes column j0 + t).
__device__ __forceinline__ DhChunk dh_meta(const int16_t* m_lo, const uint8_t* nlag, const int64_t* off, int64_t row0,
                                           int64_t ne, int64_t j0) {
  DhChunk m;
  const int64_t j = j0 + threadIdx.x;
  if (j < ne) {
    m.lo = m_lo[row0 + j];
    m.n = nlag[row0 + j];
    m.o = off[row0 + j];
  }
  const int64_t last = min(j0 + kDhThreads, ne) - 1;
  m.start = off[row0 + j0];
  m.cnt = off[row0 + last] + nlag[row0 + last] - m.start;
  return m;
}

// R_i = V_i - sum_j sum_{m >= 2, alpha-m >= 0} Zt^(m)_ij J_j^{alpha-m} (eq. R;
// V may be null: zero; V may alias R); one block per row i, thread t taking
// column j0 + t of each chunk of 256 columns.  The row's stored lags are
// contiguous in column order, so a chunk owns one contiguous coefficient
// range: it is copied into shared memory with asynchronous copies one chunk
// ahead of the arithmetic (a chunk larger than a buffer is read from global
// memory in place) while the metadata is loaded two chunks ahead.  val holds
// split coefficients (k_split_values), ring2 the split, transposed history
// (k_ring_split).
__global__ void __launch_bounds__(kDhThreads) k_direct_history(const int16_t* m_lo, const uint8_t* nlag,
                                                               const int64_t* off, const float2* val, int64_t ne,
                                                               const float2* ring2, int32_t L, int32_t alpha,
                                                               const double* V, double* R) {
  extern __shared__ float2 zbuf[];  // [2][kDhCap]
  __shared__ double red[kDhThreads / 32];
  const int64_t row0 = (int64_t)blockIdx.x * ne;
  const int64_t nchunk = (ne + kDhThreads - 1) / kDhThreads;
  float sh = 0.f, sl = 0.f;
  DhChunk cur = dh_meta(m_lo, nlag, off, row0, ne, 0);
  if (cur.cnt <= kDhCap)
    for (int64_t k = threadIdx.x; k < cur.cnt; k += kDhThreads) cp_async8(zbuf + k, val + cur.start + k);
  cp_async_commit();
  DhChunk nxt;
  if (nchunk > 1) nxt = dh_meta(m_lo, nlag, off, row0, ne, kDhThreads);
  for (int64_t c = 0; c < nchunk; ++c) {
    float2* buf = zbuf + (c & 1) * kDhCap;
    if (c + 1 < nchunk && nxt.cnt <= kDhCap) {
      float2* nb = zbuf + ((c + 1) & 1) * kDhCap;
      for (int64_t k = threadIdx.x; k < nxt.cnt; k += kDhThreads) cp_async8(nb + k, val + nxt.start + k);
    }
    cp_async_commit();
    DhChunk nn;
    if (c + 2 < nchunk) nn = dh_meta(m_lo, nlag, off, row0, ne, (c + 2) * kDhThreads);
    cp_async_wait1();
    __syncthreads();
    {
      // this column's lags m = lo + w with m >= 2 and alpha - m >= 0
      const int64_t j = c * kDhThreads + threadIdx.x;
      const float2* z = (cur.cnt <= kDhCap) ? buf + (cur.o - cur.start) : val + cur.o;
      const int w0 = max(0, 2 - cur.lo), w1 = min(cur.n, alpha - cur.lo + 1);
#pragma unroll 4
      for (int w = w0; w < w1; ++w) {
        const int slot = (alpha - cur.lo - w) & (L - 1);
        df_fma_acc(sh, sl, z[w], __ldg(ring2 + (int64_t)slot * ne + j));
      }
    }
    const float s = __fadd_rn(sh, sl);  // renormalise once per chunk
    sl = __fsub_rn(sl, __fsub_rn(s, sh));
    sh = s;
    __syncthreads();
    cur = nxt;
    nxt = nn;
  }
  double s = (double)sh + (double)sl;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kDhThreads / 32; ++w) t += red[w];
    R[blockIdx.x] = (V ? V[blockIdx.x] : 0.0) - t;
  }
}

// R_i = V_i - (the nparts partials of row i plus the row's lag-2 entries l2
// against J^{alpha-2}, in FP64).  Eight lanes share a row: lane s of the group
// adds the partials k = s, s + 8, ... and the lag-2 entries e = s, s + 8, ...
// in order, and the eight sums meet in a fixed shuffle tree, so the result
// does not depend on scheduling.  V may be null (zero) and may alias R.
constexpr int kRedLanes = 8;

__global__ void k_direct_reduce(const double* partial, int32_t nparts, int64_t ne, const int64_t* l2_ptr,
                                const int32_t* l2_col, const double* l2_val, const double* ring, int32_t L,
                                int32_t alpha, const double* V, double* R) {
  const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / kRedLanes;
  const int sub = threadIdx.x % kRedLanes;
  double t = 0.0;
  if (i < ne) {
    for (int k = sub; k < nparts; k += kRedLanes) t += partial[(int64_t)k * ne + i];
    if (alpha >= 2) {
      const int slot = (alpha - 2) & (L - 1);
      for (int64_t e = l2_ptr[i] + sub; e < l2_ptr[i + 1]; e += kRedLanes)
        t += l2_val[e] * ring[(int64_t)l2_col[e] * L + slot];
    }
  }
#pragma unroll
  for (int d = kRedLanes / 2; d > 0; d >>= 1) t += __shfl_xor_sync(0xffffffffu, t, d);
  if (i < ne && sub == 0) R[i] = (V ? V[i] : 0.0) - t;
}

// Row-tile form of the single-right-hand-side history sum of the lags >= 3.
//
// Store.  Rows are taken in tiles of 32 (tile rt: rows 32 rt .. 32 rt + 31,
// lane t of a warp is row 32 rt + t).  For each (tile, column j) let nmax be
// the largest number of stored lags >= 3 over the tile's rows; the pair
// (tile, j) owns nmax groups of 32 values, group u holding for lane t the
// coefficient of lag lo3 + u of (32 rt + t, j), where lo3 = max(first stored
// lag, 3), and zero past that row's own window.  Groups run tile by tile and,
// inside a tile, column by column, so the groups of one tile and one block of
// columns are one contiguous stretch of memory.  A group is 32 values in a
// row: 128 bytes in FP32, 256 in (hi, lo) pairs, 96 in the 24-bit form (F24
// below).  goff[rt * ne + j] is the
// first group of (rt, j) (the next entry its end), lo3 one byte per
// (row, column).
//
// Kernel.  Block (cb, rg) takes the column block j0 = 64 cb .. j0 + 63 and the
// row tiles of group rg; its history J^{alpha - m}_j (m = 0 .. Lh - 1) is
// staged column-major in shared memory once, zero for the lags not summed
// (m < m_min, m > alpha, m >= L), so that zero padding and early steps need
// no test.  Each warp owns a row tile at a time and streams the tile's
// stretch for the block's columns through a private ring of about 2 KB stages
// filled by bulk copies (cp.async.bulk, one lane issues, an mbarrier per
// stage counts the bytes); every lane sums its own row over the block's
// columns and lags, so no cross-lane reduction is needed, and writes
// partial[cb * ne + row].  Per (tile, column) a lane's first lag and the
// column's end group are loaded five columns ahead.  The lanes of a warp read
// one column at lags that differ by their rows' distances, so the history
// reads are broadcasts or distinct banks.  Every wait is bounded: on expiry
// the warp writes NaN partials (the solve then misses its tolerance), sets
// *err, waits (bounded) for its copies in flight and stops.
//
// Arithmetic.  (hi, lo) pairs: the history is split into (hi, lo) pairs too
// and every product and sum is double-float (df_fma_acc).  FP32 store: the
// history is rounded to FP32, each column's lags are summed with FP32 FMAs
// (at most nmax terms) and the column sums are added in double-float.  With
// u = 2^-24 the FP32 form's error on row i is then at most about
// (2 + nmax) u sum |Zt^(m)_ij| |J_j^{alpha-m}| (two roundings per product,
// the recursive-sum bound over a column), one FMA per stored value.  The
// 24-bit store adds its own rounding, 2^-16 sum |Zt^(m)_ij| |J_j^{alpha-m}|.
constexpr int kRtWarps = 8;  // warps per block
constexpr int kRtCB = 64;    // columns per block

// A value of the 24-bit store: an FP32 number with its significand rounded
// to 16 bits (round half away from zero on the dropped byte), kept as its top
// two bytes and its third byte.  A group of 32 is 96 bytes: the 32 top halves
// (64 B), then the 32 third bytes (32 B).
struct F24 {};

__host__ __device__ inline uint32_t f24_bits(float f) {  // the 24 kept bits, right-aligned
  uint32_t b;
  memcpy(&b, &f, 4);
  return (b + 0x80u) >> 8;
}

// Per store: the history's type, the bytes of a group of 32 values, and a
// lane's read position in a staged group (at: the group's first byte; get:
// this lane's value; next: the following group).
template <typename Coef>
struct RtPrec;
template <>
struct RtPrec<float> {  // FP32 store: FP32 history, FP32 column sums
  using Hist = float;
  static constexpr int kGroupBytes = 128;
  struct Cur {
    const float* p;
    __device__ void at(const unsigned char* g, int lane) { p = reinterpret_cast<const float*>(g) + lane; }
    __device__ float get() const { return *p; }
    __device__ void next() { p += 32; }
  };
};
template <>
struct RtPrec<F24> {  // 24-bit store: as FP32 after the load
  using Hist = float;
  static constexpr int kGroupBytes = 96;
  struct Cur {
    const uint16_t* h;
    const uint8_t* l;
    __device__ void at(const unsigned char* g, int lane) {
      h = reinterpret_cast<const uint16_t*>(g) + lane;
      l = g + 64 + lane;
    }
    // bytes (top half, third byte, 0): x = third byte (bytes 1..3 zero), y = top half
    __device__ float get() const { return __uint_as_float(__byte_perm((uint32_t)*l, (uint32_t)*h, 0x5401)); }
    __device__ void next() {
      h += 48;
      l += 96;
    }
  };
};
template <>
struct RtPrec<float2> {  // (hi, lo) store: double-float throughout
  using Hist = float2;
  static constexpr int kGroupBytes = 256;
  struct Cur {
    const float2* p;
    __device__ void at(const unsigned char* g, int lane) { p = reinterpret_cast<const float2*>(g) + lane; }
    __device__ float2 get() const { return *p; }
    __device__ void next() { p += 32; }
  };
};

// shared memory of a block: NS stages of SB bytes and an mbarrier per stage
// and warp, and the history of kRtCB columns x Lh lags
template <typename Coef>
size_t rt_smem_bytes(int ns, int sb, int Lh) {
  return (size_t)kRtWarps * ns * (sb + 8) + (size_t)kRtCB * Lh * sizeof(typename RtPrec<Coef>::Hist);
}

// coefficient z (FP32) times history x (double-float) added to (sh, sl)
__device__ __forceinline__ void df_fma_acc(float& sh, float& sl, float z, float2 x) {
  const float p = __fmul_rn(z, x.x);
  float e = __fmaf_rn(z, x.x, -p);
  e = __fmaf_rn(z, x.y, e);
  const float s = __fadd_rn(sh, p);
  const float bb = __fsub_rn(s, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(err, e));
}

__device__ __forceinline__ void rt_hist(float* o, double v) { *o = __double2float_rn(v); }
__device__ __forceinline__ void rt_hist(float2* o, double v) { *o = df_split(v); }

// NS stages of SB bytes per warp; MINB blocks per SM
template <typename Coef, int NS, int SB, int MINB>
__global__ void __launch_bounds__(kRtWarps * 32, MINB)
    k_direct_history_rt(const unsigned char* __restrict__ val, const uint32_t* __restrict__ goff,
                        const uint8_t* __restrict__ lo3, int64_t ne, int32_t nrt, const double* __restrict__ ring,
                        int32_t L, int32_t Lh, int32_t alpha, int32_t m_min, int32_t tiles,
                        double* __restrict__ partial, int32_t* err) {
  using Hist = typename RtPrec<Coef>::Hist;
  constexpr int GB = RtPrec<Coef>::kGroupBytes;
  constexpr int CG = SB / GB;  // groups per stage
  static_assert(CG * GB == SB && SB % 16 == 0, "a stage holds whole groups and 16-byte copies");
  constexpr bool kF32 = !std::is_same<Coef, float2>::value;  // FP32 arithmetic (FP32 and 24-bit stores)
  extern __shared__ __align__(128) unsigned char rt_sm[];
  unsigned char* stages = rt_sm;  // [kRtWarps][NS][SB]
  uint64_t* bars = reinterpret_cast<uint64_t*>(rt_sm + (size_t)kRtWarps * NS * SB);
  Hist* hist = reinterpret_cast<Hist*>(bars + kRtWarps * NS);  // [kRtCB][Lh]
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t j0 = (int64_t)blockIdx.x * kRtCB;
  const int ncol = (int)min((int64_t)kRtCB, ne - j0);
  const int rt_begin = blockIdx.y * tiles, rt_end = min(nrt, rt_begin + tiles);
  const uint32_t bar0 = tc::smem_u32(bars + w * NS);
  unsigned char* wst = stages + (size_t)w * NS * SB;
  if (lane == 0) {
    for (int s = 0; s < NS; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8 * s));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  // producer cursor of this warp's stretches (every lane keeps it; lane 0 copies)
  int p_rt = rt_begin + w;
  uint32_t p_g = 0, p_ge = 0, issued = 0;
  if (p_rt < rt_end) {
    p_g = goff[(int64_t)p_rt * ne + j0];
    p_ge = goff[(int64_t)p_rt * ne + j0 + ncol];
  }
  auto issue = [&](int s) {  // the cursor's next chunk into stage s (none once the warp's tiles are done)
    while (p_rt < rt_end && p_g == p_ge) {
      p_rt += kRtWarps;
      if (p_rt < rt_end) {
        p_g = goff[(int64_t)p_rt * ne + j0];
        p_ge = goff[(int64_t)p_rt * ne + j0 + ncol];
      }
    }
    if (p_rt >= rt_end) return;
    const uint32_t n = min((uint32_t)CG, p_ge - p_g);
    if (lane == 0) {  // every lane's reads of the stage have returned (their values were used)
      const uint32_t bytes = n * (uint32_t)GB;
      tc::mbar_expect_tx(bar0 + 8 * s, bytes);
      tc::bulk_g2s(tc::smem_u32(wst + (size_t)s * SB), val + (size_t)p_g * GB, bytes, bar0 + 8 * s);
    }
    p_g += n;
    ++issued;
  };
  for (int s = 0; s < NS; ++s) issue(s);
  // the block's history, while the first copies are in flight
  for (int k = threadIdx.x; k < kRtCB * Lh; k += blockDim.x) {
    const int c = k / Lh, m = k - c * Lh;
    const bool on = c < ncol && m >= m_min && m <= alpha && m < L;
    rt_hist(hist + k, on ? ring[(j0 + c) * L + ((alpha - m) & (L - 1))] : 0.0);
  }
  __syncthreads();
  double* out = partial + (int64_t)blockIdx.x * ne;
  uint32_t q = 0;  // chunks taken
  bool failed = false;
  typename RtPrec<Coef>::Cur zc;
  zc.at(wst, lane);
  // per column its first lag (this lane's row) and its end group, loaded five
  // columns ahead over the warp's sequence of (tile, column)
  int pf_rt = rt_begin + w, pf_c = 0;
  auto meta = [&](int& l, uint32_t& e) {
    l = 0;
    e = 0;
    if (pf_rt < rt_end) {
      const int64_t m = (int64_t)pf_rt * ne + j0 + pf_c;
      l = lo3[m * 32 + lane];
      e = goff[m + 1];
      if (++pf_c == ncol) {
        pf_c = 0;
        pf_rt += kRtWarps;
      }
    }
  };
  int l0, l1, l2, l3, l4;
  uint32_t e0, e1, e2, e3, e4;
  meta(l0, e0);
  meta(l1, e1);
  meta(l2, e2);
  meta(l3, e3);
  meta(l4, e4);
  // the range of the warp's next tile, loaded a tile ahead
  uint32_t nx_g = 0, nx_end = 0;
  if (rt_begin + w < rt_end) {
    nx_g = goff[(int64_t)(rt_begin + w) * ne + j0];
    nx_end = goff[(int64_t)(rt_begin + w) * ne + j0 + ncol];
  }
  for (int rt = rt_begin + w; rt < rt_end; rt += kRtWarps) {
    uint32_t g = nx_g;
    const uint32_t gend = nx_end;
    if (rt + kRtWarps < rt_end) {
      nx_g = goff[(int64_t)(rt + kRtWarps) * ne + j0];
      nx_end = goff[(int64_t)(rt + kRtWarps) * ne + j0 + ncol];
    }
    uint32_t cend = g;  // end of the chunk held (none yet in this tile)
    float sh = 0.f, sl = 0.f;
    for (int c = 0; c < ncol && !failed; ++c) {
      const int lo = l0;
      const uint32_t ge = e0;
      l0 = l1;
      e0 = e1;
      l1 = l2;
      e1 = e2;
      l2 = l3;
      e2 = e3;
      l3 = l4;
      e3 = e4;
      meta(l4, e4);
      const Hist* h = hist + c * Lh + lo;
      float a = 0.f;  // FP32 arithmetic: the column's sum
      while (g < ge) {
        if (g == cend) {
          if (q > 0) {
            __syncwarp();
            issue((int)((q - 1) % NS));  // chunk q - 1 is consumed: its stage takes the next
          }
          const bool ok = tc::mbar_wait(bar0 + 8 * (q % NS), (q / NS) & 1);
          if (__any_sync(0xffffffffu, !ok)) {
            failed = true;
            break;
          }
          zc.at(wst + (size_t)(q % NS) * SB, lane);
          cend = min(g + (uint32_t)CG, gend);
          ++q;
        }
        const uint32_t gs = min(ge, cend);
        if constexpr (kF32) {
#pragma unroll 4
          for (; g < gs; ++g, ++h, zc.next()) a = __fmaf_rn(zc.get(), *h, a);
        } else {
#pragma unroll 4
          for (; g < gs; ++g, ++h, zc.next()) df_fma_acc(sh, sl, zc.get(), *h);
        }
      }
      if constexpr (kF32) df_add(sh, sl, a, 0.f);
    }
    const int64_t i = (int64_t)rt * 32 + lane;
    if (i < ne) out[i] = failed ? __longlong_as_double(0x7ff8000000000000LL) : (double)sh + (double)sl;
  }
  if (failed) {
    if (lane == 0) atomicExch(err, 1);
    for (uint32_t k = q; k < issued; ++k) tc::mbar_wait(bar0 + 8 * (k % NS), (k / NS) & 1);
  }
}

// Row-tile store, step 1: one warp per (tile, column), lane t row 32 rt + t.
// nmax[rt * ne + j] = the tile's largest count of stored lags >= 3 of column j;
// lo3[(rt * ne + j) * 32 + t] = the row's first lag >= 3 (3 where it has none);
// *lh = max over everything of lo3 + nmax (history rows the kernel reads).
__global__ void k_rt_meta(const int16_t* m_lo, const uint8_t* nlag, int64_t ne, int32_t nrt, uint8_t* nmax,
                          uint8_t* lo3, int32_t* lh) {
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= (int64_t)nrt * ne) return;  // whole warps
  const int64_t rt = wid / ne, j = wid - rt * ne, i = rt * 32 + lane;
  int n3 = 0, l3 = 3;
  if (i < ne) {
    const int lo = m_lo[i * ne + j], hi = lo + nlag[i * ne + j];  // lags lo .. hi - 1
    l3 = max(lo, 3);
    n3 = max(0, hi - l3);
    if (n3 == 0) l3 = 3;
  }
  int mx = n3;
  for (int d = 16; d > 0; d >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, d));
  int need = l3 + mx;
  for (int d = 16; d > 0; d >>= 1) need = max(need, __shfl_xor_sync(0xffffffffu, need, d));
  lo3[wid * 32 + lane] = (uint8_t)l3;
  if (lane == 0) {
    nmax[wid] = (uint8_t)mx;
    atomicMax(lh, need);
  }
}

// value v at lane t of the group starting at byte g
__device__ __forceinline__ void rt_put(float, unsigned char* g, int t, double v) {
  reinterpret_cast<float*>(g)[t] = __double2float_rn(v);
}
__device__ __forceinline__ void rt_put(float2, unsigned char* g, int t, double v) {
  reinterpret_cast<float2*>(g)[t] = df_split(v);
}
__device__ __forceinline__ void rt_put(F24, unsigned char* g, int t, double v) {
  const uint32_t b = f24_bits(__double2float_rn(v));
  reinterpret_cast<uint16_t*>(g)[t] = (uint16_t)(b >> 8);
  g[64 + t] = (uint8_t)(b & 0xffu);
}

// Row-tile store, step 2: the groups of (tile, column), zero past each row's window.
template <typename Coef>
__global__ void k_rt_fill(const int16_t* m_lo, const uint8_t* nlag, const int64_t* off, const double* val,
                          int64_t ne, int32_t nrt, const uint32_t* goff, const uint8_t* lo3, unsigned char* out) {
  const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= (int64_t)nrt * ne) return;
  const int64_t rt = wid / ne, j = wid - rt * ne, i = rt * 32 + lane;
  const uint32_t g0 = goff[wid], nm = goff[wid + 1] - g0;
  int n3 = 0;
  int64_t src = 0;
  if (i < ne) {
    const int lo = m_lo[i * ne + j], l3 = lo3[wid * 32 + lane];
    n3 = max(0, lo + (int)nlag[i * ne + j] - max(lo, 3));
    src = off[i * ne + j] + (l3 - lo);
  }
  for (uint32_t u = 0; u < nm; ++u)
    rt_put(Coef{}, out + ((size_t)g0 + u) * RtPrec<Coef>::kGroupBytes, lane, (int)u < n3 ? val[src + u] : 0.0);
}

// Lag-2 entries of the direct store, as a CSR over rows (before the split).
__global__ void k_lag2_count(const int16_t* m_lo, const uint8_t* nlag, int64_t ne, int64_t* cnt) {
  const int64_t i = blockIdx.x;
  int64_t s = 0;
  for (int64_t j = threadIdx.x; j < ne; j += blockDim.x) {
    const int lo = m_lo[i * ne + j], n = nlag[i * ne + j];
    s += (lo <= 2 && 2 < lo + n) ? 1 : 0;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ int64_t red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    cnt[i] = t;
  }
}

// one thread per row: its lag-2 entries in column order
__global__ void k_lag2_fill(const int16_t* m_lo, const uint8_t* nlag, const int64_t* off, const double* val, int64_t ne,
                            const int64_t* ptr, int32_t* col, double* v) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= ne) return;
  int64_t e = ptr[i];
  const int64_t e1 = ptr[i + 1];
  for (int64_t j = 0; j < ne && e < e1; ++j) {
    const int64_t p = i * ne + j;
    const int lo = m_lo[p], n = nlag[p];
    if (lo <= 2 && 2 < lo + n) {
      col[e] = (int32_t)j;
      v[e] = val[off[p] + (2 - lo)];
      ++e;
    }
  }
}

// Batched form of k_direct_history for R right-hand sides ([..][ne][R]
// layouts): one block per row; the block's threads are split into groups of
// RL lanes (RL = R rounded up to a power of two, at most 32), lane rr of a
// group takes the right-hand sides rr, rr+RL, ... and the groups take
// interleaved columns j, so each coefficient is read once per group and
// broadcast to its lanes while the history vectors are read contiguously.
__global__ void __launch_bounds__(256) k_direct_history_multi(const int16_t* m_lo, const uint8_t* nlag,
                                                             const int64_t* off, const double* val, int64_t ne,
                                                             const double* ring, int32_t L, int32_t alpha,
                                                             int32_t R, int32_t RL, const double* V, double* Rout) {
  __shared__ double red[8][32];
  const int64_t i = blockIdx.x;
  const int rr = threadIdx.x % RL, sub = threadIdx.x / RL, nsub = blockDim.x / RL;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int r0 = 0; r0 < R; r0 += RL) {
    const int r = r0 + rr;
    double s = 0.0;
    if (r < R) {
      for (int64_t j = sub; j < ne; j += nsub) {
        int64_t p = i * ne + j;
        int lo = m_lo[p], n = nlag[p];
        const double* z = val + off[p];
        const double* Jr = ring + j * L * R + r;
        for (int w = 0; w < n; ++w) {
          int m = lo + w;
          int b = alpha - m;
          if (m < 2 || b < 0) continue;
          s += __ldg(z + w) * Jr[(int64_t)(b & (L - 1)) * R];
        }
      }
    }
    // lanes rr, rr+RL, ... of a warp hold partial sums of the same r
    for (int o = 16; o >= RL; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane < RL) red[warp][lane] = s;
    __syncthreads();
    if (threadIdx.x < RL && r0 + threadIdx.x < R) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w][threadIdx.x];
      int64_t q = i * R + r0 + threadIdx.x;
      Rout[q] = (V ? V[q] : 0.0) - t;
    }
    __syncthreads();
  }
}

}  // namespace tdbem

using namespace tdbem;

tdbem_status tdbem_build_direct(tdbem_ctx* c) {
  const int64_t ne = c->ne, npair = ne * ne;
  PairStore& st = c->direct;
  st.npairs = npair;
  tdbem_status s;
  int32_t* d_err = nullptr;
  if ((s = c->dalloc(&st.m_lo, npair)) || (s = c->dalloc(&st.nlag, npair)) || (s = c->dalloc(&st.off, npair)) ||
      (s = c->dalloc(&d_err, 1)))
    return s;
  TDBEM_CUDA_TRY(c, cudaMemsetAsync(d_err, 0, sizeof(int32_t), c->stream));
  k_direct_windows<<<(unsigned)((npair + 255) / 256), 256, 0, c->stream>>>(c->tg, c->d_et, ne, c->phys.a, st.m_lo,
                                                                           st.nlag, d_err);
  TDBEM_CUDA_TRY(c, cudaGetLastError());
  int64_t* d_tot = nullptr;
  int64_t* d_base = nullptr;
  if ((s = c->dalloc(&d_tot, ne)) || (s = c->dalloc(&d_base, ne))) return s;
  k_row_totals<<<(unsigned)ne, 256, 0, c->stream>>>(st.nlag, ne, d_tot);
  std::vector<int64_t> tot(ne), base(ne);
  TDBEM_CUDA_TRY(c, cudaMemcpyAsync(tot.data(), d_tot, ne * sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
  int32_t herr = 0;
  TDBEM_CUDA_TRY(c, cudaMemcpyAsync(&herr, d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
  TDBEM_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (herr) {
    c->set_error("direct: lag window out of range (mesh too large relative to c*dt)");
    return TDBEM_EINVAL;
  }
  int64_t acc = 0;
  for (int64_t i = 0; i < ne; ++i) {
    base[i] = acc;
    acc += tot[i];
  }
  st.nval = acc;
  TDBEM_CUDA_TRY(c, cudaMemcpyAsync(d_base, base.data(), ne * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
  k_row_offsets<<<(unsigned)ne, 1024, 0, c->stream>>>(st.nlag, ne, d_base, st.off);
  if ((s = c->dalloc(&st.val, st.nval))) return s;
  TDBEM_CUDA_TRY(c, cudaMemsetAsync(st.val, 0, st.nval * sizeof(double), c->stream));
  // four slots per stored coefficient for the order-independent sum, if the
  // device (and the context's budget) has room; else FP64 atomics
  double* val4 = nullptr;
  const size_t b4 = (size_t)4 * st.nval * sizeof(double);
  const bool fits = c->p.max_device_bytes <= 0 || c->device_bytes + (int64_t)b4 <= c->p.max_device_bytes;
  if (fits && cudaMalloc(&val4, b4) != cudaSuccess) {
    val4 = nullptr;
    cudaGetLastError();  // clear the failed allocation
  }
  if (val4) TDBEM_CUDA_TRY(c, cudaMemsetAsync(val4, 0, b4, c->stream));
  DirectSink sink{st.m_lo, st.nlag, st.off, st.val, ne, val4};
  const int64_t ntp = c->nt * c->nt;
  k_assemble<DirectSink><<<(unsigned)((ntp + 127) / 128), 128, 0, c->stream>>>(c->tg, c->phys, c->nt, nullptr, ntp,
                                                                               sink, d_err);
  TDBEM_CUDA_TRY(c, cudaGetLastError());
  if (val4) {
    k_sum4<<<(unsigned)((st.nval + 255) / 256), 256, 0, c->stream>>>(val4, st.nval, st.val);
    cudaError_t e4 = cudaGetLastError();
    cudaStreamSynchronize(c->stream);
    cudaFree(val4);
    TDBEM_CUDA_TRY(c, e4);
  }
  TDBEM_CUDA_TRY(c, cudaMemcpyAsync(&herr, d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
  TDBEM_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (herr) {
    c->set_error("direct: assembly failed (lag window or light-cone pieces exceed the local buffers), code " +
                 std::to_string(herr));
    return TDBEM_EINVAL;
  }
  // largest stored lag (the history ring holds every step it reaches)
  int32_t mx = 0;
  {
    int32_t* d_mx = nullptr;
    if ((s = c->dalloc(&d_mx, 1))) return s;
    TDBEM_CUDA_TRY(c, cudaMemsetAsync(d_mx, 0, sizeof(int32_t), c->stream));
    k_max_lag<<<1024, 256, 0, c->stream>>>(st.m_lo, st.nlag, npair, d_mx);
    TDBEM_CUDA_TRY(c, cudaGetLastError());
    TDBEM_CUDA_TRY(c, cudaMemcpyAsync(&mx, d_mx, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    TDBEM_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  }
  c->max_lag = mx;
  return TDBEM_OK;
}

// Incident field of right-hand side r at every step into column r of the
// table (the other columns are kept; a column never set stays zero).
tdbem_status tdbem_incident_table(tdbem_ctx* c, int32_t r) {
  const int64_t ne = c->ne;
  const int64_t n = (int64_t)(c->Nt - 1) * ne * c->R;
  tdbem_status s;
  if (!c->d_Vtab) {
    if ((s = c->dalloc(&c->d_Vtab, n))) return s;
    TDBEM_CUDA_TRY(c, cudaMemsetAsync(c->d_Vtab, 0, n * sizeof(double), c->stream));
  }
  const int32_t chunk = 1024;  // steps per launch (grid.y limit)
  for (int32_t a0 = 1; a0 <= c->Nt - 1; a0 += chunk) {
    int32_t na = std::min(chunk, c->Nt - a0);
    dim3 grid((unsigned)((ne + 127) / 128), (unsigned)na);
    k_rhs_plane<<<grid, 128, 0, c->stream>>>(c->tg, c->phys, c->d_et, ne, c->d_pulse + 10 * r, a0, c->R, r,
                                              c->d_Vtab + (int64_t)(a0 - 1) * ne * c->R);
    TDBEM_CUDA_TRY(c, cudaGetLastError());
  }
  return TDBEM_OK;
}

const double* tdbem_incident_row(const tdbem_ctx* c, int32_t alpha) {
  const int64_t stride = c->ne * (int64_t)c->R;
  if (c->d_Vall) return c->d_Vall + (int64_t)(alpha - 1) * stride;
  if (c->have_pulse && c->d_Vtab) return c->d_Vtab + (int64_t)(alpha - 1) * stride;
  return nullptr;
}

// Row-tile kernel shapes (stages x stage bytes, blocks per SM).  The (hi, lo)
// store needs twice the history in shared memory and twice the stage time
// per byte: four 2 KB stages at two blocks per SM.  The FP32 store is bound
// by how many warps keep copies in flight: three 2 KB stages at three blocks
// per SM (on the 7680-RWG sphere 0.41 ms per launch alone, against 0.47 with
// five stages at two blocks and 0.49 to 0.51 with 1 KB stages).
struct RtShape {
  int ns, sb;
};
constexpr RtShape kRtShape2 = {4, 2048}, kRtShape1 = {3, 2048}, kRtShape3 = {3, 2304};
using RtFn = void (*)(const unsigned char*, const uint32_t*, const uint8_t*, int64_t, int32_t, const double*,
                      int32_t, int32_t, int32_t, int32_t, int32_t, double*, int32_t*);
// rt_prec 1: FP32 store, 2: (hi, lo) pairs, 3: 24-bit store
static RtFn rt_fn(int prec) {
  if (prec == 1) return k_direct_history_rt<float, kRtShape1.ns, kRtShape1.sb, 3>;
  if (prec == 3) return k_direct_history_rt<F24, kRtShape3.ns, kRtShape3.sb, 3>;
  return k_direct_history_rt<float2, kRtShape2.ns, kRtShape2.sb, 2>;
}
static int rt_group_bytes(int prec) {
  return prec == 1 ? RtPrec<float>::kGroupBytes : prec == 3 ? RtPrec<F24>::kGroupBytes : RtPrec<float2>::kGroupBytes;
}
static size_t rt_smem(const tdbem_ctx* c) {
  if (c->rt_prec == 1) return rt_smem_bytes<float>(kRtShape1.ns, kRtShape1.sb, c->rt_Lh);
  if (c->rt_prec == 3) return rt_smem_bytes<F24>(kRtShape3.ns, kRtShape3.sb, c->rt_Lh);
  return rt_smem_bytes<float2>(kRtShape2.ns, kRtShape2.sb, c->rt_Lh);
}

// partial sums per row of the tiled history sum
static int64_t direct_nparts(const tdbem_ctx* c) {
  return c->rt_ncb;
}

// The tiled history sum of the lags >= 3 of step alpha into partial buffer buf,
// on the context's current stream.
static tdbem_status direct_tile(tdbem_ctx* c, int32_t alpha, const double* d_ring, int buf) {
  const int64_t nrt = (c->ne + 31) / 32;
  const dim3 grid((unsigned)c->rt_ncb, (unsigned)c->rt_nrg);
  const size_t smem = rt_smem(c);
  double* part = c->d_dpart + buf * direct_nparts(c) * c->ne;
  rt_fn(c->rt_prec)<<<grid, kRtWarps * 32, smem, c->stream>>>(c->d_rt_val, c->d_rt_goff, c->d_rt_lo, c->ne,
                                                                (int32_t)nrt, d_ring, c->L, c->rt_Lh, alpha, 3,
                                                                c->rt_tiles, part, c->d_dt_err);
  TDBEM_CUDA_TRY(c, cudaGetLastError());
  return TDBEM_OK;
}

tdbem_status tdbem_direct_history(tdbem_ctx* c, int32_t alpha, const double* d_ring, const double* V) {
  const PairStore& st = c->direct;
  if (c->R == 1 && c->rt_prec) {
    // the march's own ring uses buffers alpha & 1 (possibly filled ahead, during
    // the previous step), any other history buffer 2
    const bool march = d_ring == c->d_Jring;
    const int buf = march ? (alpha & 1) : 2;
    const int64_t nparts = direct_nparts(c);
    if (march && c->dahead[buf] == alpha) {
      TDBEM_CUDA_TRY(c, cudaStreamWaitEvent(c->stream, c->ev_dahead[buf], 0));
    } else {
      cudaEvent_t e = c->prof_begin(1);
      tdbem_status s = direct_tile(c, alpha, d_ring, buf);
      if (s) return s;
      c->prof_end(1, e);
    }
    if (march) c->dahead[buf] = 0;
    cudaEvent_t e = c->prof_begin(10);
    k_direct_reduce<<<(unsigned)((c->ne * kRedLanes + 255) / 256), 256, 0, c->stream>>>(
        c->d_dpart + buf * nparts * c->ne, (int32_t)nparts, c->ne, c->d_l2_ptr, c->d_l2_col, c->d_l2_val, d_ring,
        c->L, alpha, V, c->d_R);
    c->prof_end(10, e);
  } else if (c->R == 1) {
    if (!c->d_ring2 || !st.val) {
      c->set_error("direct: untiled history sum without its split ring");
      return TDBEM_ESTATE;
    }
    cudaEvent_t e = c->prof_begin(9);
    const int64_t n = c->ne * (int64_t)c->L;
    k_ring_split<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(d_ring, c->ne, c->L, c->d_ring2);
    c->prof_end(9, e);
    TDBEM_CUDA_TRY(c, cudaGetLastError());
    e = c->prof_begin(1);
    k_direct_history<<<(unsigned)c->ne, kDhThreads, 2 * kDhCap * sizeof(float2), c->stream>>>(
        st.m_lo, st.nlag, st.off, reinterpret_cast<const float2*>(st.val), c->ne, c->d_ring2, c->L, alpha, V, c->d_R);
    c->prof_end(1, e);
  } else {
    int RL = 1;
    while (RL < c->R && RL < 32) RL <<= 1;
    cudaEvent_t e = c->prof_begin(1);
    k_direct_history_multi<<<(unsigned)c->ne, 256, 0, c->stream>>>(st.m_lo, st.nlag, st.off, st.val, c->ne, d_ring,
                                                                   c->L, alpha, c->R, RL, V, c->d_R);
    c->prof_end(1, e);
  }
  TDBEM_CUDA_TRY(c, cudaGetLastError());
  return TDBEM_OK;
}

// After step alpha's solve is enqueued: the lags >= 3 of step alpha + 2 need
// the currents up to J^{alpha-1}, so they are summed on the side stream while
// step alpha + 1 runs (its reduction, lag-2 entries and solve).  Buffer
// (alpha + 2) & 1 was last read by step alpha's reduction, ordered before the
// solve and so before this launch.
tdbem_status tdbem_direct_after_solve(tdbem_ctx* c, int32_t alpha) {
  if (!c->dstream || !c->rt_prec || c->R != 1) return TDBEM_OK;
  const int32_t a2 = alpha + 2;
  if (a2 > c->Nt - 1) return TDBEM_OK;
  const int b = a2 & 1;
  TDBEM_CUDA_TRY(c, cudaEventRecord(c->ev_dsolved, c->stream));
  TDBEM_CUDA_TRY(c, cudaStreamWaitEvent(c->dstream, c->ev_dsolved, 0));
  cudaStream_t main = c->stream;
  c->stream = c->dstream;
  cudaEvent_t e = c->prof_begin(1);
  tdbem_status s = direct_tile(c, a2, c->d_Jring, b);
  c->prof_end(1, e);
  c->stream = main;
  if (s) return s;
  TDBEM_CUDA_TRY(c, cudaEventRecord(c->ev_dahead[b], c->dstream));
  c->dahead[b] = a2;
  return TDBEM_OK;
}

// ETIMEOUT if a bounded wait of the row-tile history sum expired (its partial
// sums are NaN then, so the step's solve also misses its tolerance).
tdbem_status tdbem_direct_check(tdbem_ctx* c) {
  if (!c->d_dt_err) return TDBEM_OK;
  tdbem_status s = tdbem_direct_join(c);
  if (s) return s;
  int32_t h = 0;
  TDBEM_CUDA_TRY(c, cudaMemcpyAsync(&h, c->d_dt_err, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
  TDBEM_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (h) {
    c->set_error("direct: a bounded wait of the history sum expired");
    return TDBEM_ETIMEOUT;
  }
  return TDBEM_OK;
}

// The context's stream waits for the sums launched ahead (they stay usable).
tdbem_status tdbem_direct_join(tdbem_ctx* c) {
  for (int b = 0; b < 2; ++b)
    if (c->dahead[b]) TDBEM_CUDA_TRY(c, cudaStreamWaitEvent(c->stream, c->ev_dahead[b], 0));
  return TDBEM_OK;
}

// As tdbem_direct_join, and the sums launched ahead are discarded.
tdbem_status tdbem_direct_invalidate(tdbem_ctx* c) {
  tdbem_status s = tdbem_direct_join(c);
  c->dahead[0] = c->dahead[1] = 0;
  return s;
}

void tdbem_direct_free(tdbem_ctx* c) {
  if (c->dstream) cudaStreamSynchronize(c->dstream);
  if (c->ev_dsolved) cudaEventDestroy(c->ev_dsolved);
  for (int b = 0; b < 2; ++b)
    if (c->ev_dahead[b]) cudaEventDestroy(c->ev_dahead[b]);
  if (c->dstream) cudaStreamDestroy(c->dstream);
  c->dstream = nullptr;
}

// Builds the row-tile store of the lags >= 3 from the FP64 store (prec 1: FP32
// values, 2: (hi, lo) pairs, 3: 24-bit values), frees the FP64 values and sets
// the grid.
static tdbem_status build_row_tiles(tdbem_ctx* c, int prec) {
  PairStore& st = c->direct;
  const int64_t ne = c->ne, nrt = (ne + 31) / 32, ntc = nrt * ne;
  tdbem_status s;
  uint8_t* d_nmax = nullptr;
  int32_t* d_lh = nullptr;
  if ((s = c->dalloc(&d_nmax, ntc)) || (s = c->dalloc(&c->d_rt_lo, ntc * 32)) || (s = c->dalloc(&d_lh, 1)) ||
      (s = c->dalloc(&c->d_dt_err, 1)))
    return s;
  TDBEM_CUDA_TRY(c, cudaMemsetAsync(d_lh, 0, sizeof(int32_t), c->stream));
  TDBEM_CUDA_TRY(c, cudaMemsetAsync(c->d_dt_err, 0, sizeof(int32_t), c->stream));
  const unsigned nb = (unsigned)((ntc * 32 + 255) / 256);
  k_rt_meta<<<nb, 256, 0, c->stream>>>(st.m_lo, st.nlag, ne, (int32_t)nrt, d_nmax, c->d_rt_lo, d_lh);
  TDBEM_CUDA_TRY(c, cudaGetLastError());
  std::vector<uint8_t> nmax(ntc);
  int32_t lh = 0;
  TDBEM_CUDA_TRY(c, cudaMemcpyAsync(nmax.data(), d_nmax, ntc, cudaMemcpyDeviceToHost, c->stream));
  TDBEM_CUDA_TRY(c, cudaMemcpyAsync(&lh, d_lh, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
  TDBEM_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->dfree(d_nmax);
  c->dfree(d_lh);
  std::vector<uint32_t> goff(ntc + 1);
  uint64_t acc = 0;
  for (int64_t k = 0; k < ntc; ++k) {
    goff[k] = (uint32_t)acc;
    acc += nmax[k];
  }
  if (acc >= (1ull << 32) || lh > 255) {
    c->set_error("direct: row-tile store too large (32-bit group offsets, 8-bit first lags)");
    return TDBEM_EINVAL;
  }
  goff[ntc] = (uint32_t)acc;
  if ((s = c->dalloc(&c->d_rt_goff, ntc + 1))) return s;
  TDBEM_CUDA_TRY(c, cudaMemcpyAsync(c->d_rt_goff, goff.data(), (ntc + 1) * sizeof(uint32_t), cudaMemcpyHostToDevice,
                                    c->stream));
  const size_t nbytes = (size_t)acc * rt_group_bytes(prec);
  unsigned char* v = nullptr;
  if ((s = c->dalloc(&v, nbytes))) return s;
  if (prec == 1)
    k_rt_fill<float><<<nb, 256, 0, c->stream>>>(st.m_lo, st.nlag, st.off, st.val, ne, (int32_t)nrt, c->d_rt_goff,
                                                c->d_rt_lo, v);
  else if (prec == 3)
    k_rt_fill<F24><<<nb, 256, 0, c->stream>>>(st.m_lo, st.nlag, st.off, st.val, ne, (int32_t)nrt, c->d_rt_goff,
                                              c->d_rt_lo, v);
  else
    k_rt_fill<float2><<<nb, 256, 0, c->stream>>>(st.m_lo, st.nlag, st.off, st.val, ne, (int32_t)nrt, c->d_rt_goff,
                                                 c->d_rt_lo, v);
  c->d_rt_val = v;
  TDBEM_CUDA_TRY(c, cudaGetLastError());
  // the goff vector (host) and the FP64 values are read by the fill: wait before both go
  TDBEM_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  c->dfree(st.val);
  st.val = nullptr;
  c->rt_Lh = std::max(lh, 4);
  c->rt_prec = prec;
  c->rt_bytes = (int64_t)nbytes + ntc * 32 + (ntc + 1) * 4;
  const size_t smem = rt_smem(c);
  int nsm = 0, per_sm = 0;
  TDBEM_CUDA_TRY(c, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device));
  TDBEM_CUDA_TRY(c, cudaFuncSetAttribute(rt_fn(prec), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  TDBEM_CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rt_fn(prec), kRtWarps * 32, smem));
  const int64_t slots = (int64_t)std::max(1, per_sm) * nsm;
  const int ncb = (int)((ne + kRtCB - 1) / kRtCB);
  // row-tile groups: the fewest waves of blocks times the tiles a warp takes
  // per block (a small charge per block for its history staging)
  double best = 1e300;
  int tiles_best = (int)nrt;
  for (int64_t nrg = 1; nrg <= nrt; ++nrg) {
    const int64_t tiles = (nrt + nrg - 1) / nrg, groups = (nrt + tiles - 1) / tiles;
    const int64_t waves = (ncb * groups + slots - 1) / slots;
    const double cost = (double)waves * ((double)((tiles + kRtWarps - 1) / kRtWarps) + 0.25);
    if (cost < best - 1e-9) {
      best = cost;
      tiles_best = (int)tiles;
    }
  }
  c->rt_ncb = ncb;
  c->rt_tiles = tiles_best;
  c->rt_nrg = (int)((nrt + tiles_best - 1) / tiles_best);
  return TDBEM_OK;
}

// Single right-hand side, after Z0 and the lag-2 entries have been read from
// the FP64 store: the row-tile store of the lags >= 3 in the precision of
// p2p_prec (ring length L <= 128), which replaces the FP64 values; else the
// FP64 values split in place into (hi, lo) pairs for the untiled kernel and
// its split ring.
tdbem_status tdbem_direct_split(tdbem_ctx* c) {
  if (c->R != 1) return TDBEM_OK;
  PairStore& st = c->direct;
  const bool tiled = c->L <= 128;  // the row-tile store's first lags are bytes, its history fits shared memory
  if (tiled) {
    // lag-2 entries (read from the FP64 store before the row tiles replace it)
    const int64_t ne = c->ne;
    int64_t* d_cnt = nullptr;
    tdbem_status s0;
    if ((s0 = c->dalloc(&c->d_l2_ptr, ne + 1)) || (s0 = c->dalloc(&d_cnt, ne))) return s0;
    k_lag2_count<<<(unsigned)ne, 256, 0, c->stream>>>(st.m_lo, st.nlag, ne, d_cnt);
    TDBEM_CUDA_TRY(c, cudaGetLastError());
    std::vector<int64_t> cnt(ne), ptr(ne + 1, 0);
    // the counts come from the context's stream: copy on it and wait
    TDBEM_CUDA_TRY(c, cudaMemcpyAsync(cnt.data(), d_cnt, ne * sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
    TDBEM_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    for (int64_t i = 0; i < ne; ++i) ptr[i + 1] = ptr[i] + cnt[i];
    TDBEM_CUDA_TRY(c, cudaMemcpyAsync(c->d_l2_ptr, ptr.data(), (ne + 1) * sizeof(int64_t), cudaMemcpyHostToDevice,
                                      c->stream));
    if ((s0 = c->dalloc(&c->d_l2_col, std::max<int64_t>(1, ptr[ne]))) ||
        (s0 = c->dalloc(&c->d_l2_val, std::max<int64_t>(1, ptr[ne]))))
      return s0;
    k_lag2_fill<<<(unsigned)((ne + 127) / 128), 128, 0, c->stream>>>(st.m_lo, st.nlag, st.off, st.val, ne,
                                                                      c->d_l2_ptr, c->d_l2_col, c->d_l2_val);
    TDBEM_CUDA_TRY(c, cudaGetLastError());
    TDBEM_CUDA_TRY(c, cudaStreamSynchronize(c->stream));  // before ptr (host) goes out of scope
  }
  if (!tiled && c->p.p2p_prec != TDBEM_P_FP64) {
    c->set_error("p2p_prec FP32 and FP24 need one right-hand side and a history ring of at most 128 steps");
    return TDBEM_EINVAL;
  }
  if (tiled) {
    tdbem_status s =
        build_row_tiles(c, c->p.p2p_prec == TDBEM_P_FP32 ? 1 : c->p.p2p_prec == TDBEM_P_FP24 ? 3 : 2);
    if (s) return s;
    if ((s = c->dalloc(&c->d_dpart, (size_t)3 * c->rt_ncb * c->ne))) return s;
    TDBEM_CUDA_TRY(c, cudaMemsetAsync(c->d_dpart, 0, (size_t)3 * c->rt_ncb * c->ne * sizeof(double), c->stream));
    if (c->p.far_overlap) {
      // between the library stream's highest priority and the lowest: the
      // next solve's cluster is dispatched ahead of this stream's blocks
      int prio_lo = 0, prio_hi = 0;
      TDBEM_CUDA_TRY(c, cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
      TDBEM_CUDA_TRY(c, cudaStreamCreateWithPriority(&c->dstream, cudaStreamNonBlocking, (prio_lo + prio_hi) / 2));
      TDBEM_CUDA_TRY(c, cudaEventCreateWithFlags(&c->ev_dsolved, cudaEventDisableTiming));
      for (int b = 0; b < 2; ++b) TDBEM_CUDA_TRY(c, cudaEventCreateWithFlags(&c->ev_dahead[b], cudaEventDisableTiming));
    }
    return TDBEM_OK;
  }
  k_split_values<<<(unsigned)((st.nval + 255) / 256), 256, 0, c->stream>>>(st.val, st.nval);
  TDBEM_CUDA_TRY(c, cudaGetLastError());
  TDBEM_CUDA_TRY(c, cudaFuncSetAttribute(k_direct_history, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(2 * kDhCap * sizeof(float2))));
  tdbem_status s = c->dalloc(&c->d_ring2, c->ne * (int64_t)c->L);
  if (s) return s;
  TDBEM_CUDA_TRY(c, cudaMemsetAsync(c->d_ring2, 0, c->ne * (int64_t)c->L * sizeof(float2), c->stream));
  return TDBEM_OK;
}

// Assemble the listed (test triangle, source triangle) pairs into a CSR store
// of edge pairs (the near field of fast mode).  row_ptr/col must already hold
// every edge pair touched by the listed triangle pairs.
tdbem_status tdbem_assemble_csr(tdbem_ctx* c, const int2* d_pairs, int64_t npairs, const int64_t* d_row_ptr,
                                const int32_t* d_col, int64_t nnz, int16_t** m_lo, uint8_t** nlag, int64_t** off,
                                double** val, int64_t* nval) {
  tdbem_status s;
  int32_t* d_err = nullptr;
  if ((s = c->dalloc(m_lo, nnz)) || (s = c->dalloc(nlag, nnz)) || (s = c->dalloc(off, nnz)) ||
      (s = c->dalloc(&d_err, 1)))
    return s;
  TDBEM_CUDA_TRY(c, cudaMemsetAsync(d_err, 0, sizeof(int32_t), c->stream));
  k_csr_windows<<<(unsigned)c->ne, 128, 0, c->stream>>>(c->tg, c->d_et, d_row_ptr, d_col, c->ne, c->phys.a, *m_lo,
                                                        *nlag, d_err);
  TDBEM_CUDA_TRY(c, cudaGetLastError());
  std::vector<uint8_t> hn(nnz);
  TDBEM_CUDA_TRY(c, cudaMemcpyAsync(hn.data(), *nlag, nnz, cudaMemcpyDeviceToHost, c->stream));
  TDBEM_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  std::vector<int64_t> ho(nnz);
  int64_t acc = 0;
  for (int64_t p = 0; p < nnz; ++p) {
    ho[p] = acc;
    acc += hn[p];
  }
  *nval = acc;
  TDBEM_CUDA_TRY(c, cudaMemcpyAsync(*off, ho.data(), nnz * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
  if ((s = c->dalloc(val, acc))) return s;
  TDBEM_CUDA_TRY(c, cudaMemsetAsync(*val, 0, acc * sizeof(double), c->stream));
  CsrSink sink{d_row_ptr, d_col, *m_lo, *nlag, *off, *val};
  if (npairs > 0) {
    k_assemble<CsrSink><<<(unsigned)((npairs + 127) / 128), 128, 0, c->stream>>>(c->tg, c->phys, c->nt, d_pairs,
                                                                                npairs, sink, d_err);
    TDBEM_CUDA_TRY(c, cudaGetLastError());
  }
  int32_t herr = 0;
  TDBEM_CUDA_TRY(c, cudaMemcpyAsync(&herr, d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
  TDBEM_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (herr) {
    c->set_error("near field: assembly failed, code " + std::to_string(herr));
    return TDBEM_EINVAL;
  }
  return TDBEM_OK;
}
