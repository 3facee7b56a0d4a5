/*
 * oracle.c -- plain FP64 CPU conventional marching-on-in-time TDBEM.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the
 * CUDA library is checked against.  Only the tests, the package smoke check
 * and the CPU-baseline leg of the benchmark may build, load or call it; the
 * product path never does.  It shares no code, header, table or helper with
 * the CUDA library.
 *
 * What it computes (paper section 2, "conventional TDBEM", specialised as in
 * section 3.6.3: near field at the root only, no far field):
 *
 *   * RWG space basis f_j (section 2.2): +-l_j/(2A_j^+-) (x - o_j^+-) on the
 *     two triangles of edge j, divergence +-l_j/A_j^+-.
 *   * Order-d B-spline time basis (section 2.2) written, as in the paper, as
 *     d+2 truncated powers: N(tau) = sum_k w^{k,d} (tau-k)_+^d with
 *     w^{k,d} = (d+1) / prod_{i != k} (i-k).  Its support is [0, d+1].
 *   * Galerkin testing (section 2.4, eqs. z_ij and v_i) of the CFIE built from
 *     the time-differentiated EFIE, the time-differentiated MFIE and the MFIE
 *     (eq. cfie).  The coefficient of J_j^beta in the tested equation at t_alpha
 *     depends on m = alpha - beta only (eq. layer_disc_tmp): with
 *     tau = m - r/(c dt),
 *       Zt^(m)_ij = sum_{rho,sigma} int_{S_i^rho} dS_x int_{S_j^sigma} dS_y [
 *           (mu/4pi) f_i(x).f_j(y) Nddot(tau)/(dt^2 r)                (A-term)
 *         + (1/(4 pi eps)) div f_i div f_j N(tau)/r                    (phi-term)
 *         + theta eta (1/4pi) f_i(x).( n(x) x ( f_j(y) x grad_y g ) ) ] (P-term)
 *       with g(r) = (chi Ndot(tau)/dt + zeta N(tau)) / r, chi the weight of the
 *       time-differentiated MFIE (1 in the paper's eq. cfie; 0 gives the
 *       paper's CFIE3 of section 4.3),
 *     which is the paper's sum_k w^{k,d} Z^(m-k) (eq. layer_disc_tmp with
 *     U^d of eq. U), since sum_k w^k (tau-k)_+^d = N(tau).
 *   * The identity term of the MFIE (reading of the paper's eq. cfie, see the
 *     module notes): + s_J theta eta (1/2) G_ij (chi Ndot(m)/dt + zeta N(m)),
 *     G_ij = int f_i.f_j, which is non-zero only for m = 1, 2.
 *   * Incident right-hand side V_i^{alpha-1} (eq. v_i).
 *   * Time stepping (eqs. solve and R): Zt^(1) J^{alpha-1} =
 *     V^{alpha-1} - sum_{m>=2} Zt^(m) J^{alpha-m}.  (The Python side factors
 *     Zt^(1) once with a library LU and marches.)
 *
 * Outer integral: 7-point degree-5 Radon rule on every test triangle.  Inner
 * integral: exact.  The y-integrals are functions of r = |x - y| only (times a
 * linear factor in y), so in polar coordinates about the projection p of x onto
 * the source plane (r dr = rho drho) the radial integral is a closed-form
 * antiderivative Phi(r), and the in-plane vector parts follow from the 2D
 * divergence theorem; both leave 1D integrals along the three edges, which are
 * split at every crossing of the light-cone circles r = j c dt (where the
 * B-spline pieces change) and integrated by adaptive Gauss-Legendre to ~1e-14.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_EINVAL 1
#define ORC_EMESH 2
#define ORC_ENOMEM 3

#define NGL 12            /* Gauss-Legendre order of the adaptive rule */
#define MAXLAG 64         /* max lags handled for one (x, triangle) pair */
#define MAXDEPTH 30

static const double PI = 3.14159265358979323846264338327950288;

/* ------------------------------------------------------------------ */
/* Gauss-Legendre nodes on [-1,1] by Newton iteration on P_n.          */
static double gl_x[NGL], gl_w[NGL];
static int gl_ready = 0;

static void gl_init(void) {
  if (gl_ready) return;
  int n = NGL;
  for (int i = 0; i < n; ++i) {
    double x = cos(PI * (i + 0.75) / (n + 0.5)), dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (x * p1 - p0) / (x * x - 1.0);
      double dx = p1 / dp;
      x -= dx;
      if (fabs(dx) < 1e-17) break;
    }
    /* recompute derivative at the converged node */
    double p0 = 1.0, p1 = x;
    for (int k = 2; k <= n; ++k) {
      double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = n * (x * p1 - p0) / (x * x - 1.0);
    gl_x[i] = x;
    gl_w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
  gl_ready = 1;
}

/* ------------------------------------------------------------------ */
/* B-spline in truncated powers (section 2.2).                         */
typedef struct {
  int d;
  double w[8]; /* w^{k,d}, k = 0..d+1 */
} bspline;

static void bs_init(bspline* b, int d) {
  b->d = d;
  for (int k = 0; k <= d + 1; ++k) {
    double prod = 1.0;
    for (int i = 0; i <= d + 1; ++i)
      if (i != k) prod *= (double)(i - k);
    b->w[k] = (double)(d + 1) / prod;
  }
}

static double ipow(double x, int n) {
  double r = 1.0;
  for (int i = 0; i < n; ++i) r *= x;
  return r;
}

/* derivative order q of N: sum_k w_k (d!/(d-q)!) (tau-k)_+^{d-q};
   q = -1 gives the running integral C(tau) = int_{-inf}^tau N.
   *scale receives sum_k |term_k|, the size of the rounding in the result. */
static double bs_eval2(const bspline* b, double tau, int q, double* scale) {
  int d = b->d;
  *scale = 0.0;
  if (tau <= 0.0) return 0.0;
  if (tau >= d + 1) { *scale = (q == -1) ? 1.0 : 0.0; return *scale; } /* vanishing property */
  double s = 0.0, a = 0.0;
  for (int k = 0; k <= d + 1; ++k) {
    double u = tau - k, t;
    if (u <= 0.0) continue;
    if (q == -1) {
      t = b->w[k] * ipow(u, d + 1) / (d + 1);
    } else {
      double c = 1.0;
      for (int i = 0; i < q; ++i) c *= (double)(d - i);
      t = b->w[k] * c * ipow(u, d - q);
    }
    s += t;
    a += fabs(t);
  }
  *scale = a;
  return s;
}

static double bs_eval(const bspline* b, double tau, int q) {
  double sc;
  return bs_eval2(b, tau, q, &sc);
}

/* ------------------------------------------------------------------ */
/* Context                                                             */
typedef struct {
  int64_t nv, nt, ne;
  double* V;      /* nv*3 */
  int32_t* T;     /* nt*3 */
  double* area;   /* nt */
  double* nout;   /* nt*3 outward unit normal */
  double* cen;    /* nt*3 centroid */
  double* rad;    /* nt max centroid-vertex distance */
  double* lmax;   /* nt longest edge */
  int32_t* ev;    /* ne*2 vertices (min, max) */
  int32_t* et;    /* ne*2 triangles (+, -) */
  int32_t* eo;    /* ne*2 opposite vertices (+, -) */
  double* elen;   /* ne */
  int32_t* te;    /* nt*3 edge of local edge k (v_k -> v_{k+1}) */
  int8_t* ts;     /* nt*3 +1 if the triangle is T+ of that edge, else -1 */
  double dt, eps, mu, c, eta, a, theta, zeta, sJ, chi;
  bspline bs;
  double qb[7][3], qw[7]; /* 7-point rule, barycentric */
} orc_ctx;

typedef struct {
  int32_t a, b, tri, k, dir; /* dir = +1 if traversed min->max */
} erec;

static int erec_cmp(const void* p, const void* q) {
  const erec* x = (const erec*)p;
  const erec* y = (const erec*)q;
  if (x->a != y->a) return x->a < y->a ? -1 : 1;
  if (x->b != y->b) return x->b < y->b ? -1 : 1;
  return 0;
}

static void sub3(const double* a, const double* b, double* o) {
  o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2];
}
static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double* a, const double* b, double* o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}
static double norm3(const double* a) { return sqrt(dot3(a, a)); }

void orc_destroy(orc_ctx* c) {
  if (!c) return;
  free(c->V); free(c->T); free(c->area); free(c->nout); free(c->cen); free(c->rad); free(c->lmax);
  free(c->ev); free(c->et); free(c->eo); free(c->elen); free(c->te); free(c->ts);
  free(c);
}

/* Build the mesh tables.  Edges are numbered lexicographically by (min vertex,
   max vertex); T+ is the triangle whose winding traverses the edge min->max. */
int orc_create(const double* verts, int64_t nv, const int32_t* tris, int64_t nt, double dt, double eps,
               double mu, double theta, double zeta, double sJ, double chi, int d, orc_ctx** out) {
  *out = NULL;
  if (nv < 3 || nt < 2 || dt <= 0 || eps <= 0 || mu <= 0 || d < 2 || d > 5) return ORC_EINVAL;
  orc_ctx* c = (orc_ctx*)calloc(1, sizeof(orc_ctx));
  if (!c) return ORC_ENOMEM;
  gl_init();
  c->nv = nv; c->nt = nt;
  c->V = (double*)malloc(sizeof(double) * 3 * nv);
  c->T = (int32_t*)malloc(sizeof(int32_t) * 3 * nt);
  memcpy(c->V, verts, sizeof(double) * 3 * nv);
  memcpy(c->T, tris, sizeof(int32_t) * 3 * nt);
  c->dt = dt; c->eps = eps; c->mu = mu;
  c->c = 1.0 / sqrt(eps * mu);
  c->eta = sqrt(mu / eps);
  c->a = c->c * dt;
  c->theta = theta; c->zeta = zeta; c->sJ = sJ; c->chi = chi;
  bs_init(&c->bs, d);
  /* 7-point degree-5 rule (Radon; Stroud T2:5-1), weights sum to 1 */
  {
    double s15 = sqrt(15.0);
    double a1 = (6.0 - s15) / 21.0, a2 = (6.0 + s15) / 21.0;
    double w1 = (155.0 - s15) / 1200.0, w2 = (155.0 + s15) / 1200.0;
    double P[7][3] = {{1.0 / 3, 1.0 / 3, 1.0 / 3},
                      {a1, a1, 1 - 2 * a1}, {a1, 1 - 2 * a1, a1}, {1 - 2 * a1, a1, a1},
                      {a2, a2, 1 - 2 * a2}, {a2, 1 - 2 * a2, a2}, {1 - 2 * a2, a2, a2}};
    double W[7] = {9.0 / 40, w1, w1, w1, w2, w2, w2};
    memcpy(c->qb, P, sizeof(P));
    memcpy(c->qw, W, sizeof(W));
  }
  c->area = (double*)malloc(sizeof(double) * nt);
  c->nout = (double*)malloc(sizeof(double) * 3 * nt);
  c->cen = (double*)malloc(sizeof(double) * 3 * nt);
  c->rad = (double*)malloc(sizeof(double) * nt);
  c->lmax = (double*)malloc(sizeof(double) * nt);
  for (int64_t t = 0; t < nt; ++t) {
    const int32_t* tv = c->T + 3 * t;
    for (int k = 0; k < 3; ++k)
      if (tv[k] < 0 || tv[k] >= nv) { orc_destroy(c); return ORC_EMESH; }
    const double *p0 = c->V + 3 * tv[0], *p1 = c->V + 3 * tv[1], *p2 = c->V + 3 * tv[2];
    double e1[3], e2[3], n[3];
    sub3(p1, p0, e1); sub3(p2, p0, e2); cross3(e1, e2, n);
    double nn = norm3(n);
    if (!(nn > 0)) { orc_destroy(c); return ORC_EMESH; }
    c->area[t] = 0.5 * nn;
    for (int k = 0; k < 3; ++k) {
      c->nout[3 * t + k] = n[k] / nn;
      c->cen[3 * t + k] = (p0[k] + p1[k] + p2[k]) / 3.0;
    }
    double r = 0, lm = 0;
    for (int k = 0; k < 3; ++k) {
      double dd[3];
      sub3(c->V + 3 * tv[k], c->cen + 3 * t, dd);
      r = fmax(r, norm3(dd));
      sub3(c->V + 3 * tv[(k + 1) % 3], c->V + 3 * tv[k], dd);
      lm = fmax(lm, norm3(dd));
    }
    c->rad[t] = r;
    c->lmax[t] = lm;
  }
  /* edge table */
  erec* R = (erec*)malloc(sizeof(erec) * 3 * nt);
  for (int64_t t = 0; t < nt; ++t)
    for (int k = 0; k < 3; ++k) {
      int32_t u = c->T[3 * t + k], v = c->T[3 * t + (k + 1) % 3];
      erec e;
      e.a = u < v ? u : v; e.b = u < v ? v : u; e.tri = (int32_t)t; e.k = k; e.dir = (u < v) ? 1 : -1;
      R[3 * t + k] = e;
    }
  qsort(R, 3 * nt, sizeof(erec), erec_cmp);
  if ((3 * nt) % 2) { free(R); orc_destroy(c); return ORC_EMESH; }
  int64_t ne = 3 * nt / 2;
  c->ne = ne;
  c->ev = (int32_t*)malloc(sizeof(int32_t) * 2 * ne);
  c->et = (int32_t*)malloc(sizeof(int32_t) * 2 * ne);
  c->eo = (int32_t*)malloc(sizeof(int32_t) * 2 * ne);
  c->elen = (double*)malloc(sizeof(double) * ne);
  c->te = (int32_t*)malloc(sizeof(int32_t) * 3 * nt);
  c->ts = (int8_t*)malloc(sizeof(int8_t) * 3 * nt);
  for (int64_t e = 0; e < ne; ++e) {
    erec r0 = R[2 * e], r1 = R[2 * e + 1];
    int bad = (r0.a != r1.a || r0.b != r1.b || r0.dir == r1.dir);
    if (!bad && 2 * e + 2 < 3 * nt) bad = (R[2 * e + 2].a == r0.a && R[2 * e + 2].b == r0.b);
    if (bad) { free(R); orc_destroy(c); return ORC_EMESH; }
    erec pl = r0.dir > 0 ? r0 : r1, mi = r0.dir > 0 ? r1 : r0;
    c->ev[2 * e] = r0.a; c->ev[2 * e + 1] = r0.b;
    c->et[2 * e] = pl.tri; c->et[2 * e + 1] = mi.tri;
    c->eo[2 * e] = c->T[3 * pl.tri + (pl.k + 2) % 3];
    c->eo[2 * e + 1] = c->T[3 * mi.tri + (mi.k + 2) % 3];
    double dd[3];
    sub3(c->V + 3 * r0.b, c->V + 3 * r0.a, dd);
    c->elen[e] = norm3(dd);
    c->te[3 * pl.tri + pl.k] = (int32_t)e; c->ts[3 * pl.tri + pl.k] = 1;
    c->te[3 * mi.tri + mi.k] = (int32_t)e; c->ts[3 * mi.tri + mi.k] = -1;
  }
  free(R);
  *out = c;
  return ORC_OK;
}

int64_t orc_num_edges(const orc_ctx* c) { return c->ne; }

void orc_edges(const orc_ctx* c, int32_t* ev, int32_t* et, int32_t* eo) {
  memcpy(ev, c->ev, sizeof(int32_t) * 2 * c->ne);
  memcpy(et, c->et, sizeof(int32_t) * 2 * c->ne);
  memcpy(eo, c->eo, sizeof(int32_t) * 2 * c->ne);
}

/* ------------------------------------------------------------------ */
/* Inner integrals over one source triangle for one observation point. */
typedef struct {
  const orc_ctx* c;
  int m0, nm, hasP;
  double h, hh, d, R0sq;
  long budget; /* remaining integrand evaluations for this segment */
  double phi0[MAXLAG], A0[MAXLAG], P0[MAXLAG]; /* radial antiderivatives at r = |h| */
  double sphi0[MAXLAG], sA0[MAXLAG], sP0[MAXLAG];
} ig_ctx;

/* radial antiderivatives (r dr = rho drho):
   scalar phi-term  F = N(tau)/r     -> Phi_phi(r) = -a C(tau)
   A-term           F = Nddot(tau)/r -> Phi_A(r)   = -a Ndot(tau)
   P-term           g(r) = (chi Ndot(tau)/dt + zeta N(tau))/r, d/dr g = F_P r  */
/* sphi/sA/sP receive the rounding scale of each value: the sum of the absolute
   truncated-power terms plus a tenth of the sensitivity to the rounding of
   tau = m - r/(c dt), whose operands are of size m + r/(c dt). */
static void radial_vals(const ig_ctx* g, double r, double* phi, double* A, double* P, double* sphi, double* sA,
                        double* sP) {
  const orc_ctx* c = g->c;
  for (int i = 0; i < g->nm; ++i) {
    double tau = (g->m0 + i) - r / c->a;
    double stau = 0.1 * ((g->m0 + i) + r / c->a);
    double s1, s2, s3;
    phi[i] = -c->a * bs_eval2(&c->bs, tau, -1, &s1);
    double nd = bs_eval2(&c->bs, tau, 1, &s2);
    A[i] = -c->a * nd;
    sphi[i] = c->a * (s1 + 2.0 * stau);
    sA[i] = c->a * (s2 + 4.0 * stau);
    if (g->hasP) {
      double n0 = bs_eval2(&c->bs, tau, 0, &s3);
      P[i] = (c->chi * nd / c->dt + c->zeta * n0) / r;
      sP[i] = (c->chi * s2 / c->dt + c->zeta * s3 + (4.0 * c->chi / c->dt + 4.0 * c->zeta) * stau) / r;
    }
  }
}

/* angular integrand: psi -> Phi(r_e(psi)) - Phi(|h|), three blocks of nm;
   mag[] receives |Phi(r_e)| + |Phi(|h|)|, the scale of rounding in out[] */
static void f_ang(double psi, ig_ctx* g, double* out, double* mag) {
  double rho = fabs(g->d) / cos(psi);
  double r = sqrt(g->h * g->h + rho * rho);
  int nm = g->nm;
  double phi[MAXLAG], A[MAXLAG], P[MAXLAG], sphi[MAXLAG], sA[MAXLAG], sP[MAXLAG];
  radial_vals(g, r, phi, A, P, sphi, sA, sP);
  for (int i = 0; i < nm; ++i) {
    out[i] = phi[i] - g->phi0[i];
    out[nm + i] = A[i] - g->A0[i];
    out[2 * nm + i] = g->hasP ? (P[i] - g->P0[i]) : 0.0;
    mag[i] = sphi[i] + g->sphi0[i];
    mag[nm + i] = sA[i] + g->sA0[i];
    mag[2 * nm + i] = g->hasP ? sP[i] + g->sP0[i] : 0.0;
  }
}

/* edge integrand: s -> (Phi_A(r), g(r)) */
static void f_edge(double s, ig_ctx* g, double* out, double* mag) {
  double r = sqrt(g->R0sq + s * s);
  int nm = g->nm;
  double phi[MAXLAG], A[MAXLAG], P[MAXLAG], sphi[MAXLAG], sA[MAXLAG], sP[MAXLAG];
  radial_vals(g, r, phi, A, P, sphi, sA, sP);
  for (int i = 0; i < nm; ++i) {
    out[i] = A[i];
    out[nm + i] = g->hasP ? P[i] : 0.0;
    mag[i] = sA[i];
    mag[nm + i] = g->hasP ? sP[i] : 0.0;
  }
}

typedef void (*vfun)(double, ig_ctx*, double*, double*);

static void gl_apply(vfun f, ig_ctx* g, int nc, double lo, double hi, double* I, double* L1) {
  g->budget -= NGL;
  double hw = 0.5 * (hi - lo), mid = 0.5 * (hi + lo);
  double v[3 * MAXLAG], mg[3 * MAXLAG];
  for (int k = 0; k < nc; ++k) I[k] = L1[k] = 0.0;
  for (int q = 0; q < NGL; ++q) {
    f(mid + hw * gl_x[q], g, v, mg);
    for (int k = 0; k < nc; ++k) {
      I[k] += gl_w[q] * hw * v[k];
      L1[k] += gl_w[q] * fabs(hw) * mg[k];
    }
  }
}

/* adaptive bisection: accept when halving changes no component by more than
   1e-14 of the L1 norm of its unsubtracted terms (the rounding scale) plus an
   absolute floor of 1e-15 of the component's L1 norm over the whole segment,
   pro rata to the interval length (floor[] is that norm per unit length) */
static void adapt(vfun f, ig_ctx* g, int nc, double lo, double hi, const double* whole, double* acc,
                  int depth, const double* floor) {
  double mid = 0.5 * (lo + hi);
  double Il[3 * MAXLAG], Ll[3 * MAXLAG], Ir[3 * MAXLAG], Lr[3 * MAXLAG];
  gl_apply(f, g, nc, lo, mid, Il, Ll);
  gl_apply(f, g, nc, mid, hi, Ir, Lr);
  int ok = 1;
  for (int k = 0; k < nc && ok; ++k) {
    double diff = fabs(Il[k] + Ir[k] - whole[k]);
    double tol = 1e-14 * (Ll[k] + Lr[k]) + 1e-15 * floor[k] * (hi - lo) + 1e-300;
    if (diff > tol) ok = 0;
  }
  if (ok || depth >= MAXDEPTH || g->budget < 0) {
    for (int k = 0; k < nc; ++k) acc[k] += Il[k] + Ir[k];
    return;
  }
  adapt(f, g, nc, lo, mid, Il, acc, depth + 1, floor);
  adapt(f, g, nc, mid, hi, Ir, acc, depth + 1, floor);
}

static int dcmp(const void* p, const void* q) {
  double x = *(const double*)p, y = *(const double*)q;
  return x < y ? -1 : (x > y ? 1 : 0);
}

/* integrate f over [lo, hi] split at the given interior break points */
static void integrate_split(vfun f, ig_ctx* g, int nc, double lo, double hi, double* br, int nb,
                            double* acc) {
  qsort(br, nb, sizeof(double), dcmp);
  g->budget = 200000;
  double pts[2 * MAXLAG + 8];
  int np = 0;
  pts[np++] = lo;
  for (int i = 0; i < nb; ++i)
    if (br[i] > lo && br[i] < hi) pts[np++] = br[i];
  pts[np++] = hi;
  double Wp[2 * MAXLAG + 8][3 * MAXLAG], L[3 * MAXLAG], fl[3 * MAXLAG];
  for (int k = 0; k < nc; ++k) fl[k] = 0.0;
  for (int i = 0; i + 1 < np; ++i) {
    if (!(pts[i + 1] > pts[i])) continue;
    gl_apply(f, g, nc, pts[i], pts[i + 1], Wp[i], L);
    for (int k = 0; k < nc; ++k) fl[k] += L[k];
  }
  for (int k = 0; k < nc; ++k) fl[k] /= (hi - lo);
  for (int i = 0; i + 1 < np; ++i) {
    if (!(pts[i + 1] > pts[i])) continue;
    adapt(f, g, nc, pts[i], pts[i + 1], Wp[i], acc, 0, fl);
  }
}

/* Inner integrals over source triangle t for observation point x and lags
   m0 .. m0+nm-1:
     phi[m]    = int_T N(tau)/r dS
     A0[m]     = int_T Nddot(tau)/r dS
     A1[m][3]  = int_T Nddot(tau)/r (y - x) dS
     P1[m][3]  = int_T (g'(r)/r) (y - x) dS,  g = (chi Ndot(tau)/dt + zeta N(tau))/r
   P1 is set to zero when x lies in the plane of t (then the tested P-term
   vanishes identically, see the notes on coplanar pairs). */
int orc_inner(const orc_ctx* c, const double* x, int64_t t, int m0, int nm, double* phi, double* A0, double* A1,
              double* P1) {
  if (nm < 1 || nm > MAXLAG || m0 < 1) return ORC_EINVAL;
  const int32_t* tv = c->T + 3 * t;
  const double* v[3] = {c->V + 3 * tv[0], c->V + 3 * tv[1], c->V + 3 * tv[2]};
  const double* nT = c->nout + 3 * t;
  double xv0[3];
  sub3(x, v[0], xv0);
  double h = dot3(xv0, nT);
  int hasP = fabs(h) > 1e-10 * c->lmax[t];
  if (!hasP) h = 0.0;
  double p[3] = {x[0] - h * nT[0], x[1] - h * nT[1], x[2] - h * nT[2]};
  ig_ctx g;
  g.c = c; g.m0 = m0; g.nm = nm; g.hasP = hasP; g.h = h; g.hh = fabs(h);
  radial_vals(&g, g.hh, g.phi0, g.A0, g.P0, g.sphi0, g.sA0, g.sP0);
  double S_phi[MAXLAG] = {0}, S_A0[MAXLAG] = {0}, S_Pn[MAXLAG] = {0};
  double VA[MAXLAG][3], VP[MAXLAG][3];
  memset(VA, 0, sizeof(VA));
  memset(VP, 0, sizeof(VP));
  /* knot circles r = j c dt that can cross the triangle */
  double rmax = 0, dc[3];
  for (int k = 0; k < 3; ++k) {
    double dd[3];
    sub3(v[k], x, dd);
    rmax = fmax(rmax, norm3(dd));
  }
  sub3(x, c->cen + 3 * t, dc);
  double rlow = norm3(dc) - c->rad[t];
  int jmin = (int)floor((rlow > 0 ? rlow : 0) / c->a);
  if (jmin < 1) jmin = 1;
  int jmax = (int)floor(rmax / c->a) + 1;
  if (jmax - jmin + 1 > MAXLAG) return ORC_EINVAL;
  for (int k = 0; k < 3; ++k) {
    const double *va = v[k], *vb = v[(k + 1) % 3];
    double tk[3], nuk[3], w[3];
    sub3(vb, va, tk);
    double L = norm3(tk);
    for (int i = 0; i < 3; ++i) tk[i] /= L;
    cross3(tk, nT, nuk);
    sub3(va, p, w);
    double d = dot3(w, nuk);
    double sm = dot3(w, tk);
    double wb[3];
    sub3(vb, p, wb);
    double sp = dot3(wb, tk);
    g.d = d;
    g.R0sq = h * h + d * d;
    /* angular part over the sub-triangle (p, va, vb), signed by d */
    if (fabs(d) > 1e-14 * L) {
      double psa = atan(sm / fabs(d)), psb = atan(sp / fabs(d));
      double br[2 * MAXLAG];
      int nb = 0;
      for (int j = jmin; j <= jmax; ++j) {
        double R = j * c->a;
        double q = R * R - h * h;
        if (q > d * d) {
          double ps = acos(fabs(d) / sqrt(q));
          br[nb++] = ps;
          br[nb++] = -ps;
        }
      }
      double acc[3 * MAXLAG] = {0};
      integrate_split(f_ang, &g, 3 * nm, psa, psb, br, nb, acc);
      double sg = d > 0 ? 1.0 : -1.0;
      for (int i = 0; i < nm; ++i) {
        S_phi[i] += sg * acc[i];
        S_A0[i] += sg * acc[nm + i];
        S_Pn[i] += sg * acc[2 * nm + i];
      }
    }
    /* edge part: int_edge Phi_A(r) ds and int_edge g(r) ds, times nu_k */
    {
      double br[2 * MAXLAG];
      int nb = 0;
      for (int j = jmin; j <= jmax; ++j) {
        double R = j * c->a;
        double q = R * R - g.R0sq;
        if (q > 0) {
          br[nb++] = sqrt(q);
          br[nb++] = -sqrt(q);
        }
      }
      double acc[2 * MAXLAG] = {0};
      integrate_split(f_edge, &g, 2 * nm, sm, sp, br, nb, acc);
      for (int i = 0; i < nm; ++i)
        for (int q = 0; q < 3; ++q) {
          VA[i][q] += nuk[q] * acc[i];
          VP[i][q] += nuk[q] * acc[nm + i];
        }
    }
  }
  for (int i = 0; i < nm; ++i) {
    phi[i] = S_phi[i];
    A0[i] = S_A0[i];
    for (int q = 0; q < 3; ++q) {
      A1[3 * i + q] = VA[i][q] - h * nT[q] * S_A0[i];
      P1[3 * i + q] = hasP ? (VP[i][q] - h * nT[q] * S_Pn[i]) : 0.0;
    }
  }
  return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Lag windows.                                                        */
static void lag_range(const orc_ctx* c, double rlo, double rhi, int* mlo, int* mhi) {
  int lo = (int)floor(rlo / c->a) + 1;
  if (lo < 1) lo = 1;
  int hi = (int)ceil(rhi / c->a + c->bs.d + 1) - 1;
  *mlo = lo;
  *mhi = hi;
}

/* conservative window of lags with a possibly non-zero coefficient for the
   edge pair (i, j): distance bounds over the four triangle pairs */
static void pair_window(const orc_ctx* c, int64_t i, int64_t j, int* mlo, int* mhi) {
  double rlo = 1e300, rhi = 0;
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      int32_t ta = c->et[2 * i + a], tb = c->et[2 * j + b];
      double dd[3];
      sub3(c->cen + 3 * ta, c->cen + 3 * tb, dd);
      double lo = norm3(dd) - c->rad[ta] - c->rad[tb];
      rlo = fmin(rlo, lo < 0 ? 0 : lo);
      for (int u = 0; u < 3; ++u)
        for (int w = 0; w < 3; ++w) {
          sub3(c->V + 3 * c->T[3 * ta + u], c->V + 3 * c->T[3 * tb + w], dd);
          rhi = fmax(rhi, norm3(dd));
        }
    }
  lag_range(c, rlo, rhi, mlo, mhi);
}

int orc_window(const orc_ctx* c) {
  int W = 0;
#pragma omp parallel for reduction(max : W) schedule(dynamic, 16)
  for (int64_t i = 0; i < c->ne; ++i)
    for (int64_t j = 0; j < c->ne; ++j) {
      int lo, hi;
      pair_window(c, i, j, &lo, &hi);
      if (hi - lo + 1 > W) W = hi - lo + 1;
    }
  return W;
}

/* The same over the pairs of the given rows only (storage for assembling those rows). */
int orc_window_rows(const orc_ctx* c, const int64_t* rows, int64_t nrows) {
  int W = 0;
#pragma omp parallel for reduction(max : W) schedule(dynamic, 1)
  for (int64_t r = 0; r < nrows; ++r)
    for (int64_t j = 0; j < c->ne; ++j) {
      int lo, hi;
      pair_window(c, rows[r], j, &lo, &hi);
      if (hi - lo + 1 > W) W = hi - lo + 1;
    }
  return W;
}

/* ------------------------------------------------------------------ */
/* Assembly of the rows `rows` of every Zt^(m):
     m_lo[r*ne + j] = first lag of the window of (rows[r], j)
     Zw[(r*ne + j)*W + w] = Zt^(m_lo + w)_{rows[r], j}                  */
int orc_assemble(const orc_ctx* c, const int64_t* rows, int64_t nrows, int W, int32_t* m_lo, double* Zw) {
  const int64_t ne = c->ne;
  const double mu4pi = c->mu / (4 * PI), ieps4pi = 1.0 / (4 * PI * c->eps), p4pi = 1.0 / (4 * PI);
  int err = ORC_OK;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t r = 0; r < nrows; ++r) {
    int64_t i = rows[r];
    int32_t* mlo_row = m_lo + r * ne;
    double* Zrow = Zw + r * ne * W;
    memset(Zrow, 0, sizeof(double) * ne * W);
    for (int64_t j = 0; j < ne; ++j) {
      int lo, hi;
      pair_window(c, i, j, &lo, &hi);
      if (hi - lo + 1 > W) {
#pragma omp atomic write
        err = ORC_EINVAL;
      }
      mlo_row[j] = lo;
    }
    for (int rho = 0; rho < 2; ++rho) {
      int64_t ti = c->et[2 * i + rho];
      double sgn_i = rho == 0 ? 1.0 : -1.0;
      const double* oi = c->V + 3 * c->eo[2 * i + rho];
      const int32_t* tv = c->T + 3 * ti;
      double Ai = c->area[ti];
      double fi_c = sgn_i * c->elen[i] / (2 * Ai);
      double divi = sgn_i * c->elen[i] / Ai;
      double nin[3] = {-c->nout[3 * ti], -c->nout[3 * ti + 1], -c->nout[3 * ti + 2]};
      for (int q = 0; q < 7; ++q) {
        double x[3], fi[3];
        for (int k = 0; k < 3; ++k)
          x[k] = c->qb[q][0] * c->V[3 * tv[0] + k] + c->qb[q][1] * c->V[3 * tv[1] + k] +
                 c->qb[q][2] * c->V[3 * tv[2] + k];
        for (int k = 0; k < 3; ++k) fi[k] = fi_c * (x[k] - oi[k]);
        double wq = c->qw[q] * Ai;
        for (int64_t s = 0; s < c->nt; ++s) {
          double dd[3];
          sub3(x, c->cen + 3 * s, dd);
          double rlo = norm3(dd) - c->rad[s];
          double rhi = 0;
          for (int u = 0; u < 3; ++u) {
            sub3(x, c->V + 3 * c->T[3 * s + u], dd);
            rhi = fmax(rhi, norm3(dd));
          }
          int mlo, mhi;
          lag_range(c, rlo < 0 ? 0 : rlo, rhi, &mlo, &mhi);
          int nm = mhi - mlo + 1;
          if (nm < 1) continue;
          double phi[MAXLAG], A0[MAXLAG], A1[3 * MAXLAG], P1[3 * MAXLAG];
          if (orc_inner(c, x, s, mlo, nm, phi, A0, A1, P1) != ORC_OK) {
#pragma omp atomic write
            err = ORC_EINVAL;
            continue;
          }
          for (int k = 0; k < 3; ++k) {
            int64_t j = c->te[3 * s + k];
            double sgn_j = c->ts[3 * s + k];
            int sig = sgn_j > 0 ? 0 : 1;
            const double* oj = c->V + 3 * c->eo[2 * j + sig];
            double fj_c = sgn_j * c->elen[j] / (2 * c->area[s]);
            double divj = sgn_j * c->elen[j] / c->area[s];
            double xo[3];
            sub3(x, oj, xo);
            for (int im = 0; im < nm; ++im) {
              int m = mlo + im;
              int w = m - mlo_row[j];
              if (w < 0 || w >= W) {
#pragma omp atomic write
                err = ORC_EINVAL;
                continue;
              }
              double IA[3], IP[3], cr[3], ncr[3];
              for (int u = 0; u < 3; ++u) IA[u] = fj_c * (A1[3 * im + u] + xo[u] * A0[im]);
              cross3(xo, P1 + 3 * im, cr);
              for (int u = 0; u < 3; ++u) IP[u] = fj_c * cr[u];
              cross3(nin, IP, ncr);
              double val = mu4pi / (c->dt * c->dt) * dot3(fi, IA) + ieps4pi * divi * divj * phi[im] +
                           c->theta * c->eta * p4pi * dot3(fi, ncr);
              Zrow[j * W + w] += wq * val;
            }
          }
        }
        /* MFIE identity term on the test triangle itself */
        if (c->sJ != 0.0) {
          for (int k = 0; k < 3; ++k) {
            int64_t j = c->te[3 * ti + k];
            double sgn_j = c->ts[3 * ti + k];
            int sig = sgn_j > 0 ? 0 : 1;
            const double* oj = c->V + 3 * c->eo[2 * j + sig];
            double fj_c = sgn_j * c->elen[j] / (2 * Ai);
            double fj[3];
            for (int u = 0; u < 3; ++u) fj[u] = fj_c * (x[u] - oj[u]);
            double G = wq * dot3(fi, fj);
            for (int m = 1; m <= c->bs.d + 1; ++m) {
              double coef = c->chi * bs_eval(&c->bs, (double)m, 1) / c->dt + c->zeta * bs_eval(&c->bs, (double)m, 0);
              if (coef == 0.0) continue;
              int w = m - mlo_row[j];
              if (w < 0 || w >= W) {
#pragma omp atomic write
                err = ORC_EINVAL;
                continue;
              }
              Zrow[j * W + w] += c->sJ * c->theta * c->eta * 0.5 * G * coef;
            }
          }
        }
      }
    }
  }
  return err;
}

/* ------------------------------------------------------------------ */
/* History sum for the rows `rows`:
     out[r] = sum_j sum_{m >= 2} Zt^(m)_{rows[r], j} J^{alpha-m}_j
   J_hist holds J^0 .. J^{n_hist-1} (row-major [n_hist][ne]); J^b = 0 for b < 0
   or b >= n_hist. */
void orc_history(const orc_ctx* c, const int32_t* m_lo, const double* Zw, int W, int64_t nrows, const double* J_hist,
                 int64_t n_hist, int64_t alpha, double* out) {
  const int64_t ne = c->ne;
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < nrows; ++r) {
    double s = 0.0;
    for (int64_t j = 0; j < ne; ++j) {
      int lo = m_lo[r * ne + j];
      const double* z = Zw + (r * ne + j) * W;
      for (int w = 0; w < W; ++w) {
        int64_t m = lo + w;
        if (m < 2) continue;
        int64_t b = alpha - m;
        if (b < 0 || b >= n_hist) continue;
        s += z[w] * J_hist[b * ne + j];
      }
    }
    out[r] = s;
  }
}

/* ------------------------------------------------------------------ */
/* Incident right-hand side (eq. v_i) at t_alpha for the rows `rows`.
   pulse = {k[3], pol[3], f0, sigma, t0, z_min}:
     E(x,t) = pol g(u), H = k x E / eta, u = t - (k.x - z_min)/c,
     g(u) = cos(2 pi f0 (u - t0)) exp(-(u - t0)^2/(2 sigma^2)).           */
/* Pulse shape g and its time derivative at u.  sigma > 0: modulated Gaussian
   cos(2 pi f0 (u - t0)) exp(-(u - t0)^2 / (2 sigma^2)); sigma < 0: the Sin^2
   pulse of the paper's test problem (section 4.1), A sin^2(2 pi c (u - t0) /
   Lambda) on one period 0 .. 2 pi of its argument, Lambda = f0, A = -sigma. */
static void pulse_g(const double* P, double u, double c, double* g, double* gd) {
  double f0 = P[6], sg = P[7], t0 = P[8];
  double v = u - t0;
  if (sg > 0) {
    double e = exp(-v * v / (2 * sg * sg));
    double cw = cos(2 * PI * f0 * v), sw = sin(2 * PI * f0 * v);
    *g = cw * e;
    *gd = (-2 * PI * f0 * sw - v / (sg * sg) * cw) * e;
    return;
  }
  double w = 2 * PI * c / f0, x = w * v;
  *g = 0.0;
  *gd = 0.0;
  if (x >= 0.0 && x <= 2 * PI) {
    *g = -sg * sin(x) * sin(x);
    *gd = -sg * 2.0 * sin(x) * cos(x) * w;
  }
}

void orc_rhs(const orc_ctx* c, const double* pulse, int64_t alpha, const int64_t* rows, int64_t nrows, double* V) {
  const double* k = pulse;
  const double* pol = pulse + 3;
  double kxp[3];
  cross3(k, pol, kxp);
  double t = alpha * c->dt;
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < nrows; ++r) {
    int64_t i = rows[r];
    double s = 0.0;
    for (int rho = 0; rho < 2; ++rho) {
      int64_t ti = c->et[2 * i + rho];
      double sgn_i = rho == 0 ? 1.0 : -1.0;
      const double* oi = c->V + 3 * c->eo[2 * i + rho];
      const int32_t* tv = c->T + 3 * ti;
      double Ai = c->area[ti];
      double fi_c = sgn_i * c->elen[i] / (2 * Ai);
      double nin[3] = {-c->nout[3 * ti], -c->nout[3 * ti + 1], -c->nout[3 * ti + 2]};
      for (int q = 0; q < 7; ++q) {
        double x[3], fi[3];
        for (int u = 0; u < 3; ++u)
          x[u] = c->qb[q][0] * c->V[3 * tv[0] + u] + c->qb[q][1] * c->V[3 * tv[1] + u] +
                 c->qb[q][2] * c->V[3 * tv[2] + u];
        for (int u = 0; u < 3; ++u) fi[u] = fi_c * (x[u] - oi[u]);
        double uu = t - (dot3(k, x) - pulse[9]) / c->c;
        double g, gd;
        pulse_g(pulse, uu, c->c, &g, &gd);
        double Ed[3], Hm[3], nH[3];
        for (int u = 0; u < 3; ++u) {
          Ed[u] = pol[u] * gd;
          Hm[u] = kxp[u] * (c->chi * gd + c->zeta * g) / c->eta; /* chi Hdot + zeta H */
        }
        cross3(nin, Hm, nH);
        double val = 0;
        for (int u = 0; u < 3; ++u) val += fi[u] * (-Ed[u] + c->theta * c->eta * nH[u]);
        s += c->qw[q] * Ai * val;
      }
    }
    V[r] = s;
  }
}

int orc_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Exposed for the pins: the B-spline (and its derivatives / running integral)
   and the Gauss-Legendre rule used by the adaptive integrator. */
double orc_bspline(int d, double tau, int q) {
  bspline b;
  bs_init(&b, d);
  return bs_eval(&b, tau, q);
}

void orc_bspline_weights(int d, double* w) {
  bspline b;
  bs_init(&b, d);
  for (int k = 0; k <= d + 1; ++k) w[k] = b.w[k];
}

int orc_gl(double* x, double* w) {
  gl_init();
  for (int i = 0; i < NGL; ++i) {
    x[i] = gl_x[i];
    w[i] = gl_w[i];
  }
  return NGL;
}
