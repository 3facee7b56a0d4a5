// mesh.cu -- host planner, part 1: RWG edge table and device triangle geometry.
//
// RWG basis (paper section 2.2): one basis function per interior edge, on the
// two triangles that share it.  Edges are numbered in increasing (min vertex,
// max vertex) order; the "+" triangle is the one whose winding runs min -> max.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "internal.h"

namespace {

struct HalfEdge {
  int32_t lo, hi, tri, side;
  bool fwd;  // traversed lo -> hi
};

}  // namespace

tdbem_status tdbem_build_mesh(tdbem_ctx* c, const double* verts, int64_t nv, const int32_t* tris, int64_t ntri) {
  if (nv < 4 || ntri < 4 || nv > (int64_t)1 << 30 || ntri > (int64_t)1 << 29) {
    c->set_error("mesh: need at least 4 vertices and 4 triangles");
    return TDBEM_EINVAL;
  }
  c->nv = nv;
  c->nt = ntri;
  c->V.assign(verts, verts + 3 * nv);
  c->T.assign(tris, tris + 3 * ntri);
  std::vector<HalfEdge> he(3 * ntri);
  for (int64_t t = 0; t < ntri; ++t) {
    for (int k = 0; k < 3; ++k) {
      int32_t a = tris[3 * t + k], b = tris[3 * t + (k + 1) % 3];
      if (a < 0 || a >= nv || b < 0 || b >= nv || a == b) {
        c->set_error("mesh: triangle index out of range or repeated vertex");
        return TDBEM_EMESH;
      }
      he[3 * t + k] = HalfEdge{std::min(a, b), std::max(a, b), (int32_t)t, k, a < b};
    }
  }
  std::sort(he.begin(), he.end(), [](const HalfEdge& x, const HalfEdge& y) {
    return x.lo != y.lo ? x.lo < y.lo : x.hi < y.hi;
  });
  if (he.size() % 2) {
    c->set_error("mesh: odd number of half-edges (not closed)");
    return TDBEM_EMESH;
  }
  int64_t ne = (int64_t)he.size() / 2;
  c->ne = ne;
  c->ev.resize(2 * ne);
  c->et.resize(2 * ne);
  c->eo.resize(2 * ne);
  c->te.assign(3 * ntri, -1);
  c->ts.assign(3 * ntri, 0);
  for (int64_t e = 0; e < ne; ++e) {
    const HalfEdge& x = he[2 * e];
    const HalfEdge& y = he[2 * e + 1];
    bool bad = x.lo != y.lo || x.hi != y.hi || x.fwd == y.fwd;
    if (!bad && 2 * e + 2 < (int64_t)he.size()) bad = he[2 * e + 2].lo == x.lo && he[2 * e + 2].hi == x.hi;
    if (bad) {
      c->set_error("mesh: edge not shared by exactly two oppositely wound triangles");
      return TDBEM_EMESH;
    }
    const HalfEdge& pl = x.fwd ? x : y;
    const HalfEdge& mi = x.fwd ? y : x;
    c->ev[2 * e] = x.lo;
    c->ev[2 * e + 1] = x.hi;
    c->et[2 * e] = pl.tri;
    c->et[2 * e + 1] = mi.tri;
    c->eo[2 * e] = tris[3 * pl.tri + (pl.side + 2) % 3];
    c->eo[2 * e + 1] = tris[3 * mi.tri + (mi.side + 2) % 3];
    c->te[3 * pl.tri + pl.side] = (int32_t)e;
    c->ts[3 * pl.tri + pl.side] = 1;
    c->te[3 * mi.tri + mi.side] = (int32_t)e;
    c->ts[3 * mi.tri + mi.side] = -1;
  }
  // per-triangle geometry
  std::vector<double> hv(9 * ntri), hn(3 * ntri), hc(3 * ntri), ha(ntri), hr(ntri), hl(ntri), ho(9 * ntri),
      hel(3 * ntri);
  for (int64_t t = 0; t < ntri; ++t) {
    const double* P[3];
    for (int k = 0; k < 3; ++k) P[k] = verts + 3 * tris[3 * t + k];
    double e1[3], e2[3], n[3];
    for (int q = 0; q < 3; ++q) {
      e1[q] = P[1][q] - P[0][q];
      e2[q] = P[2][q] - P[0][q];
    }
    n[0] = e1[1] * e2[2] - e1[2] * e2[1];
    n[1] = e1[2] * e2[0] - e1[0] * e2[2];
    n[2] = e1[0] * e2[1] - e1[1] * e2[0];
    double nn = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    if (!(nn > 0)) {
      c->set_error("mesh: degenerate triangle");
      return TDBEM_EMESH;
    }
    ha[t] = 0.5 * nn;
    double r = 0, lm = 0;
    for (int q = 0; q < 3; ++q) {
      hn[3 * t + q] = n[q] / nn;
      hc[3 * t + q] = (P[0][q] + P[1][q] + P[2][q]) / 3.0;
    }
    for (int k = 0; k < 3; ++k) {
      double dc = 0, dl = 0;
      for (int q = 0; q < 3; ++q) {
        hv[9 * t + 3 * k + q] = P[k][q];
        ho[9 * t + 3 * k + q] = P[(k + 2) % 3][q];
        double u = P[k][q] - hc[3 * t + q];
        double w = P[(k + 1) % 3][q] - P[k][q];
        dc += u * u;
        dl += w * w;
      }
      r = std::max(r, std::sqrt(dc));
      lm = std::max(lm, std::sqrt(dl));
      hel[3 * t + k] = std::sqrt(dl);
    }
    hr[t] = r;
    c->max_tri_rad = std::max(c->max_tri_rad, r);
    // the far field samples a triangle only at its outer-rule points
    for (int qq = 0; qq < tdbem::kNq; ++qq) {
      double d2 = 0;
      for (int q = 0; q < 3; ++q) {
        const double x = c->phys.qb[qq][0] * P[0][q] + c->phys.qb[qq][1] * P[1][q] + c->phys.qb[qq][2] * P[2][q];
        d2 += (x - hc[3 * t + q]) * (x - hc[3 * t + q]);
      }
      c->max_quad_rad = std::max(c->max_quad_rad, std::sqrt(d2));
    }
    hl[t] = lm;
  }
  tdbem_status s;
  tdbem::TriGeom& g = c->tg;
  if ((s = c->dalloc(&g.v, 9 * ntri)) || (s = c->dalloc(&g.nrm, 3 * ntri)) || (s = c->dalloc(&g.cen, 3 * ntri)) ||
      (s = c->dalloc(&g.area, ntri)) || (s = c->dalloc(&g.rad, ntri)) || (s = c->dalloc(&g.lmax, ntri)) ||
      (s = c->dalloc(&g.edge, 3 * ntri)) || (s = c->dalloc(&g.sgn, 3 * ntri)) || (s = c->dalloc(&g.opp, 9 * ntri)) ||
      (s = c->dalloc(&g.elen, 3 * ntri)) || (s = c->dalloc(&c->d_et, 2 * ne)))
    return s;
  TDBEM_CUDA_TRY(c, cudaMemcpy(g.v, hv.data(), 9 * ntri * sizeof(double), cudaMemcpyHostToDevice));
  TDBEM_CUDA_TRY(c, cudaMemcpy(g.nrm, hn.data(), 3 * ntri * sizeof(double), cudaMemcpyHostToDevice));
  TDBEM_CUDA_TRY(c, cudaMemcpy(g.cen, hc.data(), 3 * ntri * sizeof(double), cudaMemcpyHostToDevice));
  TDBEM_CUDA_TRY(c, cudaMemcpy(g.area, ha.data(), ntri * sizeof(double), cudaMemcpyHostToDevice));
  TDBEM_CUDA_TRY(c, cudaMemcpy(g.rad, hr.data(), ntri * sizeof(double), cudaMemcpyHostToDevice));
  TDBEM_CUDA_TRY(c, cudaMemcpy(g.lmax, hl.data(), ntri * sizeof(double), cudaMemcpyHostToDevice));
  TDBEM_CUDA_TRY(c, cudaMemcpy(g.edge, c->te.data(), 3 * ntri * sizeof(int32_t), cudaMemcpyHostToDevice));
  TDBEM_CUDA_TRY(c, cudaMemcpy(g.sgn, c->ts.data(), 3 * ntri * sizeof(int8_t), cudaMemcpyHostToDevice));
  TDBEM_CUDA_TRY(c, cudaMemcpy(g.opp, ho.data(), 9 * ntri * sizeof(double), cudaMemcpyHostToDevice));
  TDBEM_CUDA_TRY(c, cudaMemcpy(g.elen, hel.data(), 3 * ntri * sizeof(double), cudaMemcpyHostToDevice));
  TDBEM_CUDA_TRY(c, cudaMemcpy(c->d_et, c->et.data(), 2 * ne * sizeof(int32_t), cudaMemcpyHostToDevice));
  return TDBEM_OK;
}
