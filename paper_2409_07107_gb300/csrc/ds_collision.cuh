// Collision detection between convex shapes (Sec. 2.1): the signed distance, the witness points,
// the contact point and the contact frame (Z along the normal from A to B) of two shapes at given
// world poses.  FP64, host- and device-callable, one pair per thread.
//
// Every shape is a core swept by a radius: a sphere is a point + r, a capsule a segment along its
// body z axis (from -half_length to +half_length) + r, a box its 8 corners + 0, a hull the convex
// hull of up to 32 vertices (a range of a shared vertex pool, body frame) + r.  The signed
// distance is the distance of the cores minus rA + rB when the cores are apart, and minus
// (penetration depth of the cores + rA + rB) when they overlap.
//
// * Cores apart: GJK (Gilbert, Johnson & Keerthi 1988) on the Minkowski difference D = A - B with
//   the closest point of each simplex to the origin found by region tests (Ericson, Real-Time
//   Collision Detection, 2005, Sec. 5.1.5 for the triangle); the final simplex's barycentric
//   weights give the witness points on A and B.
// * Cores overlapping: the penetration depth is min over unit m of h_D(m) (h the support
//   function), attained at a facet normal of D.  Every facet of a Minkowski sum of a box with a
//   box, segment or point has as normal a face normal of a box or the cross product of an edge
//   direction of each core, so the minimum over those (15 axes for two boxes, 6 for a segment and
//   a box, 3 for a point and a box) is the depth (the separating-axis form; GJK/EPA's polytope
//   expansion reaches the same facet).  The same axes decide whether cores with a box overlap at
//   all (a negative minimum is a separating axis), so GJK runs only on separated cores there.
//   A hull has no such short axis list: overlapping cores with a hull take the expanding polytope
//   (EPA, van den Bergen 2001) from GJK's tetrahedron around the origin (or, where GJK stopped on
//   the origin before forming one, a tetrahedron built by GJK's intersection iteration).  The
//   witness points are the projection of the origin on that facet, split over the two cores'
//   support features.
// * The contact point is the midpoint of the witness points moved to the surfaces (pA + rA n,
//   pB - rB n); the tangent axes follow the plane contacts' rule: t1 = normalize(e_x - (n.e_x) n),
//   e_y in place of e_x when |n_x| > 0.9, t2 = n x t1.
#pragma once
#include <cmath>

#include "ds_common.cuh"

namespace ds {
namespace cd {

constexpr int kGjkMaxIter = 64;
constexpr int kCoreMax = DS_CONVEX_HULL_MAX;   // vertices of a hull core (32)
enum CoreKind { kPoint = 0, kSegment = 1, kBox = 2, kHull = 3 };

// A core in world coordinates: 1 point, 2 segment end points, 8 box corners or up to NMAX hull
// vertices, plus the radius and (for a box) its axes, the directions of its faces and edges.
// Code that may meet hulls uses Core (32 vertices); code that rules them out uses BoxCore (8),
// which keeps its per-thread state small.
template <int NMAX>
struct CoreT {
  static constexpr int kMax = NMAX;
  int kind;
  int nv;
  double v[NMAX][3];
  double r;
  double axis[3][3];   // box: the columns of R; segment: axis[0] = its direction
  int naxis;           // 3 for a box, 1 for a segment, 0 for a point
};
using Core = CoreT<kCoreMax>;
using BoxCore = CoreT<8>;

DS_HDI void sub3(const double* a, const double* b, double* o) {
  o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2];
}

DS_HDI void copy3(const double* a, double* o) { o[0] = a[0]; o[1] = a[1]; o[2] = a[2]; }

// Build the world core of shape (type, size) at pose (R row-major, p); a hull's vertices come
// from the pool hv (n_hv vertices, body frame).  Returns false for an unknown type or a hull whose
// vertex range is not an integral range of 4..32 vertices inside the pool (always for a BoxCore).
template <class C>
DS_HDI bool make_core(int type, const double* size, const double* R, const double* p, const double* hv,
                      int n_hv, C& c) {
  if (type == DS_CONVEX_HULL) {
    if (C::kMax < kCoreMax) return false;
    const double f = size[0], n = size[1];
    if (!(f >= 0.0 && n >= 4.0 && n <= C::kMax && f == floor(f) && n == floor(n))) return false;
    const int first = static_cast<int>(f), count = static_cast<int>(n);
    if (hv == nullptr || first > n_hv - count) return false;
    c.kind = kHull; c.nv = count; c.naxis = 0; c.r = size[2];
    for (int i = 0; i < count; ++i) {
      const double* x = hv + 3 * (first + i);
      for (int k = 0; k < 3; ++k) c.v[i][k] = p[k] + R[3 * k] * x[0] + R[3 * k + 1] * x[1] + R[3 * k + 2] * x[2];
    }
    return true;
  }
  if (type == DS_CONVEX_SPHERE) {
    c.kind = kPoint; c.nv = 1; c.naxis = 0; c.r = size[0];
    copy3(p, c.v[0]);
    return true;
  }
  if (type == DS_CONVEX_CAPSULE) {
    const double h = size[0];
    c.kind = kSegment; c.nv = 2; c.naxis = 1; c.r = size[1];
    for (int k = 0; k < 3; ++k) {
      const double z = R[3 * k + 2];
      c.v[0][k] = p[k] - h * z;
      c.v[1][k] = p[k] + h * z;
      c.axis[0][k] = z;
    }
    return true;
  }
  if (type == DS_CONVEX_BOX) {
    c.kind = kBox; c.nv = 8; c.naxis = 3; c.r = 0.0;
    for (int i = 0; i < 8; ++i) {
      const double s0 = (i & 4) ? size[0] : -size[0];
      const double s1 = (i & 2) ? size[1] : -size[1];
      const double s2 = (i & 1) ? size[2] : -size[2];
      for (int k = 0; k < 3; ++k) c.v[i][k] = p[k] + R[3 * k] * s0 + R[3 * k + 1] * s1 + R[3 * k + 2] * s2;
    }
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k) c.axis[j][k] = R[3 * k + j];
    return true;
  }
  return false;
}

// Index of the core vertex with the largest d . v (the first of equals).
template <class C>
DS_HDI int support(const C& c, const double* d) {
  int best = 0;
  double bv = dot3(d, c.v[0]);
  for (int i = 1; i < c.nv; ++i) {
    const double x = dot3(d, c.v[i]);
    if (x > bv) { bv = x; best = i; }
  }
  return best;
}

// ------------------------------------------------------------------------------------------ GJK
// A simplex of D: up to 4 points w_j = A.v[ia_j] - B.v[ib_j] with barycentric weights.
struct Simplex {
  int n;
  double w[4][3];
  int ia[4], ib[4];
  double lam[4];
};

// Weights (1 - t, t) of the point of segment ab closest to the origin.
DS_HDI void seg_weights(const double* a, const double* b, double* l) {
  double ab[3];
  sub3(b, a, ab);
  const double den = dot3(ab, ab);
  double t = den > 0.0 ? -dot3(a, ab) / den : 0.0;
  t = t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
  l[0] = 1.0 - t;
  l[1] = t;
}

// Weights of the point of triangle abc closest to the origin: the vertex, edge and face regions
// tested in turn (Ericson 2005, Sec. 5.1.5).  A degenerate (collinear) triangle takes the best of
// its edges.
DS_HDI void tri_weights(const double* a, const double* b, const double* c, double* l) {
  double ab[3], ac[3];
  sub3(b, a, ab);
  sub3(c, a, ac);
  const double d1 = -dot3(ab, a), d2 = -dot3(ac, a);
  if (d1 <= 0.0 && d2 <= 0.0) { l[0] = 1.0; l[1] = 0.0; l[2] = 0.0; return; }
  const double d3 = -dot3(ab, b), d4 = -dot3(ac, b);
  if (d3 >= 0.0 && d4 <= d3) { l[0] = 0.0; l[1] = 1.0; l[2] = 0.0; return; }
  const double vc = d1 * d4 - d3 * d2;
  if (vc <= 0.0 && d1 >= 0.0 && d3 <= 0.0) {
    const double t = d1 / (d1 - d3);
    l[0] = 1.0 - t; l[1] = t; l[2] = 0.0;
    return;
  }
  const double d5 = -dot3(ab, c), d6 = -dot3(ac, c);
  if (d6 >= 0.0 && d5 <= d6) { l[0] = 0.0; l[1] = 0.0; l[2] = 1.0; return; }
  const double vb = d5 * d2 - d1 * d6;
  if (vb <= 0.0 && d2 >= 0.0 && d6 <= 0.0) {
    const double t = d2 / (d2 - d6);
    l[0] = 1.0 - t; l[1] = 0.0; l[2] = t;
    return;
  }
  const double va = d3 * d6 - d5 * d4;
  if (va <= 0.0 && d4 - d3 >= 0.0 && d5 - d6 >= 0.0) {
    const double t = (d4 - d3) / ((d4 - d3) + (d5 - d6));
    l[0] = 0.0; l[1] = 1.0 - t; l[2] = t;
    return;
  }
  const double den = va + vb + vc;
  if (den > 0.0) {
    l[1] = vb / den;
    l[2] = vc / den;
    l[0] = 1.0 - l[1] - l[2];
    return;
  }
  // collinear: the nearest of the three edges
  const double* P[3] = {a, b, c};
  double best = -1.0;
  for (int e = 0; e < 3; ++e) {
    const int i = e, j = (e + 1) % 3;
    double le[2], x[3];
    seg_weights(P[i], P[j], le);
    for (int k = 0; k < 3; ++k) x[k] = le[0] * P[i][k] + le[1] * P[j][k];
    const double d = dot3(x, x);
    if (best < 0.0 || d < best) {
      best = d;
      l[0] = l[1] = l[2] = 0.0;
      l[i] = le[0];
      l[j] = le[1];
    }
  }
}

// Keep the simplex points listed in idx[0..m) with weights l (in that order).
DS_HDI void keep(Simplex& s, const int* idx, const double* l, int m) {
  Simplex t;
  t.n = m;
  for (int j = 0; j < m; ++j) {
    copy3(s.w[idx[j]], t.w[j]);
    t.ia[j] = s.ia[idx[j]];
    t.ib[j] = s.ib[idx[j]];
    t.lam[j] = l[j];
  }
  s = t;
}

// Replace the simplex by the smallest face carrying its point closest to the origin (weights > 0)
// and return that point in v.  Returns true when the origin lies inside a tetrahedron.
DS_HDI bool closest_reduce(Simplex& s, double* v) {
  double l[4] = {1.0, 0.0, 0.0, 0.0};
  int idx[4] = {0, 1, 2, 3};
  int m = s.n;
  if (s.n == 2) {
    seg_weights(s.w[0], s.w[1], l);
  } else if (s.n == 3) {
    tri_weights(s.w[0], s.w[1], s.w[2], l);
  } else if (s.n == 4) {
    // faces (i, j, k) with the opposite vertex o; the origin is outside a face when it lies on
    // the other side of the face's plane from o.  A flat tetrahedron (o within 1e-9 of the face's
    // plane relative to the sizes) has no inside: every face counts as outside, so that rounding
    // in the side tests cannot report the origin inside it
    const int F[4][4] = {{0, 1, 2, 3}, {0, 1, 3, 2}, {0, 2, 3, 1}, {1, 2, 3, 0}};
    bool inside = true;
    double best = -1.0;
    for (int f = 0; f < 4; ++f) {
      const double *wi = s.w[F[f][0]], *wj = s.w[F[f][1]], *wk = s.w[F[f][2]], *wo = s.w[F[f][3]];
      double e1[3], e2[3], nrm[3], eo[3];
      sub3(wj, wi, e1);
      sub3(wk, wi, e2);
      cross3(e1, e2, nrm);
      sub3(wo, wi, eo);
      const double so = -dot3(nrm, wi), sd = dot3(nrm, eo);
      const bool flat = fabs(sd) <= 1e-9 * sqrt(dot3(nrm, nrm) * dot3(eo, eo));
      if (!flat && so * sd >= 0.0) continue;
      inside = false;
      double lf[3], x[3];
      tri_weights(wi, wj, wk, lf);
      for (int k = 0; k < 3; ++k) x[k] = lf[0] * wi[k] + lf[1] * wj[k] + lf[2] * wk[k];
      const double d = dot3(x, x);
      if (best < 0.0 || d < best) {
        best = d;
        l[0] = l[1] = l[2] = l[3] = 0.0;
        for (int k = 0; k < 3; ++k) l[F[f][k]] = lf[k];
      }
    }
    if (inside) {
      v[0] = v[1] = v[2] = 0.0;
      return true;
    }
  }
  // keep the points with positive weight
  int kept = 0;
  double lk[4];
  for (int j = 0; j < m; ++j)
    if (l[j] > 0.0) {
      idx[kept] = j;
      lk[kept] = l[j];
      ++kept;
    }
  if (kept == 0) {   // cannot happen for weights summing to 1; keep the first point
    idx[0] = 0;
    lk[0] = 1.0;
    kept = 1;
  }
  keep(s, idx, lk, kept);
  v[0] = v[1] = v[2] = 0.0;
  for (int j = 0; j < s.n; ++j)
    for (int k = 0; k < 3; ++k) v[k] += s.lam[j] * s.w[j][k];
  return false;
}

// Distance of the cores by GJK: returns true when they overlap (the origin in D, or a distance
// below 1e-12); the witness points pa (on A), pb (on B) are those of the last simplex that did
// not contain the origin.  When the origin lies inside a tetrahedron of support points, that
// tetrahedron is copied to *tet (if given) and tet->n = 4; otherwise tet->n = 0.
template <class C>
DS_HDI bool gjk(const C& A, const C& B, double* pa, double* pb, Simplex* tet = nullptr) {
  if (tet) tet->n = 0;
  Simplex s;
  s.n = 1;
  s.ia[0] = 0;
  s.ib[0] = 0;
  s.lam[0] = 1.0;
  sub3(A.v[0], B.v[0], s.w[0]);
  double v[3];
  copy3(s.w[0], v);
  double vv = dot3(v, v);
  bool overlap = false;
  for (int it = 0; it < kGjkMaxIter; ++it) {
    if (vv <= 1e-24) { overlap = true; break; }
    const double nv[3] = {-v[0], -v[1], -v[2]};
    const int ia = support(A, nv), ib = support(B, v);
    bool dup = false;
    for (int j = 0; j < s.n; ++j) dup = dup || (s.ia[j] == ia && s.ib[j] == ib);
    double w[3];
    sub3(A.v[ia], B.v[ib], w);
    // stop when the new support point cannot bring the simplex closer to the origin
    if (dup || vv - dot3(v, w) <= 1e-12 * vv) break;
    Simplex prev = s;
    copy3(w, s.w[s.n]);
    s.ia[s.n] = ia;
    s.ib[s.n] = ib;
    ++s.n;
    double vn[3];
    if (closest_reduce(s, vn)) {
      if (tet) *tet = s;
      s = prev;
      overlap = true;
      break;
    }
    const double vvn = dot3(vn, vn);
    if (!(vvn < vv)) {   // no progress in floating point: keep the previous simplex
      s = prev;
      break;
    }
    copy3(vn, v);
    vv = vvn;
  }
  for (int k = 0; k < 3; ++k) {
    pa[k] = 0.0;
    pb[k] = 0.0;
    for (int j = 0; j < s.n; ++j) {
      pa[k] += s.lam[j] * A.v[s.ia[j]][k];
      pb[k] += s.lam[j] * B.v[s.ib[j]][k];
    }
  }
  return overlap;
}

// ---------------------------------------------------------------------- overlapping cores
// Closest points of segments [p1, q1] and [p2, q2] (the unconstrained minimiser of the squared
// distance, clamped to the square; used for two support edges whose closest points are interior).
DS_HDI void seg_seg(const double* p1, const double* q1, const double* p2, const double* q2,
                    double* x1, double* x2) {
  double d1[3], d2[3], r[3];
  sub3(q1, p1, d1);
  sub3(q2, p2, d2);
  sub3(p1, p2, r);
  const double a = dot3(d1, d1), b = dot3(d1, d2), e = dot3(d2, d2);
  const double c = dot3(d1, r), f = dot3(d2, r);
  const double den = a * e - b * b;
  double s = den > 1e-14 * a * e ? (b * f - c * e) / den : 0.0;
  s = s < 0.0 ? 0.0 : (s > 1.0 ? 1.0 : s);
  double t = e > 0.0 ? (b * s + f) / e : 0.0;
  t = t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
  if (a > 0.0) {
    s = (b * t - c) / a;
    s = s < 0.0 ? 0.0 : (s > 1.0 ? 1.0 : s);
  }
  for (int k = 0; k < 3; ++k) {
    x1[k] = p1[k] + s * d1[k];
    x2[k] = p2[k] + t * d2[k];
  }
}

// The range [lo, hi] of u . v over the vertices v of a core.
template <class C>
DS_HDI void project(const C& c, const double* u, double& lo, double& hi) {
  lo = hi = dot3(u, c.v[0]);
  for (int i = 1; i < c.nv; ++i) {
    const double x = dot3(u, c.v[i]);
    lo = fmin(lo, x);
    hi = fmax(hi, x);
  }
}

// Separating-axis test of two cores of which one is a box: depth = the minimum of h_D over the
// candidate axes, with its unit axis m.  depth < 0: m separates the cores (they are apart).
// depth >= 0: the cores overlap, depth is their penetration depth and m the axis from A to B
// (moving A by -depth m separates them); then the witness points pa on A, pb on B with
// pa - pb = depth m are written too.
template <class C>
DS_HDI void penetration(const C& A, const C& B, double& depth, double* m, double* pa, double* pb) {
  double cand[15][3];
  int nc = 0;
  if (A.kind == kBox)
    for (int i = 0; i < 3; ++i) copy3(A.axis[i], cand[nc++]);
  if (B.kind == kBox)
    for (int j = 0; j < 3; ++j) copy3(B.axis[j], cand[nc++]);
  for (int i = 0; i < A.naxis; ++i)
    for (int j = 0; j < B.naxis; ++j) cross3(A.axis[i], B.axis[j], cand[nc++]);
  bool found = false;
  depth = -1.0;
  double hi_best = 0.0, lo_best = 0.0;
  for (int c = 0; c < nc; ++c) {
    const double len2 = dot3(cand[c], cand[c]);
    if (len2 < 1e-20) continue;   // parallel edges: no facet of their own
    const double inv = 1.0 / sqrt(len2);
    const double u[3] = {inv * cand[c][0], inv * cand[c][1], inv * cand[c][2]};
    // h_D(u) = max_a u.a - min_b u.b and h_D(-u) = max_b u.b - min_a u.a from one projection
    double alo, ahi, blo, bhi;
    project(A, u, alo, ahi);
    project(B, u, blo, bhi);
    for (int sgn = 0; sgn < 2; ++sgn) {
      const double h = sgn ? bhi - alo : ahi - blo;
      if (!found || h < depth) {
        found = true;
        depth = h;
        for (int k = 0; k < 3; ++k) m[k] = sgn ? -u[k] : u[k];
        hi_best = sgn ? -alo : ahi;   // max over A of m.a
        lo_best = sgn ? -bhi : blo;   // min over B of m.b
      }
    }
  }
  if (depth < 0.0) return;
  // the support features of A along m and of B along -m
  const double tol = 1e-9 * (1.0 + fabs(hi_best) + fabs(lo_best));
  int fa[C::kMax], fb[C::kMax], na = 0, nb = 0;
  for (int i = 0; i < A.nv; ++i)
    if (dot3(m, A.v[i]) >= hi_best - tol) fa[na++] = i;
  for (int j = 0; j < B.nv; ++j)
    if (dot3(m, B.v[j]) <= lo_best + tol) fb[nb++] = j;
  if (na == 1) {
    copy3(A.v[fa[0]], pa);
    for (int k = 0; k < 3; ++k) pb[k] = pa[k] - depth * m[k];
  } else if (nb == 1) {
    copy3(B.v[fb[0]], pb);
    for (int k = 0; k < 3; ++k) pa[k] = pb[k] + depth * m[k];
  } else if (na == 2 && nb == 2) {
    seg_seg(A.v[fa[0]], A.v[fa[1]], B.v[fb[0]], B.v[fb[1]], pa, pb);
  } else {
    // an edge or face against a face: the witness pairs form a set; take the centroid of B's
    // feature and its partner on A
    for (int k = 0; k < 3; ++k) {
      double s = 0.0;
      for (int j = 0; j < nb; ++j) s += B.v[fb[j]][k];
      pb[k] = s / nb;
      pa[k] = pb[k] + depth * m[k];
    }
  }
}

// ------------------------------------------------------------------------------------------ EPA
// Overlapping cores with a hull on either side have no short list of candidate axes; their
// nearest facet of D is found by the expanding polytope (van den Bergen 2001): start from GJK's
// tetrahedron around the origin and repeatedly push out the face nearest the origin by the support
// point along its normal, replacing the faces that point sees by a fan from it to their horizon.
constexpr int kEpaMaxV = 64;
constexpr int kEpaMaxF = 128;
constexpr int kEpaMaxE = 96;
constexpr int kEpaMaxIter = 64;

struct Polytope {
  int nv, nf;
  double w[kEpaMaxV][3];
  int ia[kEpaMaxV], ib[kEpaMaxV];
  int f[kEpaMaxF][3];
  double n[kEpaMaxF][3];   // unit outward normal
  double d[kEpaMaxF];      // distance of the face's plane from the origin (>= 0 up to rounding)
};

// Face slot k = (i, j, l), counter-clockwise seen from outside; false for a face of zero area.
DS_HDI bool epa_face(Polytope& P, int k, int i, int j, int l) {
  double e1[3], e2[3], nr[3];
  sub3(P.w[j], P.w[i], e1);
  sub3(P.w[l], P.w[i], e2);
  cross3(e1, e2, nr);
  const double len = sqrt(dot3(nr, nr));
  if (!(len > 1e-15 * sqrt(dot3(e1, e1) * dot3(e2, e2)))) return false;
  P.f[k][0] = i;
  P.f[k][1] = j;
  P.f[k][2] = l;
  for (int c = 0; c < 3; ++c) P.n[k][c] = nr[c] / len;
  P.d[k] = dot3(P.n[k], P.w[i]);
  return true;
}

DS_HDI int epa_nearest(const Polytope& P) {
  int best = 0;
  for (int k = 1; k < P.nf; ++k)
    if (P.d[k] < P.d[best]) best = k;
  return best;
}

// A tetrahedron of support points around the origin, for overlapping cores where GJK stopped on
// the origin before forming one (e.g. identical cores at one pose, whose first support difference
// is the origin itself): support points along the four tetrahedral directions, then, while a face
// separates the origin from the opposite vertex, that vertex replaced by the support point along
// the face's outward normal (GJK's intersection iteration).  Returns false when D is flat, the
// origin is not strictly inside it, or 64 replacements do not enclose it.
template <class C>
DS_HDI bool enclose_origin(const C& A, const C& B, Simplex& t) {
  const double dirs[4][3] = {{1.0, 1.0, 1.0}, {1.0, -1.0, -1.0}, {-1.0, 1.0, -1.0}, {-1.0, -1.0, 1.0}};
  double scale = 0.0;
  for (int i = 0; i < 4; ++i) {
    const double neg[3] = {-dirs[i][0], -dirs[i][1], -dirs[i][2]};
    t.ia[i] = support(A, dirs[i]);
    t.ib[i] = support(B, neg);
    sub3(A.v[t.ia[i]], B.v[t.ib[i]], t.w[i]);
    scale = fmax(scale, sqrt(dot3(t.w[i], t.w[i])));
  }
  t.n = 4;
  const int F[4][4] = {{0, 1, 2, 3}, {0, 1, 3, 2}, {0, 2, 3, 1}, {1, 2, 3, 0}};
  for (int it = 0; it < kEpaMaxIter; ++it) {
    int out_face = -1;
    double dir[3] = {0.0, 0.0, 0.0};
    for (int f = 0; f < 4 && out_face < 0; ++f) {
      const double *wi = t.w[F[f][0]], *wj = t.w[F[f][1]], *wk = t.w[F[f][2]], *wo = t.w[F[f][3]];
      double e1[3], e2[3], nrm[3], eo[3];
      sub3(wj, wi, e1);
      sub3(wk, wi, e2);
      cross3(e1, e2, nrm);
      sub3(wo, wi, eo);
      const double sd = dot3(nrm, eo), so = -dot3(nrm, wi);
      if (fabs(sd) <= 1e-9 * sqrt(dot3(nrm, nrm) * dot3(eo, eo))) {   // flat
        t.n = 0;
        return false;
      }
      if (so * sd < 0.0) {   // the origin lies beyond face f
        out_face = f;
        for (int c = 0; c < 3; ++c) dir[c] = sd > 0.0 ? -nrm[c] : nrm[c];
      }
    }
    if (out_face < 0) return true;
    const double neg[3] = {-dir[0], -dir[1], -dir[2]};
    const int ia = support(A, dir), ib = support(B, neg);
    double w[3];
    sub3(A.v[ia], B.v[ib], w);
    // the origin is beyond the face: unless the support point passes it, D misses the origin
    if (dot3(dir, w) <= 1e-12 * scale * sqrt(dot3(dir, dir))) {
      t.n = 0;
      return false;
    }
    const int o = F[out_face][3];
    copy3(w, t.w[o]);
    t.ia[o] = ia;
    t.ib[o] = ib;
  }
  t.n = 0;
  return false;
}

// Penetration of overlapping cores from GJK's tetrahedron tet around the origin: depth, the unit
// axis m from A to B (moving A by -depth m separates the cores) and the witness points pa, pb with
// pa - pb = depth m (the projection of the origin on the nearest facet, in barycentric weights of
// its triangle).  Stops when the support point along the nearest face's normal adds less than
// 1e-12 (relative to the coordinates) to its distance.  Returns false when the polytope runs out
// of its 64 vertices, 128 faces or 96 horizon edges, or a new face has zero area.
template <class C>
DS_HDI bool epa(const C& A, const C& B, const Simplex& tet, double& depth, double* m, double* pa,
                double* pb) {
  Polytope P;
  P.nv = 4;
  P.nf = 0;
  double scale = 0.0;
  for (int i = 0; i < 4; ++i) {
    copy3(tet.w[i], P.w[i]);
    P.ia[i] = tet.ia[i];
    P.ib[i] = tet.ib[i];
    scale = fmax(scale, sqrt(dot3(P.w[i], P.w[i])));
  }
  const double tol = 1e-12 * fmax(scale, 1e-300);
  const int F[4][4] = {{0, 1, 2, 3}, {0, 1, 3, 2}, {0, 2, 3, 1}, {1, 2, 3, 0}};
  for (int f = 0; f < 4; ++f) {
    int i = F[f][0], j = F[f][1], l = F[f][2];
    double e1[3], e2[3], nr[3], eo[3];
    sub3(P.w[j], P.w[i], e1);
    sub3(P.w[l], P.w[i], e2);
    cross3(e1, e2, nr);
    sub3(P.w[F[f][3]], P.w[i], eo);
    if (dot3(nr, eo) > 0.0) {   // make the normal point away from the opposite vertex
      const int t = j;
      j = l;
      l = t;
    }
    if (!epa_face(P, P.nf, i, j, l)) return false;
    ++P.nf;
  }
  int edges[kEpaMaxE][2];
  for (int it = 0; it < kEpaMaxIter; ++it) {
    const int best = epa_nearest(P);
    const double* nb = P.n[best];
    const double neg[3] = {-nb[0], -nb[1], -nb[2]};
    const int ia = support(A, nb), ib = support(B, neg);
    bool dup = false;
    for (int v = 0; v < P.nv; ++v) dup = dup || (P.ia[v] == ia && P.ib[v] == ib);
    double w[3];
    sub3(A.v[ia], B.v[ib], w);
    if (dup || dot3(nb, w) - P.d[best] <= tol) break;
    if (P.nv == kEpaMaxV) return false;
    const int nw = P.nv++;
    copy3(w, P.w[nw]);
    P.ia[nw] = ia;
    P.ib[nw] = ib;
    // remove the faces that see w; their edges not shared by two of them form the horizon
    int ne = 0, kept = 0;
    for (int k = 0; k < P.nf; ++k) {
      double rel[3];
      sub3(w, P.w[P.f[k][0]], rel);
      if (dot3(P.n[k], rel) > 0.0) {
        for (int e = 0; e < 3; ++e) {
          const int a = P.f[k][e], b = P.f[k][(e + 1) % 3];
          int found = -1;
          for (int x = 0; x < ne; ++x)
            if (edges[x][0] == b && edges[x][1] == a) found = x;
          if (found >= 0) {
            --ne;
            edges[found][0] = edges[ne][0];
            edges[found][1] = edges[ne][1];
          } else {
            if (ne == kEpaMaxE) return false;
            edges[ne][0] = a;
            edges[ne][1] = b;
            ++ne;
          }
        }
      } else {
        if (kept != k) {
          for (int c = 0; c < 3; ++c) {
            P.f[kept][c] = P.f[k][c];
            P.n[kept][c] = P.n[k][c];
          }
          P.d[kept] = P.d[k];
        }
        ++kept;
      }
    }
    P.nf = kept;
    if (ne < 3) return false;
    for (int x = 0; x < ne; ++x) {
      if (P.nf == kEpaMaxF) return false;
      if (!epa_face(P, P.nf, edges[x][0], edges[x][1], nw)) return false;
      ++P.nf;
    }
  }
  const int best = epa_nearest(P);
  depth = P.d[best];
  copy3(P.n[best], m);
  // barycentric weights of y = depth m in the face's triangle (a, b, c)
  const int* fv = P.f[best];
  double v0[3], v1[3], v2[3];
  sub3(P.w[fv[1]], P.w[fv[0]], v0);
  sub3(P.w[fv[2]], P.w[fv[0]], v1);
  for (int c = 0; c < 3; ++c) v2[c] = depth * m[c] - P.w[fv[0]][c];
  const double d00 = dot3(v0, v0), d01 = dot3(v0, v1), d11 = dot3(v1, v1);
  const double d20 = dot3(v2, v0), d21 = dot3(v2, v1);
  const double den = d00 * d11 - d01 * d01;
  const double lb = (d11 * d20 - d01 * d21) / den, lc = (d00 * d21 - d01 * d20) / den;
  const double l[3] = {1.0 - lb - lc, lb, lc};
  for (int c = 0; c < 3; ++c) {
    pa[c] = 0.0;
    pb[c] = 0.0;
    for (int k = 0; k < 3; ++k) {
      pa[c] += l[k] * A.v[P.ia[fv[k]]][c];
      pb[c] += l[k] * B.v[P.ib[fv[k]]][c];
    }
  }
  return true;
}

// Collision detection of shape A (type, size, pose) and shape B (hull vertices from the pool hv
// of n_hv vertices).  Writes DS_COLLIDE_OUT numbers: phi, c[3], n[3], t1[3], t2[3], the witness
// points on the surfaces sa[3], sb[3].  An unknown type, a bad hull range, or a hull penetration
// the expanding polytope cannot resolve gives NaN throughout.  kHulls = false compiles the form
// without hulls (a hull is then a bad range), whose per-thread state is a tenth of the other's.
template <bool kHulls = true>
DS_HDI void collide(int type_a, const double* size_a, const double* pose_a, int type_b,
                    const double* size_b, const double* pose_b, const double* hv, int n_hv, double* out) {
  using C = typename std::conditional<kHulls, Core, BoxCore>::type;
  C A, B;
  if (!make_core(type_a, size_a, pose_a, pose_a + 9, hv, n_hv, A) ||
      !make_core(type_b, size_b, pose_b, pose_b + 9, hv, n_hv, B)) {
    for (int k = 0; k < DS_COLLIDE_OUT; ++k) out[k] = nan("");
    return;
  }
  double d, pa[3], pb[3], n[3];
  const bool hull = A.kind == kHull || B.kind == kHull;
  const bool has_box = !hull && (A.kind == kBox || B.kind == kBox);
  double depth = -1.0, m[3] = {0.0, 0.0, 1.0};
  // with a box (and no hull), the separating-axis test decides overlap exactly; GJK measures
  // separated cores
  if (has_box) penetration(A, B, depth, m, pa, pb);
  if (has_box && depth >= 0.0) {
    d = -depth;
    copy3(m, n);
  } else {
    Simplex tet;
    const bool overlap = gjk(A, B, pa, pb, &tet);
    double diff[3];
    sub3(pb, pa, diff);
    d = sqrt(dot3(diff, diff));
    if (!overlap && d > 0.0) {
      for (int k = 0; k < 3; ++k) n[k] = diff[k] / d;
    } else if (has_box) {
      // GJK met the origin although an axis separates the cores (rounding in a near-degenerate
      // simplex): the separating axis and its gap stand in
      d = -depth;
      copy3(m, n);
      for (int k = 0; k < 3; ++k) pb[k] = pa[k] + d * n[k];
    } else if (kHulls && hull && (tet.n == 4 || enclose_origin(A, B, tet))) {
      if constexpr (kHulls) {
        if (!epa(A, B, tet, depth, n, pa, pb)) {
          for (int k = 0; k < DS_COLLIDE_OUT; ++k) out[k] = nan("");
          return;
        }
      }
      d = -depth;
    } else {
      // touching cores (within 1e-12, no tetrahedron of D strictly around the origin), or
      // crossing point and segment cores: no normal; take the world z axis
      d = 0.0;
      n[0] = 0.0; n[1] = 0.0; n[2] = 1.0;
    }
  }
  double sa[3], sb[3];
  for (int k = 0; k < 3; ++k) {
    sa[k] = pa[k] + A.r * n[k];
    sb[k] = pb[k] - B.r * n[k];
  }
  // tangent axes: t1 = normalize(e - (n.e) n), e = e_x (e_y when |n_x| > 0.9); t2 = n x t1
  const bool use_y = fabs(n[0]) > 0.9;
  const double e[3] = {use_y ? 0.0 : 1.0, use_y ? 1.0 : 0.0, 0.0};
  const double ne = dot3(n, e);
  double t1[3] = {e[0] - ne * n[0], e[1] - ne * n[1], e[2] - ne * n[2]};
  const double it = 1.0 / sqrt(dot3(t1, t1));
  for (int k = 0; k < 3; ++k) t1[k] *= it;
  double t2[3];
  cross3(n, t1, t2);
  out[0] = d - A.r - B.r;
  for (int k = 0; k < 3; ++k) {
    out[1 + k] = 0.5 * (sa[k] + sb[k]);
    out[4 + k] = n[k];
    out[7 + k] = t1[k];
    out[10 + k] = t2[k];
    out[13 + k] = sa[k];
    out[16 + k] = sb[k];
  }
}

// ------------------------------------------------------------- randomized-smoothing derivative
// The pose (R row-major, p) moved by sgn times the world-frame twist xi = (u, w) (linear, then
// angular about the world origin): x -> exp([w]) x + V(w) u, so R' = exp([w]) R and
// p' = exp([w]) p + V(w) u, with exp([w]) = I + sin(t)/t W + (1 - cos t)/t^2 W^2 (Rodrigues) and
// V(w) = I + (1 - cos t)/t^2 W + (t - sin t)/t^3 W^2, t = |w|, W = [w]x (I + W and I + W/2 below
// t = 1e-12).
DS_HDI void twist_pose(const double* pose, const double* xi, double sgn, double* out) {
  const double u[3] = {sgn * xi[0], sgn * xi[1], sgn * xi[2]};
  const double w[3] = {sgn * xi[3], sgn * xi[4], sgn * xi[5]};
  const double t = sqrt(dot3(w, w));
  const double W[3][3] = {{0.0, -w[2], w[1]}, {w[2], 0.0, -w[0]}, {-w[1], w[0], 0.0}};
  double W2[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) W2[i][j] = W[i][0] * W[0][j] + W[i][1] * W[1][j] + W[i][2] * W[2][j];
  double a = 1.0, b = 0.0, c = 0.5, d = 0.0;
  if (t >= 1e-12) {
    a = sin(t) / t;
    b = (1.0 - cos(t)) / (t * t);
    c = b;
    d = (t - sin(t)) / (t * t * t);
  }
  double E[3][3], V[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      const double id = i == j ? 1.0 : 0.0;
      E[i][j] = id + a * W[i][j] + b * W2[i][j];
      V[i][j] = id + c * W[i][j] + d * W2[i][j];
    }
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j)
      out[3 * i + j] = E[i][0] * pose[j] + E[i][1] * pose[3 + j] + E[i][2] * pose[6 + j];
    out[9 + i] = E[i][0] * pose[9] + E[i][1] * pose[10] + E[i][2] * pose[11] +
                 V[i][0] * u[0] + V[i][1] * u[1] + V[i][2] * u[2];
  }
}

// App. C's zero-order randomized-smoothing estimate of the derivative of f = (phi, c, n) (the
// first 7 outputs of collide) with respect to the world-frame twists of A's and B's poses:
// J = 1 / (2 S sigma^2) sum_s (f(+eps_s) - f(-eps_s)) eps_s^T, eps_s = (A's (u, w), B's (u, w))
// the caller's samples (S x 12, drawn from N(0, sigma^2 I)).  J is 7 x 12, row-major.
template <bool kHulls = true>
DS_HDI void smoothing_jacobian(int type_a, const double* size_a, const double* pose_a, int type_b,
                               const double* size_b, const double* pose_b, const double* hv, int n_hv,
                               int samples, const double* eps, double sigma, double* J) {
  for (int k = 0; k < 84; ++k) J[k] = 0.0;
  double qa[12], qb[12], fp[DS_COLLIDE_OUT], fm[DS_COLLIDE_OUT];
  for (int s = 0; s < samples; ++s) {
    const double* e = eps + 12 * s;
    twist_pose(pose_a, e, 1.0, qa);
    twist_pose(pose_b, e + 6, 1.0, qb);
    collide<kHulls>(type_a, size_a, qa, type_b, size_b, qb, hv, n_hv, fp);
    twist_pose(pose_a, e, -1.0, qa);
    twist_pose(pose_b, e + 6, -1.0, qb);
    collide<kHulls>(type_a, size_a, qa, type_b, size_b, qb, hv, n_hv, fm);
    for (int i = 0; i < 7; ++i) {
      const double df = fp[i] - fm[i];
      for (int j = 0; j < 12; ++j) J[12 * i + j] += df * e[j];
    }
  }
  const double scale = 1.0 / (2.0 * sigma * sigma * samples);
  for (int k = 0; k < 84; ++k) J[k] *= scale;
}

}  // namespace cd
}  // namespace ds
