// App. C's contact-placement terms of the derivatives of a contact between two bodies (or a body
// and the fixed world), FP64, host- and device-callable; not yet called by the step kernels, whose
// contacts are primitive-versus-plane.
//
// A contact between bodies A and B has J_c v = E (cX_B V_B - cX_A V_A): the linear part (E) of the
// relative twist of B's and A's material points at the contact, in the contact frame (origin c,
// rotation Rc, Z along the normal from A to B); V_i = J_i v are the bodies' twists in their own
// coordinates and cX_i the motion transforms from body i to the contact frame.  When the contact
// placement moves with q (collision detection, 0M_c = CD(0M_A, 0M_B)), d(J_c v)/dq at fixed v and
// fixed body twists has, besides the bodies' own velocity change, the placement terms
//   sum_i sign_i E [ (cX_i V_i) x dc - cX_i (V_i x J_i) ],   dc = sum_i dCD/dM_i J_i,
// sign_A = -1, sign_B = +1, dc the local twist of the contact frame per unit dof velocity and
// dCD/dM_i (6 x 6) the local twist of the contact placement per local twist of body i's pose
// (M_i -> M_i exp(delta)).  The terms of d(J_c^T lambda)/dq follow by duality:
// <d(J_c^T lambda) dq, v> = <lambda, d(J_c v) dq> for every v.
//
// Vectors are (linear, angular); a body is given by its world pose (R row-major, p), its twist V
// and Jacobian J (6 x nv, row-major) in its own coordinates and dCD/dM (6 x 6, row-major); R ==
// nullptr stands for the fixed world (no twist, no Jacobian).  dCD/dM_i itself comes from
// dcd_dbody (central differences of the collision detection in the body's local twist) or, as the
// paper takes it, dcd_dbody_smoothed (its randomized-smoothing estimate).
#pragma once
#include "ds_collision.cuh"
#include "ds_common.cuh"

namespace ds {
namespace cd {

// o = cX m: the motion vector m of the body frame (R, p) expressed in the contact frame (Rc, c),
// cX = [E^T, -E^T [r]x; 0, E^T] with E = R^T Rc and r = R^T (c - p).
DS_HDI void to_contact(const double* R, const double* p, const double* Rc, const double* c, const double* m,
                       double* o) {
  double d[3] = {c[0] - p[0], c[1] - p[1], c[2] - p[2]};
  double r[3], E[3][3];
  for (int i = 0; i < 3; ++i) {
    r[i] = R[i] * d[0] + R[3 + i] * d[1] + R[6 + i] * d[2];   // R^T (c - p)
    for (int j = 0; j < 3; ++j) E[i][j] = R[i] * Rc[j] + R[3 + i] * Rc[3 + j] + R[6 + i] * Rc[6 + j];
  }
  double rw[3], lin[3];
  cross3(r, m + 3, rw);
  for (int i = 0; i < 3; ++i) lin[i] = m[i] - rw[i];
  for (int j = 0; j < 3; ++j) {
    o[j] = E[0][j] * lin[0] + E[1][j] * lin[1] + E[2][j] * lin[2];
    o[3 + j] = E[0][j] * m[3] + E[1][j] * m[4] + E[2][j] * m[5];
  }
}

// out (3 x nv, row-major) = J_c of the pair: column k is E (cX_B J_B[:, k] - cX_A J_A[:, k]).
DS_HD inline void pair_jc(int nv, const double* Rc, const double* c, const double* Ra, const double* pa,
                          const double* Ja, const double* Rb, const double* pb, const double* Jb, double* out) {
  for (int k = 0; k < nv; ++k) {
    double acc[3] = {0.0, 0.0, 0.0};
    const double* R[2] = {Ra, Rb};
    const double* P[2] = {pa, pb};
    const double* J[2] = {Ja, Jb};
    for (int b = 0; b < 2; ++b) {
      if (!R[b]) continue;
      const double jk[6] = {J[b][0 * nv + k], J[b][1 * nv + k], J[b][2 * nv + k],
                            J[b][3 * nv + k], J[b][4 * nv + k], J[b][5 * nv + k]};
      double x[6];
      to_contact(R[b], P[b], Rc, c, jk, x);
      for (int i = 0; i < 3; ++i) acc[i] += (b == 0 ? -1.0 : 1.0) * x[i];
    }
    for (int i = 0; i < 3; ++i) out[i * nv + k] = acc[i];
  }
}

// o = dCD/dM J[:, k] (6 x 6 times column k of a 6 x nv Jacobian).
DS_HDI void dcd_column(const double* dcd, const double* J, int nv, int k, double* o) {
  for (int i = 0; i < 6; ++i) {
    double s = 0.0;
    for (int j = 0; j < 6; ++j) s += dcd[6 * i + j] * J[j * nv + k];
    o[i] = s;
  }
}

// out (3 x nv, row-major) = the placement terms of d(J_c v)/dq for the body twists Va, Vb (App. C).
DS_HD inline void appc_dJcv_dq(int nv, const double* Rc, const double* c, const double* Ra, const double* pa,
                               const double* Va, const double* Ja, const double* dcda, const double* Rb,
                               const double* pb, const double* Vb, const double* Jb, const double* dcdb,
                               double* out) {
  const double* R[2] = {Ra, Rb};
  const double* P[2] = {pa, pb};
  const double* V[2] = {Va, Vb};
  const double* J[2] = {Ja, Jb};
  const double* D[2] = {dcda, dcdb};
  const double sign[2] = {-1.0, 1.0};
  double W[2][6];   // cX_i V_i
  for (int b = 0; b < 2; ++b)
    if (R[b]) to_contact(R[b], P[b], Rc, c, V[b], W[b]);
  for (int k = 0; k < nv; ++k) {
    double dc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int b = 0; b < 2; ++b) {
      if (!R[b]) continue;
      double t[6];
      dcd_column(D[b], J[b], nv, k, t);
      for (int i = 0; i < 6; ++i) dc[i] += t[i];
    }
    double acc[3] = {0.0, 0.0, 0.0};
    for (int b = 0; b < 2; ++b) {
      if (!R[b]) continue;
      // (cX V) x dc, linear part: w x dc_lin + v x dc_ang
      double t1[3], t2[3];
      cross3(W[b] + 3, dc, t1);
      cross3(W[b], dc + 3, t2);
      // cX (V x J_k): V x J_k = (w x j_lin + v x j_ang, w x j_ang)
      const double jk[6] = {J[b][0 * nv + k], J[b][1 * nv + k], J[b][2 * nv + k],
                            J[b][3 * nv + k], J[b][4 * nv + k], J[b][5 * nv + k]};
      double vj[6], a1[3], a2[3];
      cross3(V[b] + 3, jk, a1);
      cross3(V[b], jk + 3, a2);
      for (int i = 0; i < 3; ++i) vj[i] = a1[i] + a2[i];
      cross3(V[b] + 3, jk + 3, vj + 3);
      double xvj[6];
      to_contact(R[b], P[b], Rc, c, vj, xvj);
      for (int i = 0; i < 3; ++i) acc[i] += sign[b] * (t1[i] + t2[i] - xvj[i]);
    }
    for (int i = 0; i < 3; ++i) out[i * nv + k] = acc[i];
  }
}

// out (nv x nv, row-major) = the placement terms of d(J_c^T lambda)/dq: row j is lambda^T times
// the terms of d(J_c e_j)/dq, i.e. appc_dJcv_dq with the body twists J_i e_j.  scratch holds
// 3 nv numbers.
DS_HD inline void appc_dJctlam_dq(int nv, const double* lam, const double* Rc, const double* c, const double* Ra,
                                  const double* pa, const double* Ja, const double* dcda, const double* Rb,
                                  const double* pb, const double* Jb, const double* dcdb, double* scratch,
                                  double* out) {
  for (int j = 0; j < nv; ++j) {
    double va[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0}, vb[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int i = 0; i < 6; ++i) {
      if (Ra) va[i] = Ja[i * nv + j];
      if (Rb) vb[i] = Jb[i * nv + j];
    }
    appc_dJcv_dq(nv, Rc, c, Ra, pa, va, Ja, dcda, Rb, pb, vb, Jb, dcdb, scratch);
    for (int k = 0; k < nv; ++k)
      out[j * nv + k] = lam[0] * scratch[k] + lam[1] * scratch[nv + k] + lam[2] * scratch[2 * nv + k];
  }
}

// The world pose (12 numbers: R row-major, p) of a shape at offset (E row-major, r) on a body at
// world pose M = (R, p): (R E, p + R r).
DS_HDI void shape_pose(const double* M, const double* off, double* o) {
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j)
      o[3 * i + j] = M[3 * i] * off[j] + M[3 * i + 1] * off[3 + j] + M[3 * i + 2] * off[6 + j];
    o[9 + i] = M[9 + i] + M[3 * i] * off[9] + M[3 * i + 1] * off[10] + M[3 * i + 2] * off[11];
  }
}

// f = the local twist of the contact placement when body i (which = 0: A, 1: B) moves by the local
// twist xi (M_i -> M_i exp(xi): R' = R exp([w]), p' = p + R V(w) u): (Rc^T (c' - c), vee of the
// antisymmetric part of Rc^T Rc' - I), with (Rc, c) the placement read from base (collide's
// outputs at the unmoved poses).  Returns false when the moved result is not finite.
DS_HD inline bool placement_twist(int type_a, const double* size_a, const double* Ma, const double* oa,
                                  int type_b, const double* size_b, const double* Mb, const double* ob,
                                  const double* hv, int n_hv, int which, const double* base, const double* xi,
                                  double* f) {
  const double ident[12] = {1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0};
  double ex[12], Mm[12], moved[12], other[12], r[DS_COLLIDE_OUT];
  twist_pose(ident, xi, 1.0, ex);
  shape_pose(which == 0 ? Ma : Mb, ex, Mm);   // (R E_x, p + R p_x)
  shape_pose(Mm, which == 0 ? oa : ob, moved);
  shape_pose(which == 0 ? Mb : Ma, which == 0 ? ob : oa, other);
  if (which == 0) collide(type_a, size_a, moved, type_b, size_b, other, hv, n_hv, r);
  else collide(type_a, size_a, other, type_b, size_b, moved, hv, n_hv, r);
  const double* axes[3] = {base + 7, base + 10, base + 4};   // rows of Rc^T: t1, t2, n
  const double* ax2[3] = {r + 7, r + 10, r + 4};
  const double dc[3] = {r[1] - base[1], r[2] - base[2], r[3] - base[3]};
  double W[3][3];   // Rc^T Rc' - I
  for (int a = 0; a < 3; ++a) {
    f[a] = dot3(axes[a], dc);
    for (int b = 0; b < 3; ++b) W[a][b] = dot3(axes[a], ax2[b]) - (a == b ? 1.0 : 0.0);
  }
  f[3] = 0.5 * (W[2][1] - W[1][2]);
  f[4] = 0.5 * (W[0][2] - W[2][0]);
  f[5] = 0.5 * (W[1][0] - W[0][1]);
  for (int k = 0; k < 6; ++k)
    if (!(f[k] - f[k] == 0.0)) return false;
  return true;
}

// dCD/dM_i (6 x 6, row-major) by central differences of the collision detection: column j is
// (f(+h e_j) - f(-h e_j)) / (2 h) for f of placement_twist, which = 0 for A, 1 for B.  Ma, Mb are
// the bodies' world poses (the identity for the fixed world), oa, ob the shapes' offsets on them;
// shapes, hulls as for collide.  Returns false when a collision result is not finite.
DS_HD inline bool dcd_dbody(int type_a, const double* size_a, const double* Ma, const double* oa, int type_b,
                            const double* size_b, const double* Mb, const double* ob, const double* hv, int n_hv,
                            int which, double h, double* out) {
  double pa[12], pb[12], base[DS_COLLIDE_OUT];
  shape_pose(Ma, oa, pa);
  shape_pose(Mb, ob, pb);
  collide(type_a, size_a, pa, type_b, size_b, pb, hv, n_hv, base);
  for (int j = 0; j < 6; ++j) {
    double xp[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0}, xm[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0}, fp[6], fm[6];
    xp[j] = h;
    xm[j] = -h;
    if (!placement_twist(type_a, size_a, Ma, oa, type_b, size_b, Mb, ob, hv, n_hv, which, base, xp, fp) ||
        !placement_twist(type_a, size_a, Ma, oa, type_b, size_b, Mb, ob, hv, n_hv, which, base, xm, fm))
      return false;
    for (int i = 0; i < 6; ++i) out[6 * i + j] = (fp[i] - fm[i]) / (2.0 * h);
  }
  return true;
}

// dCD/dM_i by App. C's zero-order randomized smoothing: with the caller's local twists eps_s of
// body i (samples x 6, drawn from N(0, sigma^2 I)), 1 / (2 S sigma^2) sum_s (f(+eps_s) - f(-eps_s))
// eps_s^T for f of placement_twist.  Returns false when a collision result is not finite.
DS_HD inline bool dcd_dbody_smoothed(int type_a, const double* size_a, const double* Ma, const double* oa,
                                     int type_b, const double* size_b, const double* Mb, const double* ob,
                                     const double* hv, int n_hv, int which, int samples, const double* eps,
                                     double sigma, double* out) {
  double pa[12], pb[12], base[DS_COLLIDE_OUT];
  shape_pose(Ma, oa, pa);
  shape_pose(Mb, ob, pb);
  collide(type_a, size_a, pa, type_b, size_b, pb, hv, n_hv, base);
  for (int k = 0; k < 36; ++k) out[k] = 0.0;
  for (int s = 0; s < samples; ++s) {
    const double* e = eps + 6 * s;
    const double em[6] = {-e[0], -e[1], -e[2], -e[3], -e[4], -e[5]};
    double fp[6], fm[6];
    if (!placement_twist(type_a, size_a, Ma, oa, type_b, size_b, Mb, ob, hv, n_hv, which, base, e, fp) ||
        !placement_twist(type_a, size_a, Ma, oa, type_b, size_b, Mb, ob, hv, n_hv, which, base, em, fm))
      return false;
    for (int i = 0; i < 6; ++i)
      for (int j = 0; j < 6; ++j) out[6 * i + j] += (fp[i] - fm[i]) * e[j];
  }
  const double scale = 1.0 / (2.0 * sigma * sigma * samples);
  for (int k = 0; k < 36; ++k) out[k] *= scale;
  return true;
}

}  // namespace cd
}  // namespace ds
