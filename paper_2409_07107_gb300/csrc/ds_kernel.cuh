// One environment per thread: forward step, NCP solve and implicit derivatives.
//
// Template parameters: NB bodies, NV velocity dofs, NS contact slots (all exact for the model
// class), T = the arithmetic type of the bulk work (double: the plain FP64 method; float: the
// mixed-precision form, whose kinematics, contact detection, NCP polish, residual check and
// reduced implicit system stay in double).
//
// Spatial algebra is done in world axes at the world origin, which makes composite inertias plain
// sums and lets a perturbation of joint j act on its whole subtree as one rigid twist.  This is a
// different formulation from the body-frame recursions of the CPU oracle, on purpose.
#pragma once
#include "ds_common.cuh"

namespace ds {

template <typename T>
DS_HDI void proj_cone(const T* x, T mu, T* o) {
  const T nt = sqrt(x[0] * x[0] + x[1] * x[1]);
  if (nt <= mu * x[2]) { o[0] = x[0]; o[1] = x[1]; o[2] = x[2]; return; }
  if (mu * nt <= -x[2]) { o[0] = T(0); o[1] = T(0); o[2] = T(0); return; }
  const T s = (mu * nt + x[2]) / (T(1) + mu * mu);
  const T k = mu * s / nt;
  o[0] = k * x[0]; o[1] = k * x[1]; o[2] = s;
}

// The contact problem of one env: Eq. 1 data (G, g, mu over the active contacts), the solution
// lambda, and the FP64 factorisation workspace shared by the Newton steps and the implicit solve.
template <int NS, typename T>
struct Ncp {
  static constexpr int NC3 = 3 * NS;
  static constexpr bool kDouble = std::is_same<T, double>::value;
  int na;                                    // active contacts
  double mu[NS];
  T Gt[NC3][NC3];                            // Delassus matrix in the bulk type
  double Gd_[kDouble ? 1 : NC3][kDouble ? 1 : NC3];
  T gt[NC3];
  double gd[NC3], lam[NC3];
  LUcp<NC3 + NS, NC3> lu;

  DS_HDI double G(int i, int j) const {
    if constexpr (kDouble) return Gt[i][j]; else return Gd_[i][j];
  }
};

// Maximum of two values that are >= 0 (or NaN), taken on their bit patterns: for non-negative IEEE
// numbers the order of the patterns as signed integers is the numeric order.  Unlike fmax, which
// drops a NaN operand, a (positive) NaN compares above every number, so an ADMM convergence test
// on a NaN residual fails, as the oracle's does.
DS_HDI double nonneg_max(double a, double b) {
#ifdef __CUDA_ARCH__
  return __double_as_longlong(a) > __double_as_longlong(b) ? a : b;
#else
  long long ia, ib;
  memcpy(&ia, &a, sizeof ia);
  memcpy(&ib, &b, sizeof ib);
  return ia > ib ? a : b;
#endif
}

DS_HDI float nonneg_max(float a, float b) {
#ifdef __CUDA_ARCH__
  return __float_as_int(a) > __float_as_int(b) ? a : b;
#else
  int ia, ib;
  memcpy(&ia, &a, sizeof ia);
  memcpy(&ib, &b, sizeof ib);
  return ia > ib ? a : b;
#endif
}

// Pieces of the ADMM iteration with the divisions and square roots of the plain projection
// replaced by one reciprocal square root and precomputed reciprocals (1/rho, 1/(1 + mu^2)): the
// same mathematics with a shorter dependent chain (FP64 division and sqrt are long sequences).
template <typename T>
DS_HDI void norm_and_inv(T a, T b, T& n, T& inv) {
  const T t2 = a * a + b * b;
  if (t2 > T(0)) { inv = rsqrt(t2); n = t2 * inv; }
  else { inv = T(0); n = T(0); }
}

template <typename T>
DS_HDI void proj_cone_fast(const T* x, T mu, T inv1pmu2, T* o) {
  T nt, inv;
  norm_and_inv(x[0], x[1], nt, inv);
  if (nt <= mu * x[2]) { o[0] = x[0]; o[1] = x[1]; o[2] = x[2]; return; }
  if (mu * nt <= -x[2]) { o[0] = T(0); o[1] = T(0); o[2] = T(0); return; }
  const T s = (mu * nt + x[2]) * inv1pmu2;
  const T k = mu * s * inv;
  o[0] = k * x[0]; o[1] = k * x[1]; o[2] = s;
}

template <int NB, int NV, int NS, typename T>
struct Env : Ncp<NS, T> {
  static constexpr int NC3 = 3 * NS;
  static constexpr bool kDouble = std::is_same<T, double>::value;
  double q[NV + 1];                          // joint positions (FP64)
  double R[NB][9], P[NB][3];                 // world placement of every body (FP64)
  T S[NV][6];                                // world motion subspace of every dof
  T I[NB][10];                               // world spatial inertia of every body
  T V[NB][6], A[NB][6], VJ[NB][6], IV[NB][6], IA[NB][6], Fc[NB][6];
  T L[NV * (NV + 1) / 2];                    // factor of M = L^T L (packed lower, tree-sparse)
  T v[NV], tau[NV], vdf[NV], vf[NV], vn[NV], astar[NV];
  int slot[NS], body[NS];
  T x[NS][3], c[NS][3], f[NS][3];            // body point, contact point, contact force (world)
  double cx_d[NS][3];                        // contact point in FP64
  double phi[NS];                            // signed distance of the active contact (FP64)
  T fr[3][3];                                // contact frame rows t1, t2, n
  T Jc[NC3][NV];
  T Y[NC3][NV];                              // rows of M^-1 J_c^T
  // mixed form: J_c, M's factor and M^-1 J_c^T in FP64 (G must keep the exact null space of J_c^T)
  double Jd_[kDouble ? 1 : NC3][kDouble ? 1 : NV];
  double Yd_[kDouble ? 1 : NC3][kDouble ? 1 : NV];
  double Ld_[kDouble ? 1 : NV * (NV + 1) / 2];
  int mode[NS];
  double margin;
};

// ------------------------------------------------------------------------- NCP helpers (FP64)

template <class E>
DS_HD double ncp_residual(const E& s, const double* lam) {
  const int m = 3 * s.na;
  double r = 0.0;
  for (int i = 0; i < s.na; ++i) {
    double sg[3];
    for (int k = 0; k < 3; ++k) {
      double t = s.gd[3 * i + k];
      for (int j = 0; j < m; ++j) t += s.G(3 * i + k, j) * lam[j];
      sg[k] = t;
    }
    const double* l = lam + 3 * i;
    double w[3] = {sg[0], sg[1], sg[2] + s.mu[i] * sqrt(sg[0] * sg[0] + sg[1] * sg[1])};
    double p[3];
    proj_cone(l, s.mu[i], p);
    r = fmax(r, sqrt((l[0] - p[0]) * (l[0] - p[0]) + (l[1] - p[1]) * (l[1] - p[1]) + (l[2] - p[2]) * (l[2] - p[2])));
    proj_cone(w, 1.0 / s.mu[i], p);
    r = fmax(r, sqrt((w[0] - p[0]) * (w[0] - p[0]) + (w[1] - p[1]) * (w[1] - p[1]) + (w[2] - p[2]) * (w[2] - p[2])));
    r = fmax(r, fabs(l[0] * w[0] + l[1] * w[1] + l[2] * w[2]));
  }
  return r;
}

// Contact modes (breaking / sticking / sliding) from sigma = G lambda + g and lambda (Sec. 3.2, with
// relative thresholds): sticking if |sigma| <= es; else breaking if sigma_N > es or lambda_N <= el; else
// sticking if the impulse is strictly inside the cone (then Eq. 1 forces sigma = 0); else sliding.
template <class E>
DS_HD double classify(const E& s, const double* lam, double es_rel, double el_rel, int* mode) {
  const int m = 3 * s.na;
  double gmax = 1.0, lmax = 1.0;
  for (int j = 0; j < m; ++j) { gmax = fmax(gmax, fabs(s.gd[j])); lmax = fmax(lmax, fabs(lam[j])); }
  const double es = es_rel * gmax, el = el_rel * lmax;
  double margin = 1e300;
  for (int i = 0; i < s.na; ++i) {
    double sg[3];
    for (int k = 0; k < 3; ++k) {
      double t = s.gd[3 * i + k];
      for (int j = 0; j < m; ++j) t += s.G(3 * i + k, j) * lam[j];
      sg[k] = t;
    }
    const double* l = lam + 3 * i;
    const double ns = sqrt(sg[0] * sg[0] + sg[1] * sg[1] + sg[2] * sg[2]);
    const double nst = sqrt(sg[0] * sg[0] + sg[1] * sg[1]);
    const double inside = s.mu[i] * l[2] - sqrt(l[0] * l[0] + l[1] * l[1]);
    if (ns <= es) {
      mode[i] = DS_MODE_STICKING;
      margin = fmin(margin, (es - ns) / es);
    } else if (sg[2] > es || l[2] <= el) {
      mode[i] = DS_MODE_BREAKING;
      margin = fmin(margin, sg[2] > es ? (sg[2] - es) / gmax : 0.0);
    } else if (inside > el) {
      mode[i] = DS_MODE_STICKING;
      margin = fmin(margin, inside / lmax);
    } else {
      mode[i] = DS_MODE_SLIDING;
      margin = fmin(margin, fmin(nst / gmax, l[2] / lmax));
    }
  }
  return margin;
}

// Eq. 1 with lambda = 0: sigma = g, and g + Gamma(g) = (g_T, g_N + mu |g_T|) lies in the dual cone
// exactly when g_N >= 0.  So when the free motion separates every active contact, lambda = 0 is a
// solution; it is the one the step takes (no impulse acts when nothing pushes into the plane),
// although the non-monotone De Saxce form can admit others.  False on NaN.
template <class E>
DS_HDI bool separating(const E& s) {
  bool sep = s.na > 0;
  for (int i = 0; i < s.na; ++i) sep = sep && s.gd[3 * i + 2] >= 0.0;
  return sep;
}

// Active-set update after a Newton solve that did not give an NCP solution: breaking + penetrating
// -> sticking; sticking/sliding + pulling -> breaking; sticking with the impulse outside the cone
// -> sliding; sliding that stopped -> sticking.
template <class E>
DS_HD bool reclassify(const E& s, const double* lam, int* mode, double es, double el, double delta) {
  const int m = 3 * s.na;
  bool changed = false;
  for (int i = 0; i < s.na; ++i) {
    double sg[3];
    for (int k = 0; k < 3; ++k) {
      double t = s.gd[3 * i + k];
      for (int j = 0; j < m; ++j) t += s.G(3 * i + k, j) * lam[j];
      sg[k] = t;
    }
    const double* l = lam + 3 * i;
    int nm = mode[i];
    if (mode[i] == DS_MODE_BREAKING) {
      if (sg[2] < -es) nm = DS_MODE_STICKING;
    } else if (mode[i] == DS_MODE_STICKING) {
      if (l[2] < -el) nm = DS_MODE_BREAKING;
      else if (s.mu[i] * l[2] - sqrt(l[0] * l[0] + l[1] * l[1]) < -delta) nm = DS_MODE_SLIDING;
    } else {
      if (l[2] < -el) nm = DS_MODE_BREAKING;
      else if (sqrt(sg[0] * sg[0] + sg[1] * sg[1]) < es) nm = DS_MODE_STICKING;
    }
    changed |= nm != mode[i];
    mode[i] = nm;
  }
  return changed;
}

// Newton on the mode equations (breaking: lambda_i = 0; sticking: sigma_i = 0; sliding:
// sigma_N = 0, lambda_T + mu lambda_N sigma_T/|sigma_T| = 0), plus mu lambda_N - |lambda_T| = 0 for
// the sticking contacts whose starting impulse lies within sat_delta of the cone boundary (with
// redundant contacts this picks, among the equivalent impulses, one that stays in the cone).
// FP64, minimum-norm steps of a rank-revealing LU.  The breaking contacts' equations fix their
// impulses at 0 exactly, so the system is solved in the unknowns of the other contacts only (the
// null space lies in those unknowns, hence the minimum-norm step is unchanged).  Stops when the
// residual is at rounding level or stops decreasing.
template <class E>
DS_HD void newton_modes(E& s, double* lam, const int* mode, int iters, double sat_delta) {
  const int m = 3 * s.na;
  double scale = 1.0;
  for (int j = 0; j < m; ++j) scale = fmax(scale, fabs(s.gd[j]));
  int sat[E::NC3 / 3], nsat = 0;
  int ucon[E::NC3 / 3], nuc = 0;             // non-breaking contacts (their impulses are unknown)
  for (int i = 0; i < s.na; ++i) {
    const double* l = lam + 3 * i;
    if (mode[i] == DS_MODE_BREAKING) {
      lam[3 * i] = 0.0; lam[3 * i + 1] = 0.0; lam[3 * i + 2] = 0.0;
      continue;
    }
    ucon[nuc++] = i;
    const double nt = sqrt(l[0] * l[0] + l[1] * l[1]);
    if (mode[i] == DS_MODE_STICKING && nt > 0.0 && s.mu[i] * l[2] - nt <= sat_delta) sat[nsat++] = i;
  }
  const int nu = 3 * nuc;
  if (nu == 0) return;
  const int rows = nu + nsat;
  double prev = 1e300;
  for (int it = 0; it < iters; ++it) {
    double sg[E::NC3], F[E::NC3 + E::NC3 / 3];
    for (int q = 0; q < nuc; ++q)
      for (int k = 0; k < 3; ++k) {
        const int r = 3 * ucon[q] + k;
        double t = s.gd[r];
        for (int p = 0; p < nuc; ++p)
          for (int kk = 0; kk < 3; ++kk) t += s.G(r, 3 * ucon[p] + kk) * lam[3 * ucon[p] + kk];
        sg[r] = t;
      }
    s.lu.r = rows;
    s.lu.c = nu;
    for (int r = 0; r < rows; ++r)
      for (int j = 0; j < nu; ++j) s.lu.a[r][j] = 0.0;
    for (int q = 0; q < nuc; ++q) {
      const int i = ucon[q], r0 = 3 * i, u0 = 3 * q;
      if (mode[i] == DS_MODE_STICKING) {
        for (int r = 0; r < 3; ++r) {
          F[u0 + r] = sg[r0 + r];
          for (int p = 0; p < nuc; ++p)
            for (int kk = 0; kk < 3; ++kk) s.lu.a[u0 + r][3 * p + kk] = s.G(r0 + r, 3 * ucon[p] + kk);
        }
      } else {
        const double ns = sqrt(sg[r0] * sg[r0] + sg[r0 + 1] * sg[r0 + 1]);
        const double u[2] = {sg[r0] / ns, sg[r0 + 1] / ns};
        const double mu = s.mu[i], ln = lam[r0 + 2];
        const double k = mu * ln / ns;
        for (int r = 0; r < 2; ++r) {
          F[u0 + r] = lam[r0 + r] + mu * ln * u[r];
          // k (I - u u^T) G_T, then [I2, mu u] on the contact's own columns
          for (int p = 0; p < nuc; ++p)
            for (int kk = 0; kk < 3; ++kk) {
              const int cj = 3 * ucon[p] + kk;
              s.lu.a[u0 + r][3 * p + kk] =
                  k * (((r == 0) - u[r] * u[0]) * s.G(r0, cj) + ((r == 1) - u[r] * u[1]) * s.G(r0 + 1, cj));
            }
          s.lu.a[u0 + r][u0 + r] += 1.0;
          s.lu.a[u0 + r][u0 + 2] += mu * u[r];
        }
        F[u0 + 2] = sg[r0 + 2];
        for (int p = 0; p < nuc; ++p)
          for (int kk = 0; kk < 3; ++kk) s.lu.a[u0 + 2][3 * p + kk] = s.G(r0 + 2, 3 * ucon[p] + kk);
      }
    }
    for (int qs = 0; qs < nsat; ++qs) {
      const int i = sat[qs], r0 = 3 * i;
      int q = 0;
      while (ucon[q] != i) ++q;
      const double nt = sqrt(lam[r0] * lam[r0] + lam[r0 + 1] * lam[r0 + 1]);
      F[nu + qs] = s.mu[i] * lam[r0 + 2] - nt;
      s.lu.a[nu + qs][3 * q] = -lam[r0] / nt;
      s.lu.a[nu + qs][3 * q + 1] = -lam[r0 + 1] / nt;
      s.lu.a[nu + qs][3 * q + 2] = s.mu[i];
    }
    double fmaxv = 0.0;
    for (int r = 0; r < rows; ++r) fmaxv = fmax(fmaxv, fabs(F[r]));
    if (!(fmaxv > 1e-15 * scale)) break;
    if (it >= 2 && !(fmaxv < 0.5 * prev)) break;        // not converging (wrong modes)
    prev = fmaxv;
    s.lu.factor(1e-13);
    s.lu.nullspace();
    double dx[E::NC3];
    s.lu.solve_mn(F, dx);
    for (int q = 0; q < nuc; ++q)
      for (int k = 0; k < 3; ++k) lam[3 * ucon[q] + k] -= dx[3 * q + k];
  }
}

// Over-relaxed ADMM on Eq. 1 in the bulk type (rho = 0.3 mean diag G, De Saxce term at the latest
// primal iterate, relaxation 1.6).  The x-step uses the explicit inverse K = (G + rho I)^-1 (one
// matrix-vector product, no dependent triangular solves), and G x is never formed: (G + rho I) x
// = rhs gives G x + g = rhs - rho x + g.  The per-contact pieces below are shared by the
// one-thread-per-env form and the one-lane-per-contact cooperative form, so both do the same
// arithmetic in the same order.
template <typename T>
DS_HDI void admm_rhs(T mu, const T* z, const T* y, const T* g, const T* sx, T rho, T* rhs) {
  T nt, inv;
  norm_and_inv(sx[0], sx[1], nt, inv);
  const T sd = mu * nt;
  rhs[0] = rho * z[0] - y[0] - g[0];
  rhs[1] = rho * z[1] - y[1] - g[1];
  rhs[2] = rho * z[2] - y[2] - g[2] - sd;
}

// Convergence of the ADMM iteration is tested every DS_ADMM_CHECK iterations (of the env's global
// iteration count): the residual bookkeeping and, in the cooperative form, its reductions over the
// env's lanes then stay off the other iterations.  FP64 instructions are this loop's bound.
#define DS_ADMM_CHECK 4

// x, sx, z, y of one contact from its three rows of K and the full right-hand side
// (K and rhs_full are zero beyond the active size, so the product runs over the padded width).
// Only the tangential part of sx = G x + g is formed: the De Saxce term needs nothing else.
// With check, also the primal / dual residual and |z| maxima for the convergence test.
template <int NC3, typename T>
DS_HDI void admm_update(const T (*Kr)[NC3], const T* rhs_full, const T* rhs_own, const T* g, T mu, T rho,
                        T inv_rho, T inv1pmu2, T* x, T* z, T* y, T* sx, T& rp, T& rd, T& zmax, bool check) {
  const T relax = T(1.6);
  T xh[3], w[3], pr[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    T acc = T(0);
#pragma unroll
    for (int c = 0; c < NC3; ++c) acc += Kr[r][c] * rhs_full[c];
    x[r] = acc;
    if (r < 2) sx[r] = rhs_own[r] - rho * acc + g[r];
    xh[r] = relax * x[r] + (T(1) - relax) * z[r];
    w[r] = xh[r] + y[r] * inv_rho;
  }
  proj_cone_fast(w, mu, inv1pmu2, pr);
  if (check) {
    for (int r = 0; r < 3; ++r) {
      rd = nonneg_max(rd, T(fabs(pr[r] - z[r])));
      rp = nonneg_max(rp, T(fabs(x[r] - pr[r])));
      zmax = nonneg_max(zmax, T(fabs(pr[r])));
    }
  }
  for (int r = 0; r < 3; ++r) {
    z[r] = pr[r];
    y[r] += rho * (xh[r] - z[r]);
  }
}

// Largest eigenvalue of a symmetric 3x3 matrix (row-major), from the trigonometric solution of its
// characteristic cubic (O. K. Smith, "Eigenvalues of a symmetric 3x3 matrix", Commun. ACM 4(4),
// 1961): with q = tr/3 and p the scaled deviation, the eigenvalues are q + 2 p cos(phi + 2 pi k/3),
// phi = acos(det((a - q I)/p)/2)/3, and k = 0 gives the largest.
template <typename T>
DS_HDI T sym3_max_eig(const T* a) {
  const T p1 = a[1] * a[1] + a[2] * a[2] + a[5] * a[5];
  const T q = (a[0] + a[4] + a[8]) / T(3);
  const T d0 = a[0] - q, d1 = a[4] - q, d2 = a[8] - q;
  const T p2 = d0 * d0 + d1 * d1 + d2 * d2 + T(2) * p1;
  if (!(p2 > T(0))) return q;
  const T pp = sqrt(p2 / T(6));
  const T ip = T(1) / pp;
  const T b00 = d0 * ip, b11 = d1 * ip, b22 = d2 * ip, b01 = a[1] * ip, b02 = a[2] * ip, b12 = a[5] * ip;
  T r = (b00 * (b11 * b22 - b12 * b12) - b01 * (b01 * b22 - b12 * b02) + b02 * (b01 * b12 - b11 * b02)) / T(2);
  r = fmin(T(1), fmax(T(-1), r));
  return q + T(2) * pp * cos(acos(r) / T(3));
}

// Projected Gauss-Seidel on Eq. 1 (the solver family named beside ADMM in Sec. 2.2): a sweep
// visits the active contacts in order; contact i takes the fixed-point step of Eq. 1 restricted
// to its own block, lambda_i <- Proj_K(lambda_i - (sigma_i + Gamma_i(sigma_i)) / r_i), sigma =
// G lambda + g at the current (partly updated) lambda, r_i = lambda_max(G_ii) (the step that makes
// the local map non-expansive).  Its fixed points are those of Eq. 1 (Moreau).  A sweep counts as
// one iteration; it has converged when it moved lambda by at most te max(1, |lambda|_inf).  z is
// the iterate, as for the ADMM (the Newton stage reads it).
template <int NS, typename T>
struct Pgs {
  static constexpr int NC3 = 3 * NS;
  static constexpr int kCheck = 1;             // the stopping test runs after every sweep
  T z[NC3];
  T ir[NS];

  template <class P>
  DS_HD void adapt(const P&) {}                // no penalty to adapt

  template <class P>
  DS_HD bool setup(const P& p) {
    bool ok = true;
    for (int i = 0; i < p.na; ++i) {
      T blk[9];
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) blk[3 * r + c] = p.Gt[3 * i + r][3 * i + c];
      const T lm = sym3_max_eig(blk);
      ok = ok && lm > T(0);
      ir[i] = lm > T(0) ? T(1) / lm : T(0);
    }
    return ok;
  }

  template <class P>
  DS_HD void reset(const P& p) {
    for (int i = 0; i < NC3; ++i) z[i] = T(0);
  }

  template <class P>
  DS_HD bool iterate(const P& p, T te, bool check) {
    const int m = 3 * p.na;
    T dmax = T(0), lmax = T(1);
    for (int i = 0; i < p.na; ++i) {
      T sg[3];
      for (int k = 0; k < 3; ++k) {
        T t = p.gt[3 * i + k];
        for (int j = 0; j < m; ++j) t += p.Gt[3 * i + k][j] * z[j];
        sg[k] = t;
      }
      const T mu = T(p.mu[i]);
      const T nt = sqrt(sg[0] * sg[0] + sg[1] * sg[1]);
      const T x[3] = {z[3 * i] - sg[0] * ir[i], z[3 * i + 1] - sg[1] * ir[i], z[3 * i + 2] - (sg[2] + mu * nt) * ir[i]};
      T o[3];
      proj_cone(x, mu, o);
      for (int k = 0; k < 3; ++k) {
        dmax = fmax(dmax, fabs(o[k] - z[3 * i + k]));
        z[3 * i + k] = o[k];
        lmax = fmax(lmax, fabs(o[k]));
      }
    }
    return check && dmax <= te * lmax;
  }
};

// Adaptive penalty (options admm_rho_adapt): residual balancing (Boyd et al., Distributed
// optimization and statistical learning via ADMM, 2011, Sec. 3.4.1), with the residuals of this
// iteration's fixed point: primal ||x - z||_inf and dual ||y + sigma + Gamma(sigma)||_inf at
// sigma = sx = G x + g (zero at a solution of Eq. 1, where y = -(sigma + Gamma)).  A primal
// residual ten times the dual one doubles rho, the reverse halves it.  y is the unscaled
// multiplier, so it is kept as it is; the fixed points do not depend on rho.  In FP64 in both
// precisions (the pipeline reads the state from the workspace, the fused path from registers:
// the same values).
template <typename V, typename M>
DS_HDI void admm_residuals(int na, const M* mu, const V* x, const V* z, const V* y, const V* sx, double& rp,
                           double& rd) {
  rp = 0.0;
  rd = 0.0;
  for (int i = 0; i < na; ++i) {
    const double s0 = double(sx[3 * i]), s1 = double(sx[3 * i + 1]), s2 = double(sx[3 * i + 2]);
    const double gam = double(mu[i]) * sqrt(s0 * s0 + s1 * s1);
    rd = fmax(rd, fmax(fabs(double(y[3 * i]) + s0), fmax(fabs(double(y[3 * i + 1]) + s1),
                                                       fabs(double(y[3 * i + 2]) + s2 + gam))));
    for (int r = 0; r < 3; ++r) rp = fmax(rp, fabs(double(x[3 * i + r]) - double(z[3 * i + r])));
  }
}

DS_HDI double rho_balance(double rho, double rp, double rd) {
  if (rp > 10.0 * rd) return 2.0 * rho;
  if (rd > 10.0 * rp) return 0.5 * rho;
  return rho;
}

template <int NS, typename T>
struct Admm {
  static constexpr int NC3 = 3 * NS;
  static constexpr int kCheck = DS_ADMM_CHECK;   // the stopping test runs on every 4th iteration
  T K[NC3][NC3];
  T rho, gs, inv_rho;
  T inv1pmu2[NS];
  int m;
  T x[NC3], z[NC3], y[NC3], sx[NC3];

  template <class P>
  DS_HD bool setup(const P& p) {
    m = 3 * p.na;
    T trace = T(0);
    for (int i = 0; i < m; ++i) trace += p.Gt[i][i];
    rho = T(0.3) * trace / T(m);
    if (!(rho > T(1e-12))) rho = T(1e-12);
    for (int i = 0; i < p.na; ++i) inv1pmu2[i] = T(1) / (T(1) + T(p.mu[i]) * T(p.mu[i]));
    gs = T(1);
    for (int i = 0; i < m; ++i) gs = fmax(gs, fabs(p.gt[i]));
    return factor(p);
  }

  // Adaptive penalty (KArgs.rho_adapt), between rounds: residual balancing of rho
  // (rho_balance) on this iterate, and K formed again when rho changes (kept if that fails).
  template <class P>
  DS_HD void adapt(const P& p) {
    double rp = 0.0, rd = 0.0;
    admm_residuals(p.na, p.mu, x, z, y, sx, rp, rd);
    const double nr = rho_balance(double(rho), rp, rd);
    if (nr == double(rho)) return;
    const T old = rho;
    rho = T(nr);
    if (!factor(p)) { rho = old; factor(p); }
  }

  // K = (G + rho I)^-1 by Cholesky and m solves; 1 / rho.
  template <class P>
  DS_HD bool factor(const P& p) {
    inv_rho = T(1) / rho;
    T Lg[NC3 * (NC3 + 1) / 2];
    for (int i = 0; i < m; ++i)
      for (int j = 0; j <= i; ++j) Lg[tri(i, j)] = p.Gt[i][j] + (i == j ? rho : T(0));
    for (int i = 0; i < NC3; ++i)
      for (int j = 0; j < NC3; ++j) K[i][j] = T(0);
    if (!chol_packed(Lg, m)) return false;
    for (int j = 0; j < m; ++j) {
      T col[NC3];
      for (int i = 0; i < m; ++i) col[i] = T(i == j ? 1 : 0);
      fwd_packed(Lg, col, m);
      bwd_packed(Lg, col, m);
      for (int i = 0; i < m; ++i) K[i][j] = col[i];
    }
    return true;
  }

  template <class P>
  DS_HD void reset(const P& p) {
    for (int i = 0; i < m; ++i) { x[i] = T(0); z[i] = T(0); y[i] = T(0); sx[i] = p.gt[i]; }
  }

  // one iteration; with check, returns true when converged at tolerance te
  template <class P>
  DS_HD bool iterate(const P& p, T te, bool check) {
    T rhs[NC3];
    for (int i = 0; i < NC3; ++i) rhs[i] = T(0);
    for (int i = 0; i < p.na; ++i) admm_rhs(T(p.mu[i]), z + 3 * i, y + 3 * i, p.gt + 3 * i, sx + 3 * i, rho, rhs + 3 * i);
    T rp = T(0), rd = T(0), zmax = T(1);
    for (int i = 0; i < p.na; ++i)
      admm_update<NC3, T>(K + 3 * i, rhs, rhs + 3 * i, p.gt + 3 * i, T(p.mu[i]), rho, inv_rho, inv1pmu2[i],
                          x + 3 * i, z + 3 * i, y + 3 * i, sx + 3 * i, rp, rd, zmax, check);
    rd *= rho;
    return check && rp <= te * zmax && rd <= te * gs;
  }
};

template <typename T>
DS_HDI double stage_eps(const KArgs& a, int stage) {
  const bool dbl = std::is_same<T, double>::value;
  double eps = a.admm_eps;
  for (int k = 0; k < stage; ++k) eps = fmax(eps * (dbl ? 1e-2 : 0.1), dbl ? 1e-13 : 1e-6);
  return eps;
}

template <typename T>
DS_HDI int num_stages() { return std::is_same<T, double>::value ? 4 : 3; }

// End of an ADMM stage: identify the modes from z and run up to 4 active-set rounds of FP64 Newton
// on the mode equations; keeps the best candidate (by FP64 NCP residual).  With `enumerate` (the
// first round of speculative attempts), a failure falls back to the patterns of enum_mode: at most
// DS_ENUM_NEWTON_ITERS Newton steps on each pattern's mode equations from z, in order, until one
// passes.  Returns
// true when the best candidate passes the residual check.
template <class P, typename T>
DS_HD bool newton_stage(P& p, const T* z, double eps, const KArgs& a, double* best, double& best_r,
                        bool enumerate = false) {
  const int m = 3 * p.na;
  double scale = 1.0;
  for (int i = 0; i < m; ++i) scale = fmax(scale, fabs(p.gd[i]));
  const double tol = a.ncp_tol * scale;
  double lz[P::NC3], lp[P::NC3];
  double lscale = 1.0;
  for (int i = 0; i < m; ++i) { lz[i] = double(z[i]); lscale = fmax(lscale, fabs(lz[i])); }
  const double es = fmax(a.eps_sigma, 10.0 * eps), el = fmax(a.eps_lambda, 10.0 * eps);
  const double sat_delta = 10.0 * eps * lscale;
  int mode[P::NC3 / 3];
  classify(p, lz, es, el, mode);
  {
    const double r0 = ncp_residual(p, lz);
    if (r0 < best_r) { best_r = r0; for (int i = 0; i < m; ++i) best[i] = lz[i]; }
  }
  for (int i = 0; i < m; ++i) lp[i] = lz[i];
  for (int round = 0; round < 4 && best_r > tol; ++round) {
    newton_modes(p, lp, mode, a.polish_iters, sat_delta);
    const double rpol = ncp_residual(p, lp);
    if (rpol < best_r) { best_r = rpol; for (int i = 0; i < m; ++i) best[i] = lp[i]; }
    if (best_r <= tol) break;
    // the Newton iterate solves its mode equations exactly: any violation above the acceptance
    // tolerance is real and flips the mode
    if (!reclassify(p, lp, mode, 10.0 * tol, 10.0 * a.ncp_tol * lscale, 10.0 * a.ncp_tol * lscale)) break;
    for (int i = 0; i < p.na; ++i) proj_cone(lp + 3 * i, p.mu[i], lp + 3 * i);
  }
  if (enumerate && best_r > tol) {
    int rank[P::NC3 / 3];
    for (int i = 0; i < p.na; ++i) {
      rank[i] = 0;
      for (int j = 0; j < p.na; ++j)
        rank[i] += (lz[3 * j + 2] > lz[3 * i + 2]) || (lz[3 * j + 2] == lz[3 * i + 2] && j < i);
    }
    const int npat = 2 * p.na * p.na;
    for (int pat = 0; pat < npat && best_r > tol; ++pat) {
      for (int i = 0; i < p.na; ++i) mode[i] = enum_mode(pat, rank[i], p.na);
      for (int i = 0; i < m; ++i) lp[i] = lz[i];
      newton_modes(p, lp, mode, DS_ENUM_NEWTON_ITERS, sat_delta);
      const double rpol = ncp_residual(p, lp);
      if (rpol < best_r) { best_r = rpol; for (int i = 0; i < m; ++i) best[i] = lp[i]; }
    }
  }
  return best_r <= tol;
}

// Solution of the symmetric 3x3 system A x = b by the adjugate (false when A is numerically singular).
DS_HDI bool solve3(const double* A, const double* b, double* x) {
  const double c00 = A[4] * A[8] - A[5] * A[7], c01 = A[5] * A[6] - A[3] * A[8], c02 = A[3] * A[7] - A[4] * A[6];
  const double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
  const double nrm = fabs(A[0]) + fabs(A[4]) + fabs(A[8]);
  if (!(fabs(det) > 1e-14 * nrm * nrm * nrm)) return false;
  const double id = 1.0 / det;
  const double c11 = A[0] * A[8] - A[2] * A[6], c12 = A[1] * A[6] - A[0] * A[7];
  const double c22 = A[0] * A[4] - A[1] * A[3];
  const double c10 = A[2] * A[7] - A[1] * A[8], c20 = A[1] * A[5] - A[2] * A[4], c21 = A[2] * A[3] - A[0] * A[5];
  x[0] = (c00 * b[0] + c10 * b[1] + c20 * b[2]) * id;
  x[1] = (c01 * b[0] + c11 * b[1] + c21 * b[2]) * id;
  x[2] = (c02 * b[0] + c12 * b[1] + c22 * b[2]) * id;
  return true;
}

// ncp_residual of an impulse that is zero except on contact i (components l3): sigma from contact
// i's three columns of G only, and a contact j != i (lambda_j = 0) contributes nothing when its
// sigma_N >= 0 (then sigma_j + Gamma(sigma_j) lies in the dual cone and the complementarity term
// is 0), else the same terms as ncp_residual.  Equal to ncp_residual on such an impulse.
template <class P>
DS_HD double single_residual(const P& p, int i, const double* l3) {
  double r = 0.0;
  const double zero[3] = {0.0, 0.0, 0.0};
  for (int j = 0; j < p.na; ++j) {
    double sg[3];
    for (int k = 0; k < 3; ++k) {
      double t = p.gd[3 * j + k];
      for (int c = 0; c < 3; ++c) t += p.G(3 * j + k, 3 * i + c) * l3[c];
      sg[k] = t;
    }
    if (j != i && sg[2] >= 0.0) continue;
    const double* l = j == i ? l3 : zero;
    double w[3] = {sg[0], sg[1], sg[2] + p.mu[j] * sqrt(sg[0] * sg[0] + sg[1] * sg[1])};
    double q[3];
    proj_cone(l, p.mu[j], q);
    r = fmax(r, sqrt((l[0] - q[0]) * (l[0] - q[0]) + (l[1] - q[1]) * (l[1] - q[1]) + (l[2] - q[2]) * (l[2] - q[2])));
    proj_cone(w, 1.0 / p.mu[j], q);
    r = fmax(r, sqrt((w[0] - q[0]) * (w[0] - q[0]) + (w[1] - q[1]) * (w[1] - q[1]) + (w[2] - q[2]) * (w[2] - q[2])));
    r = fmax(r, fabs(l[0] * w[0] + l[1] * w[1] + l[2] * w[2]));
  }
  return r;
}

// Exact solve of Eq. 1 for an env whose solution has one contact in contact and every other one
// breaking (most arm + cube envs: the cube tips onto one corner): for each active contact, in the
// order of its free normal velocity (most approaching first), the sticking impulse
// lambda_i = -G_ii^-1 g_i, then the sliding solution by Newton on the sliding equations (Sec. 3.2)
// from that impulse's projection onto the cone; the first candidate that passes the FP64 NCP
// residual test (the Newton stage's acceptance) is the solution.  FP64 in both precisions.
// Returns false, lam unspecified, when no single-contact candidate passes; the env then goes
// through the ADMM rounds.
template <class P>
DS_HD bool presolve_single(P& p, const KArgs& a, double* lam) {
  constexpr int NSL = P::NC3 / 3;
  const int m = 3 * p.na;
  double scale = 1.0;
  for (int i = 0; i < m; ++i) scale = fmax(scale, fabs(p.gd[i]));
  const double tol = a.ncp_tol * scale;
  int order[NSL];
  for (int i = 0; i < p.na; ++i) {
    int k = i;
    while (k > 0 && p.gd[3 * order[k - 1] + 2] > p.gd[3 * i + 2]) { order[k] = order[k - 1]; --k; }
    order[k] = i;
  }
  int mode[NSL];
  for (int q = 0; q < p.na; ++q) {
    const int i = order[q];
    double Gb[9], rhs[3], ls[3];
    for (int r = 0; r < 3; ++r) {
      for (int c = 0; c < 3; ++c) Gb[3 * r + c] = p.G(3 * i + r, 3 * i + c);
      rhs[r] = -p.gd[3 * i + r];
    }
    if (!solve3(Gb, rhs, ls)) continue;
    for (int j = 0; j < m; ++j) lam[j] = 0.0;
    for (int r = 0; r < 3; ++r) lam[3 * i + r] = ls[r];
    if (single_residual(p, i, ls) <= tol) return true;
    double pr[3];
    proj_cone(ls, p.mu[i], pr);
    if (!(pr[2] > 0.0) || (pr[0] == ls[0] && pr[1] == ls[1] && pr[2] == ls[2])) continue;
    for (int r = 0; r < 3; ++r) lam[3 * i + r] = pr[r];
    for (int j = 0; j < p.na; ++j) mode[j] = j == i ? DS_MODE_SLIDING : DS_MODE_BREAKING;
    newton_modes(p, lam, mode, a.polish_iters, 0.0);
    if (single_residual(p, i, lam + 3 * i) <= tol) return true;
  }
  return false;
}

// Staged NCP solve in one thread, in the rounds of the pipeline's schedule: each round continues
// the iteration It (ADMM or PGS) for at most the round's cap (the last round: to the iteration
// limit) or until the stage tolerance is met, then runs the Newton / active-set stage on the
// iterate; the first candidate whose FP64 NCP residual passes is accepted.  A stage that ended
// without acceptance moves to the next (tighter) stage; from the schedule's speculative round on,
// an unconverged round's iterate is tried too and the stage is kept.  So the fused kernel reaches
// the same impulse as the pipeline under the same schedule.  When the free motion separates every
// contact, lambda stays 0 (see separating()).
template <class It, class P, typename T>
DS_HD void solve_ncp_with(P& s, const KArgs& a, int& iters, uint32_t& st) {
  const int m = 3 * s.na;
  It ad;
  if (!ad.setup(s)) st |= DS_ENV_NONFINITE;
  ad.reset(s);
  double best[P::NC3], best_r = 1e300;
  bool ok = false;
  const int table = (a.sched.caps >= 0 && a.sched.caps < 3) ? a.sched.caps : 0;
  int stage = 0;
  for (int r = 0; r < DS_ROUNDS; ++r) {
    if (r > 0 && a.rho_adapt) ad.adapt(s);    // as the pipeline does between its rounds
    const bool final_round = r == DS_ROUNDS - 1;
    const int cap = ds_round_cap(table, r);
    const int lim = final_round ? (a.admm_max_iter > cap ? a.admm_max_iter : cap) : cap;
    const double eps = stage_eps<T>(a, stage);
    const T te = T(eps);
    bool conv = false;
    for (int k = 0; k < lim && iters < a.admm_max_iter; ++k) {
      ++iters;
      if (ad.iterate(s, te, iters % It::kCheck == 0)) { conv = true; break; }
    }
    const bool ended = conv || iters >= a.admm_max_iter || final_round;
    const bool late = r >= a.sched.spec_from;
    if (!ended && !late) continue;
    ok = newton_stage(s, ad.z, eps, a, best, best_r, r == a.sched.spec_from);
    if (ok) break;
    if (ended) {
      if (iters >= a.admm_max_iter || stage + 1 >= num_stages<T>() || final_round) break;
      ++stage;
    }
  }
  for (int i = 0; i < m; ++i) s.lam[i] = best[i];
  if (!ok) st |= DS_ENV_NOT_CONVERGED;
}

template <class P, typename T>
DS_HD void solve_ncp(P& s, const KArgs& a, int& iters, uint32_t& st) {
  iters = 0;
  if (s.na == 0 || separating(s)) return;
  if (a.sched.presolve && presolve_single(s, a, s.lam)) return;
  if (a.solver == DS_PGS) solve_ncp_with<Pgs<P::NC3 / 3, T>, P, T>(s, a, iters, st);
  else solve_ncp_with<Admm<P::NC3 / 3, T>, P, T>(s, a, iters, st);
}

}  // namespace ds

namespace ds {

// Directional derivative of the contact-augmented inverse dynamics tau = RNEA(q, v, a*) - J_c^T f
// along one dof: kind 0 = tangent of q (the subtree of the dof's body moves by the rigid twist
// xi = S_d), kind 1 = unit change of the dof's velocity.  Uses the stored pass values V, A, VJ,
// IV, IA, Fc of the a* pass.  Writes dtau[NV].
template <int NB, int NV, int NS, typename T, class E>
DS_HD void rnea_tangent(const DevModel& m, const E& s, int kind, int d, T* dtau) {
  const int j = m.dof_body[DS_IX(d, NV)];
  const int jend = m.sub_end[DS_IX(j, NB)];
  const T* xi = s.S[d];
  T dV[NB][6], dA[NB][6], dF[NB][6];
  for (int k = 0; k < NV; ++k) dtau[k] = T(0);
  for (int i = j; i < jend; ++i) {
    const int par = m.parent[i];
    const bool inside = (i != j);
    T dVJ[6] = {0, 0, 0, 0, 0, 0}, dSa[6] = {0, 0, 0, 0, 0, 0};
    if (kind == 0) {
      for (int dd = m.iv[i]; dd < m.iv[i] + m.nd[i]; ++dd) {
        T dS[6];
        mcross(xi, s.S[DS_IX(dd, NV)], dS);
        for (int k = 0; k < 6; ++k) { dVJ[k] += dS[k] * s.v[DS_IX(dd, NV)]; dSa[k] += dS[k] * s.astar[DS_IX(dd, NV)]; }
      }
    } else if (i == j) {
      for (int k = 0; k < 6; ++k) dVJ[k] = xi[k];
    }
    T t1[6], t2[6];
    for (int k = 0; k < 6; ++k) dV[i][k] = (inside ? dV[DS_IX(par, NB)][k] : T(0)) + dVJ[k];
    mcross(dV[i], s.VJ[i], t1);
    mcross(s.V[i], dVJ, t2);
    for (int k = 0; k < 6; ++k) dA[i][k] = (inside ? dA[DS_IX(par, NB)][k] : T(0)) + dSa[k] + t1[k] + t2[k];
    // dF = I dA + dV x* (I V) + V x* (I dV)  [+ dI A + V x* (dI V) - dFext for q tangents]
    T u[6], w[6];
    iapply(s.I[i], dA[i], u);
    fcross(dV[i], s.IV[i], t1);
    for (int k = 0; k < 6; ++k) u[k] += t1[k];
    iapply(s.I[i], dV[i], w);
    if (kind == 0) {
      // dI X = xi x* (I X) - I (xi x X)
      T xa[6], ixa[6];
      fcross(xi, s.IA[i], t1);
      mcross(xi, s.A[i], xa);
      iapply(s.I[i], xa, ixa);
      for (int k = 0; k < 6; ++k) u[k] += t1[k] - ixa[k];
      fcross(xi, s.IV[i], t1);
      mcross(xi, s.V[i], xa);
      iapply(s.I[i], xa, ixa);
      for (int k = 0; k < 6; ++k) w[k] += t1[k] - ixa[k];
      for (int a = 0; a < s.na; ++a) {
        if (s.body[a] != i) continue;
        T dc[3], t[3];
        cross3(xi + 3, s.x[a], t);
        for (int k = 0; k < 3; ++k) dc[k] = xi[k] + t[k];
        cross3(dc, s.f[a], t);
        for (int k = 0; k < 3; ++k) u[3 + k] -= t[k];
      }
    }
    fcross(s.V[i], w, t1);
    for (int k = 0; k < 6; ++k) dF[i][k] = u[k] + t1[k];
  }
  for (int i = jend - 1; i >= j; --i) {
    for (int dd = m.iv[i]; dd < m.iv[i] + m.nd[i]; ++dd) {
      T r = dot6(s.S[DS_IX(dd, NV)], dF[i]);
      if (kind == 0) {
        T dS[6];
        mcross(xi, s.S[DS_IX(dd, NV)], dS);
        r += dot6(dS, s.Fc[i]);
      }
      dtau[DS_IX(dd, NV)] = r;
    }
    if (i != j) {
      const int par = m.parent[i];
      for (int k = 0; k < 6; ++k) dF[DS_IX(par, NB)][k] += dF[i][k];
    }
  }
  for (int b = m.parent[DS_IX(j, NB)]; b >= 0; b = m.parent[DS_IX(b, NB)])
    for (int dd = m.iv[DS_IX(b, NB)]; dd < m.iv[DS_IX(b, NB)] + m.nd[DS_IX(b, NB)]; ++dd) dtau[DS_IX(dd, NV)] = dot6(s.S[DS_IX(dd, NV)], dF[DS_IX(j, NB)]);
}

// The same directional derivative as rnea_tangent, with the subtree of the dof's body walked
// depth first on an explicit stack: a body's dV, dA and accumulated dF live on the stack only while
// it lies on the path from the dof's body to the body being visited, and a body's dF is final (its
// subtree's included) when it is popped, at which point its dofs' entries are formed and it is
// added into its parent's.  The per-column scratch it touches is the path's depth, not the whole
// tree; the sums over children run in preorder (rnea_tangent sums them in reverse), so the two
// agree to rounding.
template <int NB, int NV, int NS, typename T, class E>
DS_HD void rnea_tangent_stack(const DevModel& m, const E& s, int kind, int d, T* dtau) {
  const int j = m.dof_body[DS_IX(d, NV)];
  const int jend = m.sub_end[DS_IX(j, NB)];
  const T* xi = s.S[d];
  int sb[NB] = {};
  T sV[NB][6], sA[NB][6], sF[NB][6];
  int top = -1;
  for (int k = 0; k < NV; ++k) dtau[k] = T(0);
  // pop the top body: its dofs' entries from its final dF, then dF into its parent's (on the stack)
  auto pop = [&]() {
    const int b = sb[DS_IX(top, NB)];
    for (int dd = m.iv[DS_IX(b, NB)]; dd < m.iv[DS_IX(b, NB)] + m.nd[DS_IX(b, NB)]; ++dd) {
      T r = dot6(s.S[DS_IX(dd, NV)], sF[DS_IX(top, NB)]);
      if (kind == 0) {
        T dS[6];
        mcross(xi, s.S[DS_IX(dd, NV)], dS);
        r += dot6(dS, s.Fc[DS_IX(b, NB)]);
      }
      dtau[DS_IX(dd, NV)] = r;
    }
    if (top > 0)
      for (int k = 0; k < 6; ++k) sF[DS_IX(top - 1, NB)][k] += sF[DS_IX(top, NB)][k];
    --top;
  };
  for (int i = j; i < jend; ++i) {
    const int par = m.parent[i];
    while (top >= 0 && sb[DS_IX(top, NB)] != par) pop();
    const bool inside = top >= 0;
    T dVJ[6] = {0, 0, 0, 0, 0, 0}, dSa[6] = {0, 0, 0, 0, 0, 0};
    if (kind == 0) {
      for (int dd = m.iv[i]; dd < m.iv[i] + m.nd[i]; ++dd) {
        T dS[6];
        mcross(xi, s.S[DS_IX(dd, NV)], dS);
        for (int k = 0; k < 6; ++k) { dVJ[k] += dS[k] * s.v[DS_IX(dd, NV)]; dSa[k] += dS[k] * s.astar[DS_IX(dd, NV)]; }
      }
    } else if (i == j) {
      for (int k = 0; k < 6; ++k) dVJ[k] = xi[k];
    }
    ++top;
    T* dV = sV[DS_IX(top, NB)];
    T* dA = sA[DS_IX(top, NB)];
    sb[DS_IX(top, NB)] = i;
    T t1[6], t2[6];
    for (int k = 0; k < 6; ++k) dV[k] = (inside ? sV[DS_IX(top - 1, NB)][k] : T(0)) + dVJ[k];
    mcross(dV, s.VJ[i], t1);
    mcross(s.V[i], dVJ, t2);
    for (int k = 0; k < 6; ++k) dA[k] = (inside ? sA[DS_IX(top - 1, NB)][k] : T(0)) + dSa[k] + t1[k] + t2[k];
    T u[6], w[6];
    iapply(s.I[i], dA, u);
    fcross(dV, s.IV[i], t1);
    for (int k = 0; k < 6; ++k) u[k] += t1[k];
    iapply(s.I[i], dV, w);
    if (kind == 0) {
      T xa[6], ixa[6];
      fcross(xi, s.IA[i], t1);
      mcross(xi, s.A[i], xa);
      iapply(s.I[i], xa, ixa);
      for (int k = 0; k < 6; ++k) u[k] += t1[k] - ixa[k];
      fcross(xi, s.IV[i], t1);
      mcross(xi, s.V[i], xa);
      iapply(s.I[i], xa, ixa);
      for (int k = 0; k < 6; ++k) w[k] += t1[k] - ixa[k];
      for (int a = 0; a < s.na; ++a) {
        if (s.body[a] != i) continue;
        T dc[3], t[3];
        cross3(xi + 3, s.x[a], t);
        for (int k = 0; k < 3; ++k) dc[k] = xi[k] + t[k];
        cross3(dc, s.f[a], t);
        for (int k = 0; k < 3; ++k) u[3 + k] -= t[k];
      }
    }
    fcross(s.V[i], w, t1);
    for (int k = 0; k < 6; ++k) sF[DS_IX(top, NB)][k] = u[k] + t1[k];
  }
  T Fj[6];
  while (top > 0) pop();
  for (int k = 0; k < 6; ++k) Fj[k] = sF[0][k];     // the dof's body, its whole subtree included
  pop();
  for (int b = m.parent[DS_IX(j, NB)]; b >= 0; b = m.parent[DS_IX(b, NB)])
    for (int dd = m.iv[DS_IX(b, NB)]; dd < m.iv[DS_IX(b, NB)] + m.nd[DS_IX(b, NB)]; ++dd)
      dtau[DS_IX(dd, NV)] = dot6(s.S[DS_IX(dd, NV)], Fj);
}

// d(J_c v+)/dq_d for contact a at fixed v+ (App. D's FKV term, including the motion of the
// contact point with the body): Vp = body velocities under v+.
template <int NB, int NV, int NS, typename T, class E>
DS_HDI void fkv_tangent(const DevModel& m, const E& s, const T (*Vp)[6],
                                            int a, int d, T* out) {
  const int j = m.dof_body[DS_IX(d, NV)];
  const int b = s.body[a];
  out[0] = out[1] = out[2] = T(0);
  if (b < j || b >= m.sub_end[DS_IX(j, NB)]) return;
  const T* xi = s.S[d];
  const int pj = m.parent[DS_IX(j, NB)];
  T rel[6], dVb[6], t[3], dc[3], dp[3];
  for (int k = 0; k < 6; ++k) rel[k] = Vp[DS_IX(b, NB)][k] - (pj >= 0 ? Vp[DS_IX(pj, NB)][k] : T(0));
  mcross(xi, rel, dVb);
  cross3(xi + 3, s.x[a], t);
  for (int k = 0; k < 3; ++k) dc[k] = xi[k] + t[k];
  cross3(dVb + 3, s.c[a], t);
  for (int k = 0; k < 3; ++k) dp[k] = dVb[k] + t[k];
  cross3(Vp[DS_IX(b, NB)] + 3, dc, t);
  for (int k = 0; k < 3; ++k) dp[k] += t[k];
  for (int r = 0; r < 3; ++r) out[r] = dot3(s.fr[r], dp);
}

// Whether g carries the signed-distance term of App. D: gains other than (1, 0), or an activation
// margin (a contact active at phi > 0 then gains phi/dt).
DS_HDI bool gap_term(const KArgs& a) { return !(a.bkp == 1.0 && a.bkd == 0.0 && a.cmargin == 0.0); }

// Baumgarte stabilisation (App. D): each active contact's normal entry of g gains
// phi/dt - kp [phi/dt]_- - kd (J_c v)_N ([x]_- = min(x, 0)), in FP64; with kp = 1, kd = 0 and no
// activation margin (so phi <= 0 on every active contact) the term is identically zero and
// nothing is added.
template <int NB, int NV, int NS, typename T>
DS_HDI void baumgarte_g(const KArgs& a, const int e, const double (*Jd)[NV], Env<NB, NV, NS, T>& s) {
  if (!gap_term(a)) return;
  for (int ac = 0; ac < s.na; ++ac) {
    const int r = 3 * ac + 2;
    const double pr = s.phi[ac] / a.dt;
    double jv = 0.0;
    for (int k = 0; k < NV; ++k) jv += Jd[r][k] * a.v[k * a.B + e];
    const double t = s.gd[r] + (pr - a.bkp * fmin(pr, 0.0) - a.bkd * jv);
    s.gd[r] = t;
    s.gt[r] = T(t);
  }
}

// The Baumgarte term's derivative w.r.t. Jacobian column (blk, d) of contact ac (its normal row):
// d/dq_d: (1 - kp)/dt dphi/dq_d (1/dt where phi >= 0: [x]_- is flat there) - kd d(J_c v)_N/dq_d
// (dphi/dq_d = (J_c)_N,d for a body-fixed contact point; the second term is the FKV derivative at
// v); d/dv_d: -kd (J_c)_N,d; d/dtau: 0.
template <int NB, int NV, int NS, typename T, class E>
DS_HDI T baumgarte_d(const DevModel& m, const KArgs& a, const E& s, int ac, int blk, int d) {
  if (!gap_term(a) || blk == 2) return T(0);
  const T jn = s.Jc[3 * ac + 2][d];
  if (blk == 1) return -T(a.bkd) * jn;
  T r = T((s.phi[ac] < 0.0 ? 1.0 - a.bkp : 1.0) / a.dt) * jn;
  if (a.bkd != 0.0) {
    T fk[3];
    fkv_tangent<NB, NV, NS, T>(m, s, s.V, ac, d, fk);
    r -= T(a.bkd) * fk[2];
  }
  return r;
}

// F1-F6 for env e: kinematics, dynamics, contact detection, J_c, G, g.  Returns status bits.
template <int NB, int NV, int NS, typename T>
DS_HD uint32_t env_forward(const DevModel& m, const KArgs& a, const int e, Env<NB, NV, NS, T>& s) {
  const int B = a.B;
  uint32_t st = 0;
  double* q = s.q;
  for (int i = 0; i < m.nq; ++i) q[i] = a.q[i * B + e];
  bool finite = true;
  for (int i = 0; i < m.nq; ++i) finite &= isfinite(q[i]);
  for (int i = 0; i < NV; ++i) {
    const double vv = a.v[i * B + e], tt = a.tau[i * B + e];
    finite &= isfinite(vv) && isfinite(tt);
    s.v[i] = T(vv);
    s.tau[i] = T(tt);
  }
  if (!finite) st |= DS_ENV_NONFINITE;

  // ---- F1 forward kinematics (FP64) and world spatial quantities
  for (int i = 0; i < NB; ++i) {
    const int par = m.parent[i];
    double R0[9], p0[3];
    if (par < 0) {
      for (int k = 0; k < 9; ++k) R0[k] = m.jrot[i][k];
      for (int k = 0; k < 3; ++k) p0[k] = m.jpos[i][k];
    } else {
      for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c)
          R0[3 * r + c] = s.R[DS_IX(par, NB)][3 * r] * m.jrot[i][c] + s.R[DS_IX(par, NB)][3 * r + 1] * m.jrot[i][3 + c] + s.R[DS_IX(par, NB)][3 * r + 2] * m.jrot[i][6 + c];
        p0[r] = s.P[DS_IX(par, NB)][r] + s.R[DS_IX(par, NB)][3 * r] * m.jpos[i][0] + s.R[DS_IX(par, NB)][3 * r + 1] * m.jpos[i][1] + s.R[DS_IX(par, NB)][3 * r + 2] * m.jpos[i][2];
      }
    }
    double Rj[9];
    double pos[3] = {0, 0, 0};
    if (m.jtype[i] == 0) {
      const double* ax = m.axis[i];
      double sn, cs;
      sincos(q[m.iq[i]], &sn, &cs);
      const double oc = 1.0 - cs;
      Rj[0] = cs + oc * ax[0] * ax[0];        Rj[1] = oc * ax[0] * ax[1] - sn * ax[2]; Rj[2] = oc * ax[0] * ax[2] + sn * ax[1];
      Rj[3] = oc * ax[1] * ax[0] + sn * ax[2]; Rj[4] = cs + oc * ax[1] * ax[1];        Rj[5] = oc * ax[1] * ax[2] - sn * ax[0];
      Rj[6] = oc * ax[2] * ax[0] - sn * ax[1]; Rj[7] = oc * ax[2] * ax[1] + sn * ax[0]; Rj[8] = cs + oc * ax[2] * ax[2];
    } else {
      const int k0 = m.iq[i];
      for (int k = 0; k < 3; ++k) pos[k] = q[k0 + k];
      double w = q[k0 + 3], x = q[k0 + 4], y = q[k0 + 5], z = q[k0 + 6];
      const double inv = 1.0 / sqrt(w * w + x * x + y * y + z * z);
      w *= inv; x *= inv; y *= inv; z *= inv;
      Rj[0] = 1 - 2 * (y * y + z * z); Rj[1] = 2 * (x * y - w * z);     Rj[2] = 2 * (x * z + w * y);
      Rj[3] = 2 * (x * y + w * z);     Rj[4] = 1 - 2 * (x * x + z * z); Rj[5] = 2 * (y * z - w * x);
      Rj[6] = 2 * (x * z - w * y);     Rj[7] = 2 * (y * z + w * x);     Rj[8] = 1 - 2 * (x * x + y * y);
    }
    for (int r = 0; r < 3; ++r) {
      for (int c = 0; c < 3; ++c)
        s.R[i][3 * r + c] = R0[3 * r] * Rj[c] + R0[3 * r + 1] * Rj[3 + c] + R0[3 * r + 2] * Rj[6 + c];
      s.P[i][r] = p0[r] + R0[3 * r] * pos[0] + R0[3 * r + 1] * pos[1] + R0[3 * r + 2] * pos[2];
    }
    // motion subspace (world, at the origin)
    const double* Rw = s.R[i];
    const double* pw = s.P[i];
    if (m.jtype[i] == 0) {
      const double* ax = m.axis[i];
      double aw[3], l[3];
      for (int r = 0; r < 3; ++r) aw[r] = Rw[3 * r] * ax[0] + Rw[3 * r + 1] * ax[1] + Rw[3 * r + 2] * ax[2];
      cross3(pw, aw, l);
      T* S = s.S[m.iv[i]];
      for (int k = 0; k < 3; ++k) { S[k] = T(l[k]); S[3 + k] = T(aw[k]); }
    } else {
      for (int k = 0; k < 3; ++k) {
        const double col[3] = {Rw[k], Rw[3 + k], Rw[6 + k]};
        double l[3];
        cross3(pw, col, l);
        T* St = s.S[m.iv[i] + k];
        T* Sr = s.S[m.iv[i] + 3 + k];
        for (int r = 0; r < 3; ++r) { St[r] = T(col[r]); St[3 + r] = T(0); Sr[r] = T(l[r]); Sr[3 + r] = T(col[r]); }
      }
    }
    // world spatial inertia about the origin
    {
      const double mass = m.mass[i];
      const double* cb = m.com[i];
      double cw[3];
      for (int r = 0; r < 3; ++r) cw[r] = pw[r] + Rw[3 * r] * cb[0] + Rw[3 * r + 1] * cb[1] + Rw[3 * r + 2] * cb[2];
      const double* J = m.inertia[i];
      const double Ib[9] = {J[0], J[3], J[4], J[3], J[1], J[5], J[4], J[5], J[2]};
      double RI[9], Iw[9];
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) RI[3 * r + c] = Rw[3 * r] * Ib[c] + Rw[3 * r + 1] * Ib[3 + c] + Rw[3 * r + 2] * Ib[6 + c];
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) Iw[3 * r + c] = RI[3 * r] * Rw[3 * c] + RI[3 * r + 1] * Rw[3 * c + 1] + RI[3 * r + 2] * Rw[3 * c + 2];
      const double c2 = cw[0] * cw[0] + cw[1] * cw[1] + cw[2] * cw[2];
      T* Ii = s.I[i];
      Ii[0] = T(mass);
      for (int r = 0; r < 3; ++r) Ii[1 + r] = T(mass * cw[r]);
      Ii[4] = T(Iw[0] + mass * (c2 - cw[0] * cw[0]));
      Ii[5] = T(Iw[4] + mass * (c2 - cw[1] * cw[1]));
      Ii[6] = T(Iw[8] + mass * (c2 - cw[2] * cw[2]));
      Ii[7] = T(Iw[1] - mass * cw[0] * cw[1]);
      Ii[8] = T(Iw[2] - mass * cw[0] * cw[2]);
      Ii[9] = T(Iw[5] - mass * cw[1] * cw[2]);
    }
  }

  // ---- F2 bias b(q, v) = RNEA(q, v, 0) with gravity
  const T grav[3] = {T(a.gx), T(a.gy), T(a.gz)};
  T bias[NV];
  {
    for (int i = 0; i < NB; ++i) {
      const int par = m.parent[i];
      T* VJ = s.VJ[i];
      for (int k = 0; k < 6; ++k) VJ[k] = T(0);
      for (int dd = m.iv[i]; dd < m.iv[i] + m.nd[i]; ++dd)
        for (int k = 0; k < 6; ++k) VJ[k] += s.S[DS_IX(dd, NV)][k] * s.v[DS_IX(dd, NV)];
      T t[6];
      for (int k = 0; k < 6; ++k) s.V[i][k] = (par >= 0 ? s.V[DS_IX(par, NB)][k] : T(0)) + VJ[k];
      mcross(s.V[i], VJ, t);
      for (int k = 0; k < 6; ++k)
        s.A[i][k] = (par >= 0 ? s.A[DS_IX(par, NB)][k] : (k < 3 ? -grav[k] : T(0))) + t[k];
      iapply(s.I[i], s.V[i], s.IV[i]);
      iapply(s.I[i], s.A[i], s.IA[i]);
      fcross(s.V[i], s.IV[i], t);
      for (int k = 0; k < 6; ++k) s.Fc[i][k] = s.IA[i][k] + t[k];
    }
    for (int i = NB - 1; i >= 0; --i) {
      for (int dd = m.iv[i]; dd < m.iv[i] + m.nd[i]; ++dd) bias[DS_IX(dd, NV)] = dot6(s.S[DS_IX(dd, NV)], s.Fc[i]);
      const int par = m.parent[i];
      if (par >= 0)
        for (int k = 0; k < 6; ++k) s.Fc[DS_IX(par, NB)][k] += s.Fc[i][k];
    }
  }

  // ---- F3 joint-space inertia by composite inertias (world frame: plain sums), M = L^T L
  {
    T IC[NB][10];
    for (int i = 0; i < NB; ++i)
      for (int k = 0; k < 10; ++k) IC[i][k] = s.I[i][k];
    for (int i = NB - 1; i > 0; --i) {
      const int par = m.parent[i];
      if (par >= 0)
        for (int k = 0; k < 10; ++k) IC[DS_IX(par, NB)][k] += IC[i][k];
    }
    for (int k = 0; k < NV * (NV + 1) / 2; ++k) s.L[k] = T(0);
    for (int i = 0; i < NB; ++i) {
      for (int dd = m.iv[i]; dd < m.iv[i] + m.nd[i]; ++dd) {
        T F[6];
        iapply(IC[i], s.S[DS_IX(dd, NV)], F);
        for (int d2 = m.iv[i]; d2 <= dd; ++d2) s.L[tri(dd, d2)] = dot6(s.S[DS_IX(d2, NV)], F);
        for (int b = m.parent[i]; b >= 0; b = m.parent[DS_IX(b, NB)])
          for (int d2 = m.iv[DS_IX(b, NB)]; d2 < m.iv[DS_IX(b, NB)] + m.nd[DS_IX(b, NB)]; ++d2) s.L[tri(dd, d2)] = dot6(s.S[DS_IX(d2, NV)], F);
      }
    }
    if constexpr (!Env<NB, NV, NS, T>::kDouble) {
      for (int k = 0; k < NV * (NV + 1) / 2; ++k) s.Ld_[k] = double(s.L[k]);
      if (!ltl_factor(s.Ld_, NV, m.dof_parent)) st |= DS_ENV_NONFINITE;
    }
    if (!ltl_factor(s.L, NV, m.dof_parent)) st |= DS_ENV_NONFINITE;
    for (int k = 0; k < NV; ++k) s.vdf[k] = s.tau[k] - bias[k];
    ltl_solve_t(s.L, s.vdf, NV, m.dof_parent);
    ltl_solve(s.L, s.vdf, NV, m.dof_parent);
    for (int k = 0; k < NV; ++k) s.vf[k] = s.v[k] + T(a.dt) * s.vdf[k];
  }

  // ---- F4 contact detection against the plane (FP64 decision)
  const double pn[3] = {a.plane[0 * B + e], a.plane[1 * B + e], a.plane[2 * B + e]};
  const double pd = a.plane[3 * B + e];
  {
    const bool use_y = fabs(pn[0]) > 0.9;
    double t1[3] = {use_y ? 0.0 : 1.0, use_y ? 1.0 : 0.0, 0.0};
    const double dn = t1[0] * pn[0] + t1[1] * pn[1];
    for (int k = 0; k < 3; ++k) t1[k] -= dn * pn[k];
    const double nn = 1.0 / sqrt(t1[0] * t1[0] + t1[1] * t1[1] + t1[2] * t1[2]);
    for (int k = 0; k < 3; ++k) t1[k] *= nn;
    double t2[3];
    cross3(pn, t1, t2);
    for (int k = 0; k < 3; ++k) { s.fr[0][k] = T(t1[k]); s.fr[1][k] = T(t2[k]); s.fr[2][k] = T(pn[k]); }
  }
  s.na = 0;
  for (int k = 0; k < NS; ++k) {
    const int b = a.c_link[k * B + e];
    if (b < 0) continue;
    if (b >= NB) { st |= DS_ENV_NONFINITE; continue; }
    const double pl[3] = {a.c_point[(k * 3 + 0) * B + e], a.c_point[(k * 3 + 1) * B + e], a.c_point[(k * 3 + 2) * B + e]};
    const double r = a.c_radius[k * B + e];
    double xw[3];
    for (int i = 0; i < 3; ++i) xw[i] = s.P[DS_IX(b, NB)][i] + s.R[DS_IX(b, NB)][3 * i] * pl[0] + s.R[DS_IX(b, NB)][3 * i + 1] * pl[1] + s.R[DS_IX(b, NB)][3 * i + 2] * pl[2];
    const double phi = pn[0] * xw[0] + pn[1] * xw[1] + pn[2] * xw[2] - pd - r;
    if (phi <= a.cmargin) {
      const int n = s.na++;
      s.slot[n] = k;
      s.body[n] = b;
      s.mu[n] = a.c_mu[k * B + e];
      s.phi[n] = phi;
      for (int i = 0; i < 3; ++i) {
        s.x[n][i] = T(xw[i]);
        s.c[n][i] = T(xw[i] - r * pn[i]);
        s.cx_d[n][i] = xw[i] - r * pn[i];
      }
    }
  }
  for (int k = NS; k < a.ncmax; ++k)            // slots beyond this kernel's: must be unused
    if (a.c_link[k * B + e] >= 0) st |= DS_ENV_BAD_SLOT;
  const int mdim = 3 * s.na;

  // ---- F5 contact Jacobian rows (t1, t2, n) . velocity of the body point at c, in FP64 from the
  // FP64 placements: the rows of corners of one rigid body stay exactly dependent.
  constexpr bool kD = Env<NB, NV, NS, T>::kDouble;
  double (*Jd)[NV];
  double (*Yd)[NV];
  const double* Ld;
  if constexpr (kD) { Jd = s.Jc; Yd = s.Y; Ld = s.L; } else { Jd = s.Jd_; Yd = s.Yd_; Ld = s.Ld_; }
  {
    double frd[3][3];
    {
      const bool use_y = fabs(pn[0]) > 0.9;
      double t1[3] = {use_y ? 0.0 : 1.0, use_y ? 1.0 : 0.0, 0.0};
      const double dn = t1[0] * pn[0] + t1[1] * pn[1];
      for (int k = 0; k < 3; ++k) t1[k] -= dn * pn[k];
      const double nn = 1.0 / sqrt(t1[0] * t1[0] + t1[1] * t1[1] + t1[2] * t1[2]);
      for (int k = 0; k < 3; ++k) t1[k] *= nn;
      double t2[3];
      cross3(pn, t1, t2);
      for (int k = 0; k < 3; ++k) { frd[0][k] = t1[k]; frd[1][k] = t2[k]; frd[2][k] = pn[k]; }
    }
    for (int r = 0; r < mdim; ++r)
      for (int k = 0; k < NV; ++k) Jd[r][k] = 0.0;
    for (int ac = 0; ac < s.na; ++ac) {
      const double cd[3] = {double(s.cx_d[ac][0]), double(s.cx_d[ac][1]), double(s.cx_d[ac][2])};
      for (int b = s.body[ac]; b >= 0; b = m.parent[DS_IX(b, NB)]) {
        const double* Rb = s.R[DS_IX(b, NB)];
        const double* pb = s.P[DS_IX(b, NB)];
        const double rel[3] = {cd[0] - pb[0], cd[1] - pb[1], cd[2] - pb[2]};
        for (int dd = m.iv[DS_IX(b, NB)]; dd < m.iv[DS_IX(b, NB)] + m.nd[DS_IX(b, NB)]; ++dd) {
          double pv[3];
          const int k = dd - m.iv[DS_IX(b, NB)];
          if (m.jtype[DS_IX(b, NB)] == 0) {
            const double* ax = m.axis[DS_IX(b, NB)];
            double aw[3];
            for (int r = 0; r < 3; ++r) aw[r] = Rb[3 * r] * ax[0] + Rb[3 * r + 1] * ax[1] + Rb[3 * r + 2] * ax[2];
            cross3(aw, rel, pv);
          } else if (k < 3) {
            for (int r = 0; r < 3; ++r) pv[r] = Rb[3 * r + k];
          } else {
            const double col[3] = {Rb[k - 3], Rb[3 + k - 3], Rb[6 + k - 3]};
            cross3(col, rel, pv);
          }
          for (int r = 0; r < 3; ++r) Jd[3 * ac + r][DS_IX(dd, NV)] = dot3(frd[r], pv);
        }
      }
    }
  }

  // ---- F6 Delassus matrix G = (L^-T J^T)^T (L^-T J^T), Y = M^-1 J^T, g = J v_f (FP64 in both forms).
  for (int r = 0; r < mdim; ++r) {
    for (int k = 0; k < NV; ++k) Yd[r][k] = Jd[r][k];
    ltl_solve_t(Ld, Yd[r], NV, m.dof_parent);
  }
  for (int r = 0; r < mdim; ++r)
    for (int c = 0; c <= r; ++c) {
      double t = 0.0;
      for (int k = 0; k < NV; ++k) t += Yd[r][k] * Yd[c][k];
      s.Gt[r][c] = T(t);
      s.Gt[c][r] = T(t);
      if constexpr (!kD) { s.Gd_[r][c] = t; s.Gd_[c][r] = t; }
    }
  for (int r = 0; r < mdim; ++r) {
    ltl_solve(Ld, Yd[r], NV, m.dof_parent);
    double t = 0.0;
    for (int k = 0; k < NV; ++k) t += Jd[r][k] * double(s.vf[k]);
    s.gt[r] = T(t);
    s.gd[r] = t;
  }
  baumgarte_g(a, e, Jd, s);
  if constexpr (!kD)
    for (int r = 0; r < mdim; ++r)
      for (int k = 0; k < NV; ++k) { s.Jc[r][k] = T(Jd[r][k]); s.Y[r][k] = T(Yd[r][k]); }
  return st;
}

// The forward state a pipeline step keeps per env from its setup for its finish, as rows of the
// workspace's fw array (row r of env e at fw[r * B + e]), in this order: vdf, v_f (NV each), the
// world motion subspaces S (6 NV), the world spatial inertias I (10 NB), the bias pass's body
// velocities V, joint velocities VJ and momenta I V (6 NB each), M's packed factor L, the rows of
// J_c and of M^-1 J_c^T (NC3 x NV each, active contacts first), and per contact slot of the
// active list its body point x (3), contact point c (3), signed distance, slot and body.  Stored
// in FP64 whatever the bulk type (exact for FP32 values).  ds_forward_rows counts the same rows.
template <int NB, int NV, int NS>
struct FwLayout {
  static constexpr int NC3 = 3 * NS, NL = NV * (NV + 1) / 2;
  static constexpr int vdf = 0, vf = NV, S = 2 * NV, I = 8 * NV, V = I + 10 * NB, VJ = V + 6 * NB, IV = VJ + 6 * NB;
  static constexpr int L = IV + 6 * NB, Jc = L + NL, Y = Jc + NC3 * NV, C = Y + NC3 * NV;
  static constexpr int rows = C + 9 * NS;
};

template <int NB, int NV, int NS, typename T>
DS_HD void store_forward(const KArgs& a, const int e, const Env<NB, NV, NS, T>& s) {
  using F = FwLayout<NB, NV, NS>;
  static_assert(F::rows == 8 * NV + 28 * NB + NV * (NV + 1) / 2 + 6 * NS * NV + 9 * NS, "forward rows");
  const int B = a.B;
  double* fw = a.ws.fw;
  auto put = [&](int r, double x) { fw[size_t(r) * B + e] = x; };
  for (int k = 0; k < NV; ++k) { put(F::vdf + k, double(s.vdf[k])); put(F::vf + k, double(s.vf[k])); }
  for (int d = 0; d < NV; ++d)
    for (int k = 0; k < 6; ++k) put(F::S + 6 * d + k, double(s.S[d][k]));
  for (int i = 0; i < NB; ++i) {
    for (int k = 0; k < 10; ++k) put(F::I + 10 * i + k, double(s.I[i][k]));
    for (int k = 0; k < 6; ++k) {
      put(F::V + 6 * i + k, double(s.V[i][k]));
      put(F::VJ + 6 * i + k, double(s.VJ[i][k]));
      put(F::IV + 6 * i + k, double(s.IV[i][k]));
    }
  }
  for (int k = 0; k < F::NL; ++k) put(F::L + k, double(s.L[k]));
  const int mdim = 3 * s.na;
  for (int r = 0; r < mdim; ++r)
    for (int k = 0; k < NV; ++k) { put(F::Jc + r * NV + k, double(s.Jc[r][k])); put(F::Y + r * NV + k, double(s.Y[r][k])); }
  for (int ac = 0; ac < s.na; ++ac) {
    const int r0 = F::C + 9 * ac;
    for (int k = 0; k < 3; ++k) { put(r0 + k, double(s.x[ac][k])); put(r0 + 3 + k, double(s.c[ac][k])); }
    put(r0 + 6, s.phi[ac]);
    put(r0 + 7, double(s.slot[ac]));
    put(r0 + 8, double(s.body[ac]));
  }
}

// The finish's Env from the inputs, the contact problem in the workspace and the forward state the
// setup stored (instead of recomputing F1-F6): q, v, tau, the active contacts, mu, G, g, the
// contact frame and the fields store_forward wrote.
template <int NB, int NV, int NS, typename T>
DS_HD void load_forward(const DevModel& m, const KArgs& a, const int e, Env<NB, NV, NS, T>& s) {
  using F = FwLayout<NB, NV, NS>;
  const int B = a.B;
  const WsView& w = a.ws;
  const double* fw = w.fw;
  auto get = [&](int r) { return fw[size_t(r) * B + e]; };
  for (int i = 0; i < m.nq; ++i) s.q[i] = a.q[i * B + e];
  for (int k = 0; k < NV; ++k) {
    s.v[k] = T(a.v[k * B + e]);
    s.tau[k] = T(a.tau[k * B + e]);
    s.vdf[k] = T(get(F::vdf + k));
    s.vf[k] = T(get(F::vf + k));
  }
  for (int d = 0; d < NV; ++d)
    for (int k = 0; k < 6; ++k) s.S[d][k] = T(get(F::S + 6 * d + k));
  for (int i = 0; i < NB; ++i) {
    for (int k = 0; k < 10; ++k) s.I[i][k] = T(get(F::I + 10 * i + k));
    for (int k = 0; k < 6; ++k) {
      s.V[i][k] = T(get(F::V + 6 * i + k));
      s.VJ[i][k] = T(get(F::VJ + 6 * i + k));
      s.IV[i][k] = T(get(F::IV + 6 * i + k));
    }
  }
  for (int k = 0; k < F::NL; ++k) s.L[k] = T(get(F::L + k));
  s.na = w.na[e];
  const int mdim = 3 * s.na;
  for (int r = 0; r < mdim; ++r)
    for (int k = 0; k < NV; ++k) { s.Jc[r][k] = T(get(F::Jc + r * NV + k)); s.Y[r][k] = T(get(F::Y + r * NV + k)); }
  for (int ac = 0; ac < s.na; ++ac) {
    const int r0 = F::C + 9 * ac;
    for (int k = 0; k < 3; ++k) {
      s.x[ac][k] = T(get(r0 + k));
      s.c[ac][k] = T(get(r0 + 3 + k));
      s.cx_d[ac][k] = get(r0 + 3 + k);
    }
    s.phi[ac] = get(r0 + 6);
    s.slot[ac] = int(get(r0 + 7));
    s.body[ac] = int(get(r0 + 8));
    s.mu[ac] = w.mu[ac * B + e];
  }
  // contact frame rows t1, t2, n from the plane normal (as in the forward pass)
  const double pn[3] = {a.plane[0 * B + e], a.plane[1 * B + e], a.plane[2 * B + e]};
  const bool use_y = fabs(pn[0]) > 0.9;
  double t1[3] = {use_y ? 0.0 : 1.0, use_y ? 1.0 : 0.0, 0.0};
  const double dn = t1[0] * pn[0] + t1[1] * pn[1];
  for (int k = 0; k < 3; ++k) t1[k] -= dn * pn[k];
  const double nn = 1.0 / sqrt(t1[0] * t1[0] + t1[1] * t1[1] + t1[2] * t1[2]);
  for (int k = 0; k < 3; ++k) t1[k] *= nn;
  double t2[3];
  cross3(pn, t1, t2);
  for (int k = 0; k < 3; ++k) { s.fr[0][k] = T(t1[k]); s.fr[1][k] = T(t2[k]); s.fr[2][k] = T(pn[k]); }
  for (int i = 0; i < mdim; ++i) {
    for (int j = 0; j <= i; ++j) {
      const double gij = w.G[tri(i, j) * B + e];
      s.Gt[i][j] = T(gij);
      s.Gt[j][i] = T(gij);
      if constexpr (!Env<NB, NV, NS, T>::kDouble) { s.Gd_[i][j] = gij; s.Gd_[j][i] = gij; }
    }
    s.gd[i] = w.g[i * B + e];
    s.gt[i] = T(s.gd[i]);
  }
}

// F9 and, on request, B1-B7 for env e, given lambda and the modes of its active contacts.
// Adjoint of the position update q+ = q (+) dt v+ for the cotangent qn of q+ (in the tangent
// coordinates at q+): vadd = dt (dq+/d delta)^T qn and qa = (dq+/dq)^T qn.  Revolute dofs: both
// Jacobians are the identity.  Free-flyer (p+ = p + R delta_lin, R+ = R Exp(delta_ang)): with
// E = Exp(delta_ang), dq+/dq = [[E^T, -E^T [delta_lin]x], [0, E^T]] and dq+/d delta =
// [[E^T, 0], [0, Jr(delta_ang)]] (Jr: right Jacobian of SO(3)); E and Jr^T are applied as
// x + c1 phi x x + c2 phi x (phi x x) with their series near phi = 0.
DS_HDI void so3_apply(const double* phi, const double* x, double c1, double c2, double* o) {
  double t1[3], t2[3];
  cross3(phi, x, t1);
  cross3(phi, t1, t2);
  for (int k = 0; k < 3; ++k) o[k] = x[k] + c1 * t1[k] + c2 * t2[k];
}

DS_HDI void integrate_adjoint(const DevModel& m, const double* vn, double dt, const double* qn, double* vadd,
                             double* qa) {
  for (int i = 0; i < m.nb; ++i) {
    const int d0 = m.iv[i];
    if (m.jtype[i] == 0) {
      vadd[d0] = dt * qn[d0];
      qa[d0] = qn[d0];
      continue;
    }
    const double dl[3] = {dt * vn[d0], dt * vn[d0 + 1], dt * vn[d0 + 2]};
    const double ph[3] = {dt * vn[d0 + 3], dt * vn[d0 + 4], dt * vn[d0 + 5]};
    const double t2 = ph[0] * ph[0] + ph[1] * ph[1] + ph[2] * ph[2];
    double sa, ca, cb;                // sin t / t, (1 - cos t) / t^2, (t - sin t) / t^3
    if (t2 < 1e-8) {
      sa = 1.0 - t2 / 6.0 + t2 * t2 / 120.0;
      ca = 0.5 - t2 / 24.0 + t2 * t2 / 720.0;
      cb = 1.0 / 6.0 - t2 / 120.0 + t2 * t2 / 5040.0;
    } else {
      const double t = sqrt(t2);
      sa = sin(t) / t;
      ca = (1.0 - cos(t)) / t2;
      cb = (t - sin(t)) / (t2 * t);
    }
    double el[3], ea[3], jr[3], cr[3];
    so3_apply(ph, qn + d0, sa, ca, el);          // E qn_lin
    so3_apply(ph, qn + d0 + 3, sa, ca, ea);      // E qn_ang
    so3_apply(ph, qn + d0 + 3, ca, cb, jr);      // Jr^T qn_ang
    cross3(dl, el, cr);                          // [delta_lin]x E qn_lin
    for (int k = 0; k < 3; ++k) {
      qa[d0 + k] = el[k];
      qa[d0 + 3 + k] = cr[k] + ea[k];
      vadd[d0 + k] = dt * el[k];
      vadd[d0 + 3 + k] = dt * jr[k];
    }
  }
}

// Reduced implicit system of an env (App. B): offset and size of each contact's block (3 rows
// sticking, 2 sliding, 0 breaking), the sliding contacts' R and R^T P, and its dimension md.
template <int NS>
struct Reduced {
  int off[NS], sz[NS];
  double Rm[NS][3][2], RP[NS][2][3];
  int md;
};

// The part of the finish before the derivative columns: the B1 pass of
// tau = RNEA(q, v, a*) - J_c^T f at a* = (v+ - v)/dt with the contact forces (s.astar, s.f, s.A,
// s.IA, s.Fc), the body velocities under v+ (Vp), and the reduced system A = B G C + blkdiag(0, Q)
// (App. B) built and factored in s.lu (DS_ENV_SINGULAR when rank deficient).
template <int NB, int NV, int NS, typename T>
DS_HD void finish_reduced(const DevModel& m, const KArgs& a, Env<NB, NV, NS, T>& s, T (*Vp)[6], Reduced<NS>& rd,
                          uint32_t& st) {
  const int mdim = 3 * s.na;
  const T grav[3] = {T(a.gx), T(a.gy), T(a.gz)};
  int(&off)[NS] = rd.off;
  int(&sz)[NS] = rd.sz;
  double(&Rm)[NS][3][2] = rd.Rm;
  double(&RP)[NS][2][3] = rd.RP;
  int& md = rd.md;
  // ---- B1 pass of tau = RNEA(q, v, a*) - J_c^T f at a* = (v+ - v)/dt with the contact forces
  for (int k = 0; k < NV; ++k) {
    T t = s.vdf[k];
    for (int r = 0; r < mdim; ++r) t += s.Y[r][k] * T(s.lam[r] / a.dt);
    s.astar[k] = t;
  }
  for (int ac = 0; ac < s.na; ++ac)
    for (int k = 0; k < 3; ++k)
      s.f[ac][k] = T((double(s.fr[0][k]) * s.lam[3 * ac] + double(s.fr[1][k]) * s.lam[3 * ac + 1] +
                      double(s.fr[2][k]) * s.lam[3 * ac + 2]) / a.dt);
  for (int i = 0; i < NB; ++i) {
    const int par = m.parent[i];
    T t[6];
    mcross(s.V[i], s.VJ[i], t);
    for (int k = 0; k < 6; ++k) s.A[i][k] = (par >= 0 ? s.A[DS_IX(par, NB)][k] : (k < 3 ? -grav[k] : T(0))) + t[k];
    for (int dd = m.iv[i]; dd < m.iv[i] + m.nd[i]; ++dd)
      for (int k = 0; k < 6; ++k) s.A[i][k] += s.S[DS_IX(dd, NV)][k] * s.astar[DS_IX(dd, NV)];
    iapply(s.I[i], s.A[i], s.IA[i]);
    fcross(s.V[i], s.IV[i], t);
    for (int k = 0; k < 6; ++k) s.Fc[i][k] = s.IA[i][k] + t[k];
    for (int ac = 0; ac < s.na; ++ac) {
      if (s.body[ac] != i) continue;
      T cf[3];
      cross3(s.c[ac], s.f[ac], cf);
      for (int k = 0; k < 3; ++k) { s.Fc[i][k] -= s.f[ac][k]; s.Fc[i][3 + k] -= cf[k]; }
    }
  }
  for (int i = NB - 1; i > 0; --i) {
    const int par = m.parent[i];
    if (par >= 0)
      for (int k = 0; k < 6; ++k) s.Fc[DS_IX(par, NB)][k] += s.Fc[i][k];
  }
  // body velocities under v+ (for the FKV term)
  for (int i = 0; i < NB; ++i) {
    const int par = m.parent[i];
    for (int k = 0; k < 6; ++k) Vp[i][k] = (par >= 0 ? Vp[DS_IX(par, NB)][k] : T(0));
    for (int dd = m.iv[i]; dd < m.iv[i] + m.nd[i]; ++dd)
      for (int k = 0; k < 6; ++k) Vp[i][k] += s.S[DS_IX(dd, NV)][k] * s.vn[DS_IX(dd, NV)];
  }

  // ---- B3/B4 reduced implicit system A = B G C + blkdiag(0, Q) (App. B), FP64
  md = 0;
  for (int pass = 0; pass < 2; ++pass)
    for (int ac = 0; ac < s.na; ++ac) {
      const int want = pass == 0 ? DS_MODE_STICKING : DS_MODE_SLIDING;
      if (s.mode[ac] != want) continue;
      off[ac] = md;
      sz[ac] = pass == 0 ? 3 : 2;
      md += sz[ac];
    }
  for (int ac = 0; ac < s.na; ++ac) {
    if (s.mode[ac] == DS_MODE_BREAKING) { sz[ac] = 0; off[ac] = 0; }
    if (s.mode[ac] != DS_MODE_SLIDING) continue;
    double sg[3];
    for (int k = 0; k < 3; ++k) {
      double t = s.gd[3 * ac + k];
      for (int j = 0; j < mdim; ++j) t += s.G(3 * ac + k, j) * s.lam[j];
      sg[k] = t;
    }
    const double* l = s.lam + 3 * ac;
    const double ns = sqrt(sg[0] * sg[0] + sg[1] * sg[1]);
    const double u[2] = {sg[0] / ns, sg[1] / ns};
    const double nl = sqrt(l[0] * l[0] + l[1] * l[1] + l[2] * l[2]);
    const double r1[3] = {l[0] / nl, l[1] / nl, l[2] / nl};
    const double r2[3] = {-u[1], u[0], 0.0};
    const double ia = s.mu[ac] * l[2] / ns;   // 1/alpha
    for (int k = 0; k < 3; ++k) { Rm[ac][k][0] = r1[k]; Rm[ac][k][1] = r2[k]; }
    // R^T P with P = diag(H/alpha, 1), H = I - u u^T
    const double H[2][2] = {{1 - u[0] * u[0], -u[0] * u[1]}, {-u[1] * u[0], 1 - u[1] * u[1]}};
    const double* rr[2] = {r1, r2};
    for (int c = 0; c < 2; ++c) {
      RP[ac][c][0] = ia * (rr[c][0] * H[0][0] + rr[c][1] * H[1][0]);
      RP[ac][c][1] = ia * (rr[c][0] * H[0][1] + rr[c][1] * H[1][1]);
      RP[ac][c][2] = rr[c][2];
    }
  }
  s.lu.r = md;
  s.lu.c = md;
  for (int ra = 0; ra < s.na; ++ra) {
    if (sz[ra] == 0) continue;
    for (int cb = 0; cb < s.na; ++cb) {
      if (sz[cb] == 0) continue;
      double Gb[3][3];
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) Gb[r][c] = s.G(3 * ra + r, 3 * cb + c);
      double LG[3][3];   // left (I or R^T P) times G block
      for (int r = 0; r < sz[ra]; ++r)
        for (int c = 0; c < 3; ++c)
          LG[r][c] = sz[ra] == 3 ? Gb[r][c] : RP[ra][r][0] * Gb[0][c] + RP[ra][r][1] * Gb[1][c] + RP[ra][r][2] * Gb[2][c];
      for (int r = 0; r < sz[ra]; ++r)
        for (int c = 0; c < sz[cb]; ++c) {
          double t = sz[cb] == 3 ? LG[r][c] : LG[r][0] * Rm[cb][0][c] + LG[r][1] * Rm[cb][1][c] + LG[r][2] * Rm[cb][2][c];
          if (ra == cb && sz[ra] == 2 && r == 1 && c == 1) t += 1.0;   // Q = diag(0, 1)
          s.lu.a[off[ra] + r][off[cb] + c] = t;
        }
    }
  }
  if (md > 0) {
    s.lu.factor(1e-12);
    s.lu.nullspace();
    if (s.lu.rank < md) st |= DS_ENV_SINGULAR;
  }
}

// Rows of the implicit part of the Jacobian: P_k = B^T (A^-)^T C^T Y^T e_k for the output rows
// k = k0, k0 + kstep, ... (one transposed minimum-norm solve each), so that column c of
// Y C A^- B (J_c D + F) is sum_j P[k][j] (J_c D + F)_j.  Rows of breaking contacts are 0.
template <int NB, int NV, int NS, typename T>
DS_HD void finish_rows(Env<NB, NV, NS, T>& s, const Reduced<NS>& rd, double (*P)[3 * NS], int k0 = 0, int kstep = 1) {
  const int(&off)[NS] = rd.off;
  const int(&sz)[NS] = rd.sz;
  const double(&Rm)[NS][3][2] = rd.Rm;
  const double(&RP)[NS][2][3] = rd.RP;
  for (int k = k0; k < NV; k += kstep) {
    double u[3 * NS], z[3 * NS];
    for (int ac = 0; ac < s.na; ++ac) {
      if (sz[ac] == 0) continue;
      if (sz[ac] == 3) {
        for (int r = 0; r < 3; ++r) u[off[ac] + r] = double(s.Y[3 * ac + r][k]);
      } else {
        for (int c = 0; c < 2; ++c)
          u[off[ac] + c] = Rm[ac][0][c] * double(s.Y[3 * ac][k]) + Rm[ac][1][c] * double(s.Y[3 * ac + 1][k]) +
                           Rm[ac][2][c] * double(s.Y[3 * ac + 2][k]);
      }
    }
    s.lu.solve_t_mn(u, z);
    for (int ac = 0; ac < s.na; ++ac) {
      for (int r = 0; r < 3; ++r) {
        double p = 0.0;
        if (sz[ac] == 3) p = z[off[ac] + r];
        else if (sz[ac] == 2) p = RP[ac][0][r] * z[off[ac]] + RP[ac][1][r] * z[off[ac] + 1];
        P[k][3 * ac + r] = p;
      }
    }
  }
}

// The VJP's adjoint vectors (B7, B8): with v_bar (and the position update's adjoint chained in
// when there is a cotangent of q+: qadd), z = A^-T C^T Y^T v_bar, zeta = B^T z,
// ub = v_bar - J_c^T zeta and w2 = M^-1 ub.
template <int NB, int NV, int NS, typename T>
DS_HD void finish_vjp_head(const DevModel& m, const KArgs& a, const int e, Env<NB, NV, NS, T>& s,
                           const Reduced<NS>& rd, T* ub, T* w2, double* zeta, double* qadd) {
  const int B = a.B;
  const int mdim = 3 * s.na;
  const int(&off)[NS] = rd.off;
  const int(&sz)[NS] = rd.sz;
  const double(&Rm)[NS][3][2] = rd.Rm;
  const double(&RP)[NS][2][3] = rd.RP;
  const int md = rd.md;
  T vb[NV];
  double qn[NV], vadd[NV];
  if (a.qnbar) {
    double vnd[NV];
    for (int k = 0; k < NV; ++k) { qn[k] = a.qnbar[k * B + e]; vnd[k] = double(s.vn[k]); }
    integrate_adjoint(m, vnd, a.dt, qn, vadd, qadd);
  }
  for (int k = 0; k < NV; ++k) {
    vb[k] = T(a.qnbar ? a.vbar[k * B + e] + vadd[k] : a.vbar[k * B + e]);
    ub[k] = vb[k];
  }
  for (int r = 0; r < mdim; ++r) zeta[r] = 0.0;
  if (md > 0) {
    double wv[3 * NS], z[3 * NS];
    for (int ac = 0; ac < s.na; ++ac) {
      if (sz[ac] == 0) continue;
      double y3[3];
      for (int r = 0; r < 3; ++r) {
        T t = T(0);
        for (int k = 0; k < NV; ++k) t += s.Y[3 * ac + r][k] * vb[k];
        y3[r] = double(t);
      }
      if (sz[ac] == 3) { for (int r = 0; r < 3; ++r) wv[off[ac] + r] = y3[r]; }
      else { for (int c = 0; c < 2; ++c) wv[off[ac] + c] = Rm[ac][0][c] * y3[0] + Rm[ac][1][c] * y3[1] + Rm[ac][2][c] * y3[2]; }
    }
    s.lu.solve_t_mn(wv, z);
    for (int ac = 0; ac < s.na; ++ac) {
      if (sz[ac] == 0) continue;
      if (sz[ac] == 3) { for (int r = 0; r < 3; ++r) zeta[3 * ac + r] = z[off[ac] + r]; }
      else { for (int r = 0; r < 3; ++r) zeta[3 * ac + r] = RP[ac][0][r] * z[off[ac]] + RP[ac][1][r] * z[off[ac] + 1]; }
    }
    for (int r = 0; r < mdim; ++r) {
      const T zr = T(zeta[r]);
      const int b = s.body[r / 3];
      for (int k = m.iv[DS_IX(b, NB)] + m.nd[DS_IX(b, NB)] - 1; k >= 0; k = m.dof_parent[DS_IX(k, NV)])
        ub[k] -= s.Jc[r][k] * zr;
    }
  }
  for (int k = 0; k < NV; ++k) w2[k] = ub[k];
  ltl_solve_t(s.L, w2, NV, m.dof_parent);
  ltl_solve(s.L, w2, NV, m.dof_parent);
}

template <int NB, int NV, int NS, typename T>
DS_HD void env_finish(const DevModel& m, const KArgs& a, const int e, Env<NB, NV, NS, T>& s, uint32_t st, int iters,
                      int chunk = 0, int nchunk = 1) {
  // With nchunk > 1 the Jacobian columns (or the VJP's dof passes) are split over nchunk threads of
  // the same env; chunk 0 also writes the step's outputs.
  const bool lead = chunk == 0;
  const int B = a.B;
  const int mdim = 3 * s.na;
  const double* q = s.q;
  const T grav[3] = {T(a.gx), T(a.gy), T(a.gz)};
  for (int k = 0; k < NV; ++k) {
    T t = s.vf[k];
    for (int r = 0; r < mdim; ++r) t += s.Y[r][k] * T(s.lam[r]);
    s.vn[k] = t;
  }
  for (int k = 0; k < NV; ++k) {
    const double vv = double(s.vn[k]);
    if (!isfinite(vv)) st |= DS_ENV_NONFINITE;
    if (lead) a.v_next[k * B + e] = vv;
  }
  if (a.q_next && lead) {
    for (int i = 0; i < NB; ++i) {
      const int k0 = m.iq[i], d0 = m.iv[i];
      if (m.jtype[i] == 0) {
        a.q_next[k0 * B + e] = q[k0] + a.dt * double(s.vn[d0]);
      } else {
        double w = q[k0 + 3], x = q[k0 + 4], y = q[k0 + 5], z = q[k0 + 6];
        const double inv = 1.0 / sqrt(w * w + x * x + y * y + z * z);
        w *= inv; x *= inv; y *= inv; z *= inv;
        const double Rq[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                              2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                              2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)};
        const double dl[3] = {a.dt * double(s.vn[d0]), a.dt * double(s.vn[d0 + 1]), a.dt * double(s.vn[d0 + 2])};
        for (int r = 0; r < 3; ++r)
          a.q_next[(k0 + r) * B + e] = q[k0 + r] + Rq[3 * r] * dl[0] + Rq[3 * r + 1] * dl[1] + Rq[3 * r + 2] * dl[2];
        const double wv[3] = {a.dt * double(s.vn[d0 + 3]), a.dt * double(s.vn[d0 + 4]), a.dt * double(s.vn[d0 + 5])};
        const double th2 = wv[0] * wv[0] + wv[1] * wv[1] + wv[2] * wv[2];
        double ce, se;
        if (th2 < 1e-10) { ce = 1 - th2 / 8 + th2 * th2 / 384; se = 0.5 - th2 / 48 + th2 * th2 / 3840; }
        else { const double th = sqrt(th2); ce = cos(0.5 * th); se = sin(0.5 * th) / th; }
        const double ew = ce, ex = se * wv[0], ey = se * wv[1], ez = se * wv[2];
        double nw = w * ew - x * ex - y * ey - z * ez;
        double nx = w * ex + x * ew + y * ez - z * ey;
        double ny = w * ey - x * ez + y * ew + z * ex;
        double nz = w * ez + x * ey - y * ex + z * ew;
        const double ni = 1.0 / sqrt(nw * nw + nx * nx + ny * ny + nz * nz);
        a.q_next[(k0 + 3) * B + e] = nw * ni;
        a.q_next[(k0 + 4) * B + e] = nx * ni;
        a.q_next[(k0 + 5) * B + e] = ny * ni;
        a.q_next[(k0 + 6) * B + e] = nz * ni;
      }
    }
  }
  if (lead) {
    if (a.lambda)
      for (int k = 0; k < 3 * a.ncmax; ++k) a.lambda[k * B + e] = 0.0;
    if (a.modes)
      for (int k = 0; k < a.ncmax; ++k) a.modes[k * B + e] = DS_MODE_INACTIVE;
    for (int ac = 0; ac < s.na; ++ac) {
      const int k = s.slot[ac];
      if (a.lambda)
        for (int r = 0; r < 3; ++r) a.lambda[(3 * k + r) * B + e] = s.lam[3 * ac + r];
      if (a.modes) a.modes[k * B + e] = uint8_t(s.mode[ac]);
    }
    if (a.iters) a.iters[e] = iters;
  }

  if (a.run != DS_RUN_STEP && !(st & DS_ENV_NONFINITE)) {
    T Vp[NB][6];
    Reduced<NS> rd;
    finish_reduced<NB, NV, NS, T>(m, a, s, Vp, rd, st);
    const int(&off)[NS] = rd.off;
    const int(&sz)[NS] = rd.sz;
    const double(&Rm)[NS][3][2] = rd.Rm;
    const double(&RP)[NS][2][3] = rd.RP;
    const int md = rd.md;

    const T dt = T(a.dt);
    if (a.run == DS_RUN_JAC) {
      // ---- B1/B2/B5/B6: dv = D + Y C X with X = -A^- B (J_c D + F), column by column.  When this
      // thread has more columns than there are rows, the implicit part is applied by rows:
      // P_k = B^T (A^-)^T C^T Y^T e_k (one transposed minimum-norm solve per output row, nv of
      // them) gives row k of Y C A^- B, and every column then costs a dot product per row instead
      // of a solve; otherwise each column solves for its X.
      const int c0 = (3 * NV * chunk) / nchunk, c1 = (3 * NV * (chunk + 1)) / nchunk;
      const bool by_rows = md > 0 && NV < c1 - c0;
      double P[NV][3 * NS];
      if (by_rows) finish_rows<NB, NV, NS, T>(s, rd, P);
      for (int col = c0; col < c1; ++col) {
        const int blk = col / NV, d = col % NV;
        T Dc[NV];
        if (blk < 2) {
          T dtau[NV];
          rnea_tangent<NB, NV, NS, T>(m, s, blk, d, dtau);
          ltl_solve_t(s.L, dtau, NV, m.dof_parent);
          ltl_solve(s.L, dtau, NV, m.dof_parent);
          for (int k = 0; k < NV; ++k) Dc[k] = -dt * dtau[k] + (blk == 1 && k == d ? T(1) : T(0));
        } else {
          for (int k = 0; k < NV; ++k) Dc[k] = (k == d ? dt : T(0));
          ltl_solve_t(s.L, Dc, NV, m.dof_parent);
          ltl_solve(s.L, Dc, NV, m.dof_parent);
        }
        if (by_rows) {
          double rfull[3 * NS];
          for (int ac = 0; ac < s.na; ++ac) {
            T fk[3] = {T(0), T(0), T(0)};
            if (sz[ac] != 0 && blk == 0) fkv_tangent<NB, NV, NS, T>(m, s, Vp, ac, d, fk);
            if (sz[ac] != 0) fk[2] += baumgarte_d<NB, NV, NS, T>(m, a, s, ac, blk, d);
            for (int r = 0; r < 3; ++r) {
              T t = fk[r];
              if (sz[ac] != 0)
                for (int k = m.iv[DS_IX(s.body[ac], NB)] + m.nd[DS_IX(s.body[ac], NB)] - 1; k >= 0; k = m.dof_parent[DS_IX(k, NV)])
                  t += s.Jc[3 * ac + r][k] * Dc[k];           // J_c rows: the body's ancestor dofs only
              rfull[3 * ac + r] = double(t);
            }
          }
          for (int k = 0; k < NV; ++k) {
            double t = 0.0;
            for (int j = 0; j < mdim; ++j) t += P[k][j] * rfull[j];
            Dc[k] -= T(t);
          }
        } else if (md > 0) {
          double rhs[3 * NS], X[3 * NS];
          for (int ac = 0; ac < s.na; ++ac) {
            if (sz[ac] == 0) continue;
            double r3[3];
            T fk[3] = {T(0), T(0), T(0)};
            if (blk == 0) fkv_tangent<NB, NV, NS, T>(m, s, Vp, ac, d, fk);
            fk[2] += baumgarte_d<NB, NV, NS, T>(m, a, s, ac, blk, d);
            for (int r = 0; r < 3; ++r) {
              T t = fk[r];
              for (int k = m.iv[DS_IX(s.body[ac], NB)] + m.nd[DS_IX(s.body[ac], NB)] - 1; k >= 0; k = m.dof_parent[DS_IX(k, NV)])
                t += s.Jc[3 * ac + r][k] * Dc[k];
              r3[r] = double(t);
            }
            if (sz[ac] == 3) {
              for (int r = 0; r < 3; ++r) rhs[off[ac] + r] = -r3[r];
            } else {
              for (int r = 0; r < 2; ++r)
                rhs[off[ac] + r] = -(RP[ac][r][0] * r3[0] + RP[ac][r][1] * r3[1] + RP[ac][r][2] * r3[2]);
            }
          }
          s.lu.solve_mn(rhs, X);
          for (int ac = 0; ac < s.na; ++ac) {
            if (sz[ac] == 0) continue;
            double dl[3];
            if (sz[ac] == 3) { for (int r = 0; r < 3; ++r) dl[r] = X[off[ac] + r]; }
            else { for (int r = 0; r < 3; ++r) dl[r] = Rm[ac][r][0] * X[off[ac]] + Rm[ac][r][1] * X[off[ac] + 1]; }
            for (int r = 0; r < 3; ++r) {
              const T dlr = T(dl[r]);
              for (int k = 0; k < NV; ++k) Dc[k] += s.Y[3 * ac + r][k] * dlr;
            }
          }
        }
        double* out = blk == 0 ? a.dv_dq : (blk == 1 ? a.dv_dv : a.dv_dtau);
        for (int k = 0; k < NV; ++k) out[(k * NV + d) * B + e] = double(Dc[k]);
      }
    } else {
      // ---- B7 vector-Jacobian product (adjoint of the implicit solve, never forming D):
      // z = A^-T C^T Y^T vbar, zeta = B^T z, ubar = vbar - J_c^T zeta, w = M^-1 ubar,
      // q_bar = -dt dtau_q . w - F^T zeta, v_bar = ubar - dt dtau_v . w, tau_bar = dt w.
      // With a cotangent of q+ as well, the position update's adjoint is chained in first (B8).
      T ub[NV], w2[NV];
      double zeta[3 * NS], qadd[NV];
      finish_vjp_head<NB, NV, NS, T>(m, a, e, s, rd, ub, w2, zeta, qadd);
      const int p0 = (2 * NV * chunk) / nchunk, p1 = (2 * NV * (chunk + 1)) / nchunk;
      for (int blk = 0; blk < 2; ++blk)
        for (int d = 0; d < NV; ++d) {
          if (blk * NV + d < p0 || blk * NV + d >= p1) continue;
          T dtau[NV];
          rnea_tangent<NB, NV, NS, T>(m, s, blk, d, dtau);
          T r = T(0);
          for (int k = 0; k < NV; ++k) r += dtau[k] * w2[k];
          r = -dt * r;
          if (blk == 1) r += ub[d];
          const bool stab = gap_term(a);
          for (int ac = 0; ac < s.na && (blk == 0 || stab); ++ac) {
            if (sz[ac] == 0) continue;
            T fk[3] = {T(0), T(0), T(0)};
            if (blk == 0) fkv_tangent<NB, NV, NS, T>(m, s, Vp, ac, d, fk);
            fk[2] += baumgarte_d<NB, NV, NS, T>(m, a, s, ac, blk, d);
            for (int rr = 0; rr < 3; ++rr) r -= fk[rr] * T(zeta[3 * ac + rr]);
          }
          double* out = blk == 0 ? a.q_bar : a.v_bar;
          out[d * B + e] = (blk == 0 && a.qnbar) ? double(r) + qadd[d] : double(r);
        }
      if (lead)
        for (int k = 0; k < NV; ++k) a.tau_bar[k * B + e] = double(dt * w2[k]);
    }
  }
  if (a.status && lead) a.status[e] = st;
}


// Fused path: one thread does the whole step for env e.
template <int NB, int NV, int NS, typename T>
DS_HD void run_env(const DevModel& m, const KArgs& a, const int e) {
  Env<NB, NV, NS, T> s;
  uint32_t st = env_forward<NB, NV, NS, T>(m, a, e, s);
  const int mdim = 3 * s.na;
  // ---- F7/F8 NCP solve and residual check
  int iters = 0;
  for (int r = 0; r < mdim; ++r) s.lam[r] = 0.0;
  if (mdim > 0 && !(st & DS_ENV_NONFINITE)) solve_ncp<Env<NB, NV, NS, T>, T>(s, a, iters, st);
  s.margin = classify(s, s.lam, a.eps_sigma, a.eps_lambda, s.mode);
  if (mdim > 0 && s.margin < a.margin_delta) st |= DS_ENV_NEAR_SWITCH;

  env_finish<NB, NV, NS, T>(m, a, e, s, st, iters);
}

DS_HDI void load_model(DevModel& sm, const DevModel* src_model) {
#ifdef __CUDA_ARCH__
  const int* src = reinterpret_cast<const int*>(src_model);
  int* dst = reinterpret_cast<int*>(&sm);
  for (int k = threadIdx.x; k < int(sizeof(DevModel) / sizeof(int)); k += blockDim.x) dst[k] = src[k];
  __syncthreads();
#else
  sm = *src_model;
#endif
}

// Fused path: one thread per env does everything (no workspace).
template <int NB, int NV, int NS, typename T>
__global__ void __launch_bounds__(128, 4) env_kernel(KArgs a) {
  __shared__ DevModel sm;
  load_model(sm, a.model);
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.n_env) return;
  const int e = DS_IX(a.env_list ? a.env_list[t] : t, a.B);
  if (a.model_id && a.model_id[e] != a.model_index) return;
  run_env<NB, NV, NS, T>(sm, a, e);
}

// ---------------------------------------------------------------------------------- pipeline
// 1. setup: F1-F6 per env, the contact problem (mu, G, g) and a zero ADMM state to the workspace,
//    envs with contacts queued for round 0.
DS_HDI int ds_atomic_add(int32_t* p, int32_t v) {
#ifdef __CUDA_ARCH__
  return atomicAdd(p, v);
#else
  const int32_t old = *p;
  *p += v;
  return old;
#endif
}

// 1. setup: F1-F6 per env; the forward state the finish needs, the contact problem (mu, G, g), rho
//    and K = (G + rho I)^-1, and a zero ADMM state to the workspace; envs with contacts queued for
//    round 0.
template <int NB, int NV, int NS, typename T>
DS_HD void setup_env(const DevModel& m, const KArgs& a, const int e) {
  Env<NB, NV, NS, T> s;
  uint32_t st = env_forward<NB, NV, NS, T>(m, a, e, s);
  store_forward<NB, NV, NS, T>(a, e, s);
  const WsView& w = a.ws;
  const int B = a.B;
  const int mm = 3 * s.na;
  constexpr int NC3 = 3 * NS;
  w.na[e] = s.na;
  w.iters[e] = 0;
  w.stage[e] = 0;
  w.best_r[e] = 1e300;
  for (int i = 0; i < s.na; ++i) w.mu[i * B + e] = s.mu[i];
  for (int i = 0; i < mm; ++i) {
    for (int j = 0; j <= i; ++j) w.G[tri(i, j) * B + e] = s.G(i, j);
    w.g[i * B + e] = s.gd[i];
    w.lam[i * B + e] = 0.0;
    w.ax[i * B + e] = 0.0;
    w.az[i * B + e] = 0.0;
    w.ay[i * B + e] = 0.0;
    w.asx[i * B + e] = double(s.gt[i]);
  }
  if (mm > 0 && !(st & DS_ENV_NONFINITE) && separating(s)) {
    // lambda = 0 solves Eq. 1 (separating()): no ADMM; the modes of that solution go to the finish
    for (int i = 0; i < mm; ++i) s.lam[i] = 0.0;
    int mode[NS];
    const double margin = classify(s, s.lam, a.eps_sigma, a.eps_lambda, mode);
    if (margin < a.margin_delta) st |= DS_ENV_NEAR_SWITCH;
    for (int i = 0; i < s.na; ++i) w.mode[i * B + e] = int8_t(mode[i]);
  } else if (mm > 0 && !(st & DS_ENV_NONFINITE) && a.sched.presolve && presolve_single(s, a, s.lam)) {
    // one contact in contact, the rest breaking: solved here, no ADMM
    for (int i = 0; i < mm; ++i) w.lam[i * B + e] = s.lam[i];
    int mode[NS];
    const double margin = classify(s, s.lam, a.eps_sigma, a.eps_lambda, mode);
    if (margin < a.margin_delta) st |= DS_ENV_NEAR_SWITCH;
    for (int i = 0; i < s.na; ++i) w.mode[i * B + e] = int8_t(mode[i]);
  } else if (mm > 0 && !(st & DS_ENV_NONFINITE)) {
    if (a.solver == DS_ADMM) {
      Admm<NS, T> ad;
      if (!ad.setup(s)) st |= DS_ENV_NONFINITE;
      w.rho[e] = double(ad.rho);
      for (int i = 0; i < NC3; ++i)
        for (int j = 0; j < NC3; ++j) w.K[(i * NC3 + j) * B + e] = double(ad.K[i][j]);
    }
    if (!(st & DS_ENV_NONFINITE)) {
      const int k = ds_atomic_add(&w.counts[0], 1);
      w.list[0][k] = e;
      w.st[e] = st;
      return;
    }
  }
  w.st[e] = st;
  const int k = ds_atomic_add(&w.dcount[0], 1);   // nothing to solve: ready for the finish
  w.dlist[k] = e;
}

template <int NB, int NV, int NS, typename T>
__global__ void __launch_bounds__(128, 4) setup_kernel(KArgs a) {
  __shared__ DevModel sm;
  load_model(sm, a.model);
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.n_env) return;
  const int e = DS_IX(a.env_list ? a.env_list[t] : t, a.B);
  if (a.model_id && a.model_id[e] != a.model_index) return;
  setup_env<NB, NV, NS, T>(sm, a, e);
}

// End of an env's ADMM round: to the Newton queue when its stage ended (tolerance met, iteration
// limit, or the last round), else to the next round's list -- or, from the schedule's speculative
// round on, to the Newton queue as ~e (the Newton stage tries the unconverged iterate and, if that
// fails, returns the env to the next round in the same stage).
__device__ __forceinline__ void route_after_round(const KArgs& a, int e, bool conv, int iters, int32_t* next) {
  const WsView& w = a.ws;
  if (conv || iters >= a.admm_max_iter || a.final_round) {
    const int k = atomicAdd(&w.ncounts[a.round], 1);
    w.nlist[k] = e;
  } else if (a.round >= a.sched.spec_from) {
    const int k = atomicAdd(&w.ncounts[a.round], 1);
    w.nlist[k] = ~e;
  } else {
    const int k = atomicAdd(&w.counts[a.round + 1], 1);
    next[k] = e;
  }
}

// 2a. one ADMM round, one lane per contact slot (NS lanes per env, 32/NS envs per warp): each lane
//     keeps its three rows of K and its contact's x, z, y, sx in registers; the right-hand side is
//     exchanged with warp shuffles and the convergence test is a max-reduction over the env's
//     lanes.  Every env runs at most round_cap iterations; envs whose stage tolerance was met (or
//     that hit the iteration cap) go to the Newton queue, the others to the next round's list.
template <typename T>
__device__ __forceinline__ T group_max(T v, int lanes) {
  for (int off = lanes >> 1; off >= 1; off >>= 1) v = nonneg_max(v, __shfl_xor_sync(0xffffffffu, v, off));
  return v;
}

template <int NS, typename T>
__global__ void __launch_bounds__(128) admm_round_kernel(KArgs a) {
  static_assert(32 % NS == 0, "contact slots must divide the warp");
  constexpr int L = NS, EPW = 32 / NS, NC3 = 3 * NS;
  const WsView& w = a.ws;
  const int n = w.counts[a.round];
  const int B = a.B;
  const int lane = threadIdx.x & 31;
  const int grp = lane / L, li = lane - grp * L;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int32_t* cur = w.list[a.round & 1];
  int32_t* next = w.list[(a.round + 1) & 1];
  for (int base = warp * EPW; base < n; base += nwarps * EPW) {
    const int t = base + grp;
    const bool have = t < n;
    const int e = have ? DS_IX(cur[t], B) : 0;
    const int na = have ? w.na[e] : 0;
    const bool act = li < na;
    T Kr[3][NC3], x[3], z[3], y[3], sx[3], g[3];
    T mu = T(0);
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const int row = 3 * li + r;
#pragma unroll
      for (int c = 0; c < NC3; ++c) Kr[r][c] = act ? T(w.K[(row * NC3 + c) * B + e]) : T(0);
      x[r] = act ? T(w.ax[row * B + e]) : T(0);
      z[r] = act ? T(w.az[row * B + e]) : T(0);
      y[r] = act ? T(w.ay[row * B + e]) : T(0);
      sx[r] = act ? T(w.asx[row * B + e]) : T(0);
      g[r] = act ? T(w.g[row * B + e]) : T(0);
    }
    if (act) mu = T(w.mu[li * B + e]);
    const T rho = have ? T(w.rho[e]) : T(1);
    const T inv_rho = T(1) / rho;
    const T inv1pmu2 = T(1) / (T(1) + mu * mu);
    T gm = fmax(fabs(g[0]), fmax(fabs(g[1]), fabs(g[2])));
    const T gs = fmax(T(1), group_max(gm, L));
    int iters = have ? w.iters[e] : 0;
    const int stage = have ? w.stage[e] : 0;
    const T te = T(stage_eps<T>(a, stage));
    bool running = have && iters < a.admm_max_iter;
    bool conv = false;
    for (int k = 0; k < a.round_cap; ++k) {
      if (!__any_sync(0xffffffffu, running)) break;
      T rhs[3] = {T(0), T(0), T(0)};
      if (act) admm_rhs(mu, z, y, g, sx, rho, rhs);
      T full[NC3];
#pragma unroll
      for (int j = 0; j < NS; ++j)
#pragma unroll
        for (int r = 0; r < 3; ++r) full[3 * j + r] = __shfl_sync(0xffffffffu, rhs[r], grp * L + j);
      T xn[3] = {x[0], x[1], x[2]}, zn[3] = {z[0], z[1], z[2]}, yn[3] = {y[0], y[1], y[2]};
      T sn[3] = {sx[0], sx[1], sx[2]};
      T rp = T(0), rd = T(0), zmax = T(1);
      const bool chk = (iters + 1) % DS_ADMM_CHECK == 0;
      if (act) admm_update<NC3, T>(Kr, full, rhs, g, mu, rho, inv_rho, inv1pmu2, xn, zn, yn, sn, rp, rd, zmax, chk);
      if (__any_sync(0xffffffffu, running && chk)) {
        rp = group_max(rp, L);
        rd = group_max(rd, L);
        zmax = group_max(zmax, L);
      }
      if (running) {
#pragma unroll
        for (int r = 0; r < 3; ++r) { x[r] = xn[r]; z[r] = zn[r]; y[r] = yn[r]; sx[r] = sn[r]; }
        ++iters;
        rd *= rho;
        if (chk && rp <= te * zmax && rd <= te * gs) { conv = true; running = false; }
        else if (iters >= a.admm_max_iter) running = false;
      }
    }
    if (have) {
      if (act) {
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          const int row = 3 * li + r;
          w.ax[row * B + e] = double(x[r]);
          w.az[row * B + e] = double(z[r]);
          w.ay[row * B + e] = double(y[r]);
          w.asx[row * B + e] = double(sx[r]);
        }
      }
      if (li == 0) {
        w.iters[e] = iters;
        route_after_round(a, e, conv, iters, next);
      }
    }
  }
}

// 2a'. the same ADMM round with one lane per row of K (3 NS rows, rounded up to a power-of-two
//      group of lanes per env).  Each lane does a third of the 3-row form's fused multiply-adds
//      per iteration, at fewer envs per warp.  The late rounds hold few envs, and their time is
//      the latency of one warp's iterations: the FP64 pipe is charged per warp instruction, so a
//      shorter instruction stream per iteration is what shortens them.  Every row's arithmetic is
//      the 3-row form's, in the same order, so the two kernels hand envs to each other between
//      rounds without changing any result.
template <int NS>
struct WideShape {
  static constexpr int R = 3 * NS;
  static constexpr int L = R <= 4 ? 4 : (R <= 8 ? 8 : (R <= 16 ? 16 : 32));
  static constexpr bool kOk = R <= 32;
};

template <int NS, typename T>
__global__ void __launch_bounds__(128) admm_round_wide_kernel(KArgs a) {
  static_assert(WideShape<NS>::kOk, "3 NS rows must fit in a warp");
  constexpr int L = WideShape<NS>::L, EPW = 32 / L, NC3 = 3 * NS;
  const WsView& w = a.ws;
  const int n = w.counts[a.round];
  const int B = a.B;
  const int lane = threadIdx.x & 31;
  const int grp = lane / L, li = lane - grp * L;
  const int gb = grp * L;
  const int ci = li < NC3 ? li / 3 : NS - 1, kc = li < NC3 ? li - 3 * (li / 3) : 0;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const int32_t* cur = w.list[a.round & 1];
  int32_t* next = w.list[(a.round + 1) & 1];
  for (int base = warp * EPW; base < n; base += nwarps * EPW) {
    const int t = base + grp;
    const bool have = t < n;
    const int e = have ? DS_IX(cur[t], B) : 0;
    const int na = have ? w.na[e] : 0;
    const bool act = li < 3 * na;
    T Kr[NC3];
#pragma unroll
    for (int c = 0; c < NC3; ++c) Kr[c] = act ? T(w.K[(li * NC3 + c) * B + e]) : T(0);
    T x = act ? T(w.ax[li * B + e]) : T(0);
    T z = act ? T(w.az[li * B + e]) : T(0);
    T y = act ? T(w.ay[li * B + e]) : T(0);
    T sx = act ? T(w.asx[li * B + e]) : T(0);
    const T g = act ? T(w.g[li * B + e]) : T(0);
    const T mu = act ? T(w.mu[ci * B + e]) : T(0);
    const T rho = have ? T(w.rho[e]) : T(1);
    const T inv_rho = T(1) / rho;
    const T inv1pmu2 = T(1) / (T(1) + mu * mu);
    const T gs = fmax(T(1), group_max(T(fabs(g)), L));
    int iters = have ? w.iters[e] : 0;
    const int stage = have ? w.stage[e] : 0;
    const T te = T(stage_eps<T>(a, stage));
    bool running = have && iters < a.admm_max_iter;
    bool conv = false;
    const T relax = T(1.6);
    for (int k = 0; k < a.round_cap; ++k) {
      if (!__any_sync(0xffffffffu, running)) break;
      // right-hand side of this row (the De Saxce term from the contact's tangential sigma)
      const T s0 = __shfl_sync(0xffffffffu, sx, gb + 3 * ci);
      const T s1 = __shfl_sync(0xffffffffu, sx, gb + 3 * ci + 1);
      T nt, inv;
      norm_and_inv(s0, s1, nt, inv);
      T rhs = rho * z - y - g;
      if (kc == 2) rhs = rhs - mu * nt;
      if (!act) rhs = T(0);
      T acc = T(0);
#pragma unroll
      for (int c = 0; c < NC3; ++c) acc += Kr[c] * __shfl_sync(0xffffffffu, rhs, gb + c);
      const T xn = acc;
      const T sxn = kc < 2 ? rhs - rho * acc + g : sx;
      const T xh = relax * xn + (T(1) - relax) * z;
      const T wv = xh + y * inv_rho;
      T wc[3], pr[3];
#pragma unroll
      for (int r = 0; r < 3; ++r) wc[r] = __shfl_sync(0xffffffffu, wv, gb + 3 * ci + r);
      proj_cone_fast(wc, mu, inv1pmu2, pr);
      const T zn = kc == 0 ? pr[0] : (kc == 1 ? pr[1] : pr[2]);
      const bool chk = (iters + 1) % DS_ADMM_CHECK == 0;
      T rp = T(0), rd = T(0), zmax = T(1);
      if (act && chk) {
        rd = fabs(zn - z);
        rp = fabs(xn - zn);
        zmax = nonneg_max(zmax, T(fabs(zn)));
      }
      if (__any_sync(0xffffffffu, running && chk)) {
        rp = group_max(rp, L);
        rd = group_max(rd, L);
        zmax = group_max(zmax, L);
      }
      if (running) {
        x = xn;
        z = zn;
        y = y + rho * (xh - zn);
        sx = sxn;
        ++iters;
        rd *= rho;
        if (chk && rp <= te * zmax && rd <= te * gs) { conv = true; running = false; }
        else if (iters >= a.admm_max_iter) running = false;
      }
    }
    if (have) {
      if (act) {
        w.ax[li * B + e] = double(x);
        w.az[li * B + e] = double(z);
        w.ay[li * B + e] = double(y);
        w.asx[li * B + e] = double(sx);
      }
      if (li == 0) {
        w.iters[e] = iters;
        route_after_round(a, e, conv, iters, next);
      }
    }
  }
}

// 2a''. the row-per-lane round split over the two warps of a 64-thread CTA, for the late rounds:
//       they hold few envs, each round lasts as long as its slowest env's chain of iterations, and
//       an SM sub-partition's FP64 pipe takes one warp instruction at a time.  Warp 0 keeps K, x,
//       z, y and runs the x-step, the projection and the multiplier update; warp 1 (another
//       sub-partition) keeps sx and forms the next iteration's De Saxce norm and the convergence
//       test from what warp 0 leaves in shared memory, so those leave warp 0's instruction stream.
//       Where two lanes per row fit in the warp (up to 16 lanes per env, an even number of
//       rows), warp 0 splits the x-step K * rhs: each of a row's two lanes sums half the columns
//       and the row's value is low half + high half (the other per-row work is mirrored on both
//       lanes): 6 fused multiply-adds and one add instead of 12 for 4 slots; the x-step then
//       rounds differently from the other forms (results agree to the solver tolerance).  Named
//       barriers order the hand-offs (warp-uniform; 64 threads each):
//         kDs  warp 1 arrives, warp 0 waits: the De Saxce norms of the coming iteration and the
//              outcome of the previous iteration's convergence test are in place;
//         kRhs warp 0 arrives, warp 1 waits: this iteration's right-hand side, x-step and flags
//              are in place (or the env loop ends: stop flag);
//         kZ   warp 0 arrives, warp 1 waits, on test iterations only: the projected z is in place.
//       A test's outcome reaches warp 0 at the top of the next iteration, before it decides to go
//       on, so the stopping rule is the other forms'.
__device__ __forceinline__ void named_bar_sync(int id, int threads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}
__device__ __forceinline__ void named_bar_arrive(int id, int threads) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

template <int NS>
struct PairShape {
  static constexpr int L = WideShape<NS>::L;                        // lanes per half-group
  static constexpr int NC3 = 3 * NS;
  static constexpr int H = (2 * L <= 32 && NC3 % 2 == 0) ? 2 : 1;   // halves of the x-step
  static constexpr int LG = H * L;                                  // lanes per env
  static constexpr int EPW = 32 / LG;                               // envs per warp
  static constexpr int NH = NC3 / H;                                // columns of K per lane
};

template <int NS, typename T>
__global__ void __launch_bounds__(64) admm_round_pair_kernel(KArgs a) {
  static_assert(WideShape<NS>::kOk, "3 NS rows must fit in a warp");
  using PS = PairShape<NS>;
  constexpr int L = PS::L, H = PS::H, LG = PS::LG, EPW = PS::EPW, NH = PS::NH, NC3 = 3 * NS;
  constexpr int kDs = 1, kRhs = 2, kZ = 3;
  __shared__ T s_rhs[32], s_x[32], s_z[32], s_zold[32], s_nt[32];
  __shared__ int s_run[EPW], s_chk[EPW], s_conv[EPW], s_stop;
  const WsView& w = a.ws;
  const int n = w.counts[a.round];
  const int B = a.B;
  const int role = threadIdx.x >> 5;          // 0: x-step / projection, 1: De Saxce term and test
  const int lane = threadIdx.x & 31;
  // lane = env group grp, half h (H = 2: the x-step's columns split in two halves, each summed by
  // its own lane of the row and the two partial sums added low + high; the other per-row work is
  // mirrored on both halves), row li
  const int grp = lane / LG, qi = lane - grp * LG, h = qi / L, li = qi - h * L;
  const int gb = grp * LG, hb = gb + h * L;
  const int ci = li < NC3 ? li / 3 : NS - 1, kc = li < NC3 ? li - 3 * (li / 3) : 0;
  const int32_t* cur = w.list[a.round & 1];
  int32_t* next = w.list[(a.round + 1) & 1];
  for (int base = blockIdx.x * EPW; base < n; base += gridDim.x * EPW) {
    const int t = base + grp;
    const bool have = t < n;
    const int e = have ? DS_IX(cur[t], B) : 0;
    const int na = have ? w.na[e] : 0;
    const bool act = li < 3 * na;
    const T g = act ? T(w.g[li * B + e]) : T(0);
    const T rho = have ? T(w.rho[e]) : T(1);
    const T gs = fmax(T(1), group_max(T(fabs(g)), L));
    const int stage = have ? w.stage[e] : 0;
    const T te = T(stage_eps<T>(a, stage));
    if (role == 1) {
      T sx = act ? T(w.asx[li * B + e]) : T(0);
      {
        const T s0 = __shfl_sync(0xffffffffu, sx, hb + 3 * ci);
        const T s1 = __shfl_sync(0xffffffffu, sx, hb + 3 * ci + 1);
        T nt, inv;
        norm_and_inv(s0, s1, nt, inv);
        s_nt[lane] = nt;
        if (qi == 0) s_conv[grp] = 0;
      }
      named_bar_arrive(kDs, 64);
      for (;;) {
        named_bar_sync(kRhs, 64);
        if (s_stop) break;
        const bool run = s_run[grp] != 0, chk = s_chk[grp] != 0;
        bool anychk = false;
#pragma unroll
        for (int q = 0; q < EPW; ++q) anychk = anychk || (s_run[q] != 0 && s_chk[q] != 0);
        const T rhs = s_rhs[lane], xn = s_x[lane];
        if (run && kc < 2) sx = rhs - rho * xn + g;
        const T s0 = __shfl_sync(0xffffffffu, sx, hb + 3 * ci);
        const T s1 = __shfl_sync(0xffffffffu, sx, hb + 3 * ci + 1);
        T nt, inv;
        norm_and_inv(s0, s1, nt, inv);
        bool conv = false;
        if (anychk) {
          named_bar_sync(kZ, 64);
          T rp = T(0), rd = T(0), zmax = T(1);
          if (act && run && chk) {
            const T zn = s_z[lane];
            rd = fabs(zn - s_zold[lane]);
            rp = fabs(xn - zn);
            zmax = nonneg_max(zmax, T(fabs(zn)));
          }
          rp = group_max(rp, L);
          rd = group_max(rd, L);
          zmax = group_max(zmax, L);
          rd *= rho;
          conv = run && chk && rp <= te * zmax && rd <= te * gs;
        }
        s_nt[lane] = nt;
        if (qi == 0) s_conv[grp] = conv ? 1 : 0;
        named_bar_arrive(kDs, 64);
      }
      if (have && act && h == 0) w.asx[li * B + e] = double(sx);
      continue;
    }
    T Kr[NH];
#pragma unroll
    for (int j = 0; j < NH; ++j) Kr[j] = act ? T(w.K[(li * NC3 + h * NH + j) * B + e]) : T(0);
    T x = act ? T(w.ax[li * B + e]) : T(0);
    T z = act ? T(w.az[li * B + e]) : T(0);
    T y = act ? T(w.ay[li * B + e]) : T(0);
    const T mu = act ? T(w.mu[ci * B + e]) : T(0);
    const T inv_rho = T(1) / rho;
    const T inv1pmu2 = T(1) / (T(1) + mu * mu);
    int iters = have ? w.iters[e] : 0;
    bool running = have && iters < a.admm_max_iter;
    bool conv = false, pend = false;
    const T relax = T(1.6);
    for (int k = 0;; ++k) {
      named_bar_sync(kDs, 64);
      if (pend && s_conv[grp]) { conv = true; running = false; }
      pend = false;
      if (!(k < a.round_cap && __any_sync(0xffffffffu, running))) {
        if (lane == 0) s_stop = 1;
        named_bar_arrive(kRhs, 64);
        break;
      }
      const bool chk = (iters + 1) % DS_ADMM_CHECK == 0;
      const T nt = s_nt[lane];
      T rhs = rho * z - y - g;
      if (kc == 2) rhs = rhs - mu * nt;
      if (!act) rhs = T(0);
      T acc = T(0);
#pragma unroll
      for (int j = 0; j < NH; ++j) acc += Kr[j] * __shfl_sync(0xffffffffu, rhs, gb + h * NH + j);
      T xn = acc;
      if constexpr (H == 2) {
        const T other = __shfl_xor_sync(0xffffffffu, acc, L);
        xn = h == 0 ? acc + other : other + acc;
      }
      s_rhs[lane] = rhs;
      s_x[lane] = xn;
      s_zold[lane] = z;
      if (qi == 0) { s_run[grp] = running ? 1 : 0; s_chk[grp] = chk ? 1 : 0; }
      if (lane == 0) s_stop = 0;
      const bool anychk = __any_sync(0xffffffffu, running && chk);
      named_bar_arrive(kRhs, 64);
      const T xh = relax * xn + (T(1) - relax) * z;
      const T wv = xh + y * inv_rho;
      T wc[3], pr[3];
#pragma unroll
      for (int r = 0; r < 3; ++r) wc[r] = __shfl_sync(0xffffffffu, wv, hb + 3 * ci + r);
      proj_cone_fast(wc, mu, inv1pmu2, pr);
      const T zn = kc == 0 ? pr[0] : (kc == 1 ? pr[1] : pr[2]);
      if (anychk) {
        s_z[lane] = zn;
        named_bar_arrive(kZ, 64);
      }
      if (running) {
        x = xn;
        z = zn;
        y = y + rho * (xh - zn);
        ++iters;
        pend = chk;
        if (iters >= a.admm_max_iter) running = false;
      }
    }
    if (have) {
      if (act && h == 0) {
        w.ax[li * B + e] = double(x);
        w.az[li * B + e] = double(z);
        w.ay[li * B + e] = double(y);
      }
      if (qi == 0) {
        w.iters[e] = iters;
        route_after_round(a, e, conv, iters, next);
      }
    }
  }
}

// 2b. the Newton / active-set stage for the envs whose ADMM stage ended in this round (one thread
//     per env): accept, or move to the next (tighter) stage and queue for the next round.
// 2a''. one round of projected Gauss-Seidel (the ds_options ncp_solver = DS_PGS form of the NCP
//       iteration), one thread per env: loads the env's contact problem and iterate, runs at most
//       round_cap sweeps (or to the stage tolerance), stores the iterate and routes the env like
//       the ADMM rounds.
template <int NS, typename T>
struct PgsData {
  static constexpr int NC3 = 3 * NS;
  int na;
  double mu[NS];
  T Gt[NC3][NC3], gt[NC3];
};

template <int NS, typename T>
__global__ void __launch_bounds__(128) pgs_round_kernel(KArgs a) {
  const WsView& w = a.ws;
  const int n = w.counts[a.round];
  const int B = a.B;
  const int32_t* cur = w.list[a.round & 1];
  int32_t* next = w.list[(a.round + 1) & 1];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const int e = DS_IX(cur[t], B);
    PgsData<NS, T> d;
    d.na = w.na[e];
    const int m = 3 * d.na;
    for (int i = 0; i < d.na; ++i) d.mu[i] = w.mu[i * B + e];
    for (int i = 0; i < m; ++i) {
      for (int j = 0; j <= i; ++j) {
        const T gij = T(w.G[tri(i, j) * B + e]);
        d.Gt[i][j] = gij;
        d.Gt[j][i] = gij;
      }
      d.gt[i] = T(w.g[i * B + e]);
    }
    Pgs<NS, T> it;
    it.setup(d);
    for (int i = 0; i < m; ++i) it.z[i] = T(w.az[i * B + e]);
    int iters = w.iters[e];
    const T te = T(stage_eps<T>(a, w.stage[e]));
    bool conv = false;
    for (int k = 0; k < a.round_cap && iters < a.admm_max_iter; ++k) {
      ++iters;
      if (it.iterate(d, te, true)) { conv = true; break; }
    }
    for (int i = 0; i < m; ++i) w.az[i * B + e] = double(it.z[i]);
    w.iters[e] = iters;
    route_after_round(a, e, conv, iters, next);
  }
}

template <int NS, typename T>
DS_HD void newton_env(const KArgs& a, const int entry) {
  // entry = e: the env's ADMM stage ended; ~e: a speculative attempt on an unconverged iterate
  const bool spec = entry < 0;
  const int e = DS_IX(spec ? ~entry : entry, a.B);
  const WsView& w = a.ws;
  const int B = a.B;
  Ncp<NS, T> p;
  p.na = w.na[e];
  const int m = 3 * p.na;
  for (int i = 0; i < p.na; ++i) p.mu[i] = w.mu[i * B + e];
  for (int i = 0; i < m; ++i) {
    for (int j = 0; j <= i; ++j) {
      const double gij = w.G[tri(i, j) * B + e];
      p.Gt[i][j] = T(gij);
      p.Gt[j][i] = T(gij);
      if constexpr (!Ncp<NS, T>::kDouble) { p.Gd_[i][j] = gij; p.Gd_[j][i] = gij; }
    }
    p.gd[i] = w.g[i * B + e];
    p.gt[i] = T(p.gd[i]);
  }
  uint32_t st = w.st[e];
  T z[3 * NS];
  for (int i = 0; i < m; ++i) z[i] = T(w.az[i * B + e]);
  int stage = w.stage[e];
  const int iters = w.iters[e];
  double best[3 * NS], best_r = w.best_r[e];
  for (int i = 0; i < m; ++i) best[i] = w.lam[i * B + e];
  const double eps = stage_eps<T>(a, stage);
  const bool ok = newton_stage(p, z, eps, a, best, best_r, a.round == a.sched.spec_from);
  for (int i = 0; i < m; ++i) w.lam[i * B + e] = best[i];
  if (ok || (!spec && (iters >= a.admm_max_iter || stage + 1 >= num_stages<T>() || a.final_round))) {
    for (int i = 0; i < m; ++i) p.lam[i] = best[i];
    if (!ok) st |= DS_ENV_NOT_CONVERGED;
    int mode[NS];
    const double margin = classify(p, p.lam, a.eps_sigma, a.eps_lambda, mode);
    if (margin < a.margin_delta) st |= DS_ENV_NEAR_SWITCH;
    for (int i = 0; i < p.na; ++i) w.mode[i * B + e] = int8_t(mode[i]);
    w.st[e] = st;
    const int k = ds_atomic_add(&w.dcount[0], 1);
    w.dlist[k] = e;
  } else {
    if (!spec) w.stage[e] = stage + 1;
    w.best_r[e] = best_r;
    const int k = ds_atomic_add(&w.counts[a.round + 1], 1);
    w.list[(a.round + 1) & 1][k] = e;
  }
}

template <int NS, typename T>
__global__ void __launch_bounds__(128) newton_kernel(KArgs a) {
  const int n = a.ws.ncounts[a.round];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x)
    newton_env<NS, T>(a, a.ws.nlist[t]);
}

// 3. finish: the forward state the setup stored, then F9 and the derivatives with lambda and the
//    modes from the workspace.
template <int NB, int NV, int NS, typename T>
DS_HD void finish_env(const DevModel& m, const KArgs& a, const int e, int chunk = 0, int nchunk = 1) {
  // The forward quantities come from the setup (load_forward), so a finish thread, and each of the
  // threads an env's columns are split over, does only F9 and its share of the derivatives.
  Env<NB, NV, NS, T> s;
  load_forward<NB, NV, NS, T>(m, a, e, s);
  const WsView& w = a.ws;
  const int B = a.B;
  const int mm = 3 * s.na;
  for (int i = 0; i < mm; ++i) s.lam[i] = w.lam[i * B + e];
  if (mm > 0 && !(w.st[e] & DS_ENV_NONFINITE)) {
    for (int i = 0; i < s.na; ++i) s.mode[i] = w.mode[i * B + e];
  } else {
    s.margin = classify(s, s.lam, a.eps_sigma, a.eps_lambda, s.mode);
  }
  env_finish<NB, NV, NS, T>(m, a, e, s, w.st[e], w.iters[e], chunk, nchunk);
}

// Finish from a tape: F1-F6, then lambda, the modes and the status of env e from the tape of a
// preceding sim_step on the same inputs, then F9 and the derivatives (the VJP of exactly the
// solution the forward call returned, without solving the NCP again).
template <int NB, int NV, int NS, typename T>
DS_HD void finish_tape_env(const DevModel& m, const KArgs& a, const int e, int chunk, int nchunk) {
  Env<NB, NV, NS, T> s;
  const uint32_t fst = env_forward<NB, NV, NS, T>(m, a, e, s);
  const int B = a.B;
  const uint32_t st = a.tstat[e] | (fst & DS_ENV_NONFINITE);
  for (int ac = 0; ac < s.na; ++ac)
    for (int r = 0; r < 3; ++r) s.lam[3 * ac + r] = a.tlam[(3 * s.slot[ac] + r) * B + e];
  if (s.na > 0 && !(st & DS_ENV_NONFINITE)) {
    for (int ac = 0; ac < s.na; ++ac) s.mode[ac] = a.tmodes[s.slot[ac] * B + e];
  } else {
    s.margin = classify(s, s.lam, a.eps_sigma, a.eps_lambda, s.mode);
  }
  env_finish<NB, NV, NS, T>(m, a, e, s, st, 0, chunk, nchunk);
}

// ------------------------------------------------------------------------ split finish
// The finish in two kernels (schedule finish_split): a prep kernel, one thread per env, does F9,
// the B1 pass, the reduced system and its factor, and either the rows P of the implicit part
// (Jacobians) or the adjoint vectors (VJP), and stores what the derivative columns read (a
// ColState) in the env's column of the workspace's forward-state rows, which it has just read.  A
// column kernel then runs one warp per env: the warp stages the env's ColState in shared memory
// and its lanes take the 3 nv Jacobian columns (2 nv dof passes of the VJP), so that the tree
// passes of the columns read shared memory instead of a per-thread copy of the env in local
// memory.  An env's columns are the per-thread finish's by-rows columns, term for term; in the
// mixed form P is applied in FP32 (the per-thread finish applies it in FP64).
template <int NB, int NV, int NS, typename T>
struct ColState {
  static constexpr int NC3 = 3 * NS;
  T S[NV][6];
  T v[NV], astar[NV];
  T I[NB][10];
  T V[NB][6], A[NB][6], VJ[NB][6], IV[NB][6], IA[NB][6], Fc[NB][6], Vp[NB][6];
  T L[NV * (NV + 1) / 2];
  T x[NS][3], c[NS][3], f[NS][3];
  T fr[3][3];
  T Jc[NC3][NV];
  T P[NV][NC3];                 // Jacobians: rows of the implicit part
  T w2[NV], ub[NV], zeta[NC3];  // VJP: adjoint vectors
  double phi[NS];
  double qadd[NV];              // VJP: the position update's adjoint (with a cotangent of q+)
  int body[NS];
  int act[NS];                  // 1: the contact is in the reduced system (sticking or sliding)
  int na;
  int md;

  // Every member as (pointer, count), in storage order: the rows of the stored form.
  template <class F>
  DS_HD void visit(F&& fn) {
    fn(&S[0][0], NV * 6); fn(v, NV); fn(astar, NV); fn(&I[0][0], NB * 10);
    fn(&V[0][0], NB * 6); fn(&A[0][0], NB * 6); fn(&VJ[0][0], NB * 6); fn(&IV[0][0], NB * 6);
    fn(&IA[0][0], NB * 6); fn(&Fc[0][0], NB * 6); fn(&Vp[0][0], NB * 6);
    fn(L, NV * (NV + 1) / 2); fn(&x[0][0], NS * 3); fn(&c[0][0], NS * 3); fn(&f[0][0], NS * 3);
    fn(&fr[0][0], 9); fn(&Jc[0][0], NC3 * NV); fn(&P[0][0], NV * NC3); fn(w2, NV); fn(ub, NV); fn(zeta, NC3);
    fn(phi, NS); fn(qadd, NV); fn(body, NS); fn(act, NS); fn(&na, 1); fn(&md, 1);
  }
  static constexpr int kRows = ds_colstate_rows(NB, NV, NS);
  // first row of P in the stored form (the members visit() lists before it)
  static constexpr int kOffP = 6 * NV + 2 * NV + 10 * NB + 7 * 6 * NB + NV * (NV + 1) / 2 + 9 * NS + 9 + 3 * NS * NV;
};

// Prep for env e, in two parts around a warp barrier: prep_load reads the env's forward state
// (and its impulse and modes); prep_store, after every thread of the env has read it, writes the
// ColState over the same rows.  With nch > 1 threads per env (Jacobians), chunk c computes the
// rows k = c, c + nch, ... of P (each chunk factors the reduced system itself) and chunk 0 does F9,
// the step's outputs and the rest of the ColState; the status of the derivative part travels in
// w.st to the column kernel, which writes it.
template <int NB, int NV, int NS, typename T>
DS_HD void prep_load(const DevModel& m, const KArgs& a, const int e, Env<NB, NV, NS, T>& s) {
  load_forward<NB, NV, NS, T>(m, a, e, s);
  const WsView& w = a.ws;
  const int B = a.B;
  const int mm = 3 * s.na;
  for (int i = 0; i < mm; ++i) s.lam[i] = w.lam[i * B + e];
  if (mm > 0 && !(w.st[e] & DS_ENV_NONFINITE)) {
    for (int i = 0; i < s.na; ++i) s.mode[i] = w.mode[i * B + e];
  } else {
    s.margin = classify(s, s.lam, a.eps_sigma, a.eps_lambda, s.mode);
  }
}

template <int NB, int NV, int NS, typename T>
DS_HD void prep_store(const DevModel& m, const KArgs& a, const int e, Env<NB, NV, NS, T>& s, int chunk, int nch) {
  using CS = ColState<NB, NV, NS, T>;
  const WsView& w = a.ws;
  const int B = a.B;
  const int mm = 3 * s.na;
  const bool lead = chunk == 0;
  KArgs a1 = a;
  a1.run = DS_RUN_STEP;                       // F9 (and, from chunk 0, the step's outputs) only
  a1.status = nullptr;
  uint32_t st = w.st[e];
  const int iters = w.iters[e];
  env_finish<NB, NV, NS, T>(m, a1, e, s, st, iters, chunk, nch);
  for (int k = 0; k < NV; ++k)
    if (!isfinite(double(s.vn[k]))) st |= DS_ENV_NONFINITE;
  double* fw = w.fw;
  constexpr int kOffP = CS::kOffP;
  CS cs;
  cs.na = s.na;
  cs.md = 0;
  if (!(st & DS_ENV_NONFINITE)) {
    T Vp[NB][6];
    Reduced<NS> rd;
    finish_reduced<NB, NV, NS, T>(m, a, s, Vp, rd, st);
    cs.md = rd.md;
    for (int i = 0; i < NB; ++i)
      for (int k = 0; k < 6; ++k) cs.Vp[i][k] = Vp[i][k];
    for (int ac = 0; ac < NS; ++ac) cs.act[ac] = ac < s.na && rd.sz[ac] != 0;
    if (a.run == DS_RUN_JAC) {
      double P[NV][3 * NS];
      if (rd.md > 0) finish_rows<NB, NV, NS, T>(s, rd, P, chunk, nch);
      for (int k = chunk; k < NV; k += nch)
        for (int j = 0; j < 3 * NS; ++j)
          fw[size_t(kOffP + k * 3 * NS + j) * B + e] = double(T(rd.md > 0 && j < mm ? P[k][j] : 0.0));
    } else if (lead) {
      double zeta[3 * NS], qadd[NV];
      finish_vjp_head<NB, NV, NS, T>(m, a, e, s, rd, cs.ub, cs.w2, zeta, qadd);
      for (int j = 0; j < 3 * NS; ++j) cs.zeta[j] = T(j < mm ? zeta[j] : 0.0);
      for (int k = 0; k < NV; ++k) cs.qadd[k] = a.qnbar ? qadd[k] : 0.0;
    }
  }
  if (!lead) return;
  w.st[e] = st;
  for (int k = 0; k < NV; ++k) {
    for (int j = 0; j < 6; ++j) cs.S[k][j] = s.S[k][j];
    cs.v[k] = s.v[k];
    cs.astar[k] = s.astar[k];
  }
  for (int i = 0; i < NB; ++i) {
    for (int k = 0; k < 10; ++k) cs.I[i][k] = s.I[i][k];
    for (int k = 0; k < 6; ++k) {
      cs.V[i][k] = s.V[i][k]; cs.A[i][k] = s.A[i][k]; cs.VJ[i][k] = s.VJ[i][k];
      cs.IV[i][k] = s.IV[i][k]; cs.IA[i][k] = s.IA[i][k]; cs.Fc[i][k] = s.Fc[i][k];
    }
  }
  for (int k = 0; k < NV * (NV + 1) / 2; ++k) cs.L[k] = s.L[k];
  for (int ac = 0; ac < NS; ++ac) {
    for (int k = 0; k < 3; ++k) { cs.x[ac][k] = s.x[ac][k]; cs.c[ac][k] = s.c[ac][k]; cs.f[ac][k] = s.f[ac][k]; }
    cs.phi[ac] = s.phi[ac];
    cs.body[ac] = s.body[ac];
  }
  for (int r = 0; r < 3; ++r)
    for (int k = 0; k < 3; ++k) cs.fr[r][k] = s.fr[r][k];
  for (int r = 0; r < 3 * NS; ++r)
    for (int k = 0; k < NV; ++k) cs.Jc[r][k] = s.Jc[r][k];
  int row = 0;
  const void* skip = (a.run == DS_RUN_JAC) ? static_cast<const void*>(&cs.P[0][0]) : nullptr;
  cs.visit([&](auto* ptr, int n) {
    if (static_cast<const void*>(ptr) != skip) {      // the rows of P were written by their chunks
      for (int i = 0; i < n; ++i) fw[size_t(DS_IX(row + i, CS::kRows)) * B + e] = double(ptr[i]);
    } else if (row != kOffP) {
      (void)DS_IX(-1, 1);                              // checked build: the layout disagrees
    }
    row += n;
  });
}

// Jacobian column (blk, d) of the env in cs: D's column (tree tangent pass, M^-1) minus the
// implicit part sum_j P[k][j] (J_c D + F)_j (Dc, nv entries).
template <int NB, int NV, int NS, typename T>
DS_HD void split_jac_column(const DevModel& m, const KArgs& a, const ColState<NB, NV, NS, T>& cs, int blk, int d,
                            T* Dc) {
  const T dt = T(a.dt);
  if (blk < 2) {
    T dtau[NV];
    rnea_tangent_stack<NB, NV, NS, T>(m, cs, blk, d, dtau);
    ltl_solve_t(cs.L, dtau, NV, m.dof_parent);
    ltl_solve(cs.L, dtau, NV, m.dof_parent);
    for (int k = 0; k < NV; ++k) Dc[k] = -dt * dtau[k] + (blk == 1 && k == d ? T(1) : T(0));
  } else {
    for (int k = 0; k < NV; ++k) Dc[k] = (k == d ? dt : T(0));
    ltl_solve_t(cs.L, Dc, NV, m.dof_parent);
    ltl_solve(cs.L, Dc, NV, m.dof_parent);
  }
  if (cs.md == 0) return;
  const int mdim = 3 * cs.na;
  T rfull[3 * NS];
  for (int ac = 0; ac < cs.na; ++ac) {
    T fk[3] = {T(0), T(0), T(0)};
    if (cs.act[ac] && blk == 0) fkv_tangent<NB, NV, NS, T>(m, cs, cs.Vp, ac, d, fk);
    if (cs.act[ac]) fk[2] += baumgarte_d<NB, NV, NS, T>(m, a, cs, ac, blk, d);
    for (int r = 0; r < 3; ++r) {
      T t = fk[r];
      if (cs.act[ac])
        for (int k = m.iv[DS_IX(cs.body[ac], NB)] + m.nd[DS_IX(cs.body[ac], NB)] - 1; k >= 0; k = m.dof_parent[DS_IX(k, NV)])
          t += cs.Jc[3 * ac + r][k] * Dc[k];
      rfull[3 * ac + r] = t;
    }
  }
  for (int k = 0; k < NV; ++k) {
    T t = T(0);
    for (int j = 0; j < mdim; ++j) t += cs.P[k][j] * rfull[j];
    Dc[k] -= t;
  }
}

// VJP entry p (blk = p / nv, dof d = p % nv) of the env in cs: q_bar or v_bar.
template <int NB, int NV, int NS, typename T>
DS_HD double split_vjp_entry(const DevModel& m, const KArgs& a, const ColState<NB, NV, NS, T>& cs, int blk, int d) {
  const T dt = T(a.dt);
  T dtau[NV];
  rnea_tangent_stack<NB, NV, NS, T>(m, cs, blk, d, dtau);
  T r = T(0);
  for (int k = 0; k < NV; ++k) r += dtau[k] * cs.w2[k];
  r = -dt * r;
  if (blk == 1) r += cs.ub[d];
  const bool stab = gap_term(a);
  for (int ac = 0; ac < cs.na && (blk == 0 || stab); ++ac) {
    if (!cs.act[ac]) continue;
    T fk[3] = {T(0), T(0), T(0)};
    if (blk == 0) fkv_tangent<NB, NV, NS, T>(m, cs, cs.Vp, ac, d, fk);
    fk[2] += baumgarte_d<NB, NV, NS, T>(m, a, cs, ac, blk, d);
    for (int rr = 0; rr < 3; ++rr) r -= fk[rr] * cs.zeta[3 * ac + rr];
  }
  return (blk == 0 && a.qnbar) ? double(r) + cs.qadd[d] : double(r);
}

// Prep kernel: a.nchunk threads per env of the launch's range (a power of two <= 32, so that an
// env's threads share a warp), in CTAs of one warp, so that a batch of a few thousand envs still
// spreads over every SM.  Every lane runs the same trips, so the warp barrier between reading the
// forward state and overwriting it with the ColState is reached by all 32.
template <int NB, int NV, int NS, typename T>
__global__ void __launch_bounds__(32, 16) finish_prep_kernel(KArgs a) {
  __shared__ DevModel sm;
  load_model(sm, a.model);
  const int lo = a.flo ? *a.flo : 0;
  const int n = a.fhi ? *a.fhi - lo : a.n_env;
  const int nch = a.nchunk;
  const long long total = (long long)n * nch;
  const int lane = threadIdx.x & 31;
  for (long long base = (long long)blockIdx.x * 32; base < total; base += (long long)gridDim.x * 32) {
    const long long t = base + lane;
    int e = 0, chunk = 0;
    bool mine = t < total;
    if (mine) {
      const int ti = int(t / nch);
      chunk = int(t - (long long)ti * nch);
      e = DS_IX(a.fhi ? a.ws.dlist[lo + ti] : (a.env_list ? a.env_list[ti] : ti), a.B);
      mine = !a.model_id || a.model_id[e] == a.model_index;
    }
    Env<NB, NV, NS, T> s;
    if (mine) prep_load<NB, NV, NS, T>(sm, a, e, s);
    __syncwarp();
    if (mine) prep_store<NB, NV, NS, T>(sm, a, e, s, chunk, nch);
  }
}

// Warps per env of the column kernel: two when an env has more than 32 columns (Jacobians) or dof
// passes (VJP) to spread, so that more warps are in flight for the same shared memory.
template <int NV>
struct ColsShape {
  static constexpr int WPE = 3 * NV > 32 ? 2 : 1;
};

// Column kernel: ColsShape::WPE warps per env (blockDim = 32 WPE x envs per block, dynamic shared
// memory = one ColState per env); the CTAs stride over the range's envs, a CTA's envs in step, with
// a CTA barrier between staging the states and reading them (every thread runs the same trips).
template <int NB, int NV, int NS, typename T>
__global__ void __launch_bounds__(256, 2) finish_cols_kernel(KArgs a) {
  using CS = ColState<NB, NV, NS, T>;
  constexpr int WPE = ColsShape<NV>::WPE;
  constexpr int GL = 32 * WPE;                         // lanes per env
  __shared__ DevModel sm;
  extern __shared__ __align__(16) unsigned char ds_cs_smem[];
  load_model(sm, a.model);
  const int slot = int(threadIdx.x) / GL;
  const int li = int(threadIdx.x) - slot * GL;
  const int epb = int(blockDim.x) / GL;
  CS& cs = reinterpret_cast<CS*>(ds_cs_smem)[slot];
  const int lo = a.flo ? *a.flo : 0;
  const int n = a.fhi ? *a.fhi - lo : a.n_env;
  const int B = a.B;
  for (int base = int(blockIdx.x) * epb; base < n; base += int(gridDim.x) * epb) {
    const int t = base + slot;
    int e = 0;
    bool mine = t < n;
    uint32_t st = 0;
    if (mine) {
      e = DS_IX(a.fhi ? a.ws.dlist[lo + t] : (a.env_list ? a.env_list[t] : t), B);
      mine = !a.model_id || a.model_id[e] == a.model_index;
    }
    if (mine) st = a.ws.st[e];
    const bool cols = mine && !(st & DS_ENV_NONFINITE);
    if (cols) {
      int row = 0;
      const double* fw = a.ws.fw;
      cs.visit([&](auto* ptr, int cnt) {
        using V = typename std::remove_reference<decltype(*ptr)>::type;
        for (int i = li; i < cnt; i += GL) ptr[i] = V(fw[size_t(row + i) * B + e]);
        row += cnt;
      });
    }
    __syncthreads();
    if (cols) {
      if (a.run == DS_RUN_JAC) {
        for (int col = li; col < 3 * NV; col += GL) {
          const int blk = col / NV, d = col % NV;
          T Dc[NV];
          split_jac_column<NB, NV, NS, T>(sm, a, cs, blk, d, Dc);
          double* out = blk == 0 ? a.dv_dq : (blk == 1 ? a.dv_dv : a.dv_dtau);
          for (int k = 0; k < NV; ++k) out[(k * NV + d) * B + e] = double(Dc[k]);
        }
      } else {
        for (int p = li; p < 2 * NV; p += GL) {
          const int blk = p / NV, d = p % NV;
          double* out = blk == 0 ? a.q_bar : a.v_bar;
          out[d * B + e] = split_vjp_entry<NB, NV, NS, T>(sm, a, cs, blk, d);
        }
        for (int k = li; k < NV; k += GL) a.tau_bar[k * B + e] = double(T(a.dt) * cs.w2[k]);
      }
    }
    if (mine && li == 0 && a.status) a.status[e] = st;
    __syncthreads();
  }
}

// 2c. adaptive penalty (options admm_rho_adapt), after round a.round's Newton stage: for every env
//     queued for the next round, residual balancing of rho on its stored ADMM state
//     (admm_residuals, rho_balance) and, when rho changes, K = (G + rho I)^-1 formed again from the
//     stored G (the old rho and K are kept if the factorisation fails).  One thread per env.
template <int NS, typename T>
__global__ void __launch_bounds__(128) rho_adapt_kernel(KArgs a) {
  constexpr int NC3 = 3 * NS;
  const WsView& w = a.ws;
  const int n = w.counts[a.round + 1];
  const int32_t* lst = w.list[(a.round + 1) & 1];
  const int B = a.B;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
    const int e = DS_IX(lst[t], B);
    const int na = w.na[e];
    const int m = 3 * na;
    double x[NC3], z[NC3], y[NC3], sx[NC3], mu[NS];
    for (int i = 0; i < m; ++i) {
      x[i] = w.ax[i * B + e];
      z[i] = w.az[i * B + e];
      y[i] = w.ay[i * B + e];
      sx[i] = w.asx[i * B + e];
    }
    for (int i = 0; i < na; ++i) mu[i] = w.mu[i * B + e];
    double rp, rd;
    admm_residuals(na, mu, x, z, y, sx, rp, rd);
    const double rho = w.rho[e];
    const T nr = T(rho_balance(rho, rp, rd));
    if (double(nr) == rho) continue;
    T Lg[NC3 * (NC3 + 1) / 2];
    for (int i = 0; i < m; ++i)
      for (int j = 0; j <= i; ++j) Lg[tri(i, j)] = T(w.G[tri(i, j) * B + e]) + (i == j ? nr : T(0));
    if (!chol_packed(Lg, m)) continue;
    for (int j = 0; j < m; ++j) {
      T col[NC3];
      for (int i = 0; i < m; ++i) col[i] = T(i == j ? 1 : 0);
      fwd_packed(Lg, col, m);
      bwd_packed(Lg, col, m);
      for (int i = 0; i < m; ++i) w.K[(i * NC3 + j) * B + e] = double(col[i]);
    }
    w.rho[e] = double(nr);
  }
}

template <int NB, int NV, int NS, typename T>
__global__ void __launch_bounds__(128, 4) finish_tape_kernel(KArgs a) {
  __shared__ DevModel sm;
  load_model(sm, a.model);
  const long long total = (long long)a.n_env * a.nchunk;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int chunk = int(t / a.n_env), e = int(t - (long long)chunk * a.n_env);
    if (a.model_id && a.model_id[e] != a.model_index) continue;
    finish_tape_env<NB, NV, NS, T>(sm, a, e, chunk, a.nchunk);
  }
}

// Copies the completed-env count to its snapshot slot (the split point of an overlapped finish).
static __global__ void dcount_snapshot_kernel(int32_t* dcount) { dcount[1] = dcount[0]; }

template <int NB, int NV, int NS, typename T>
__global__ void __launch_bounds__(128, 4) finish_kernel(KArgs a) {
  // The overlapped finish can keep off some SMs, so that the few slow envs of the late ADMM rounds
  // (launched meanwhile on the other stream) find whole SMs free and do not share an SM
  // sub-partition's FP64 pipe with the finish's warps.  The test is uniform over the CTA.
  if (a.fin_reserve > 0) {
    unsigned smid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    if (smid % unsigned(a.fin_reserve) == 0) return;
  }
  __shared__ DevModel sm;
  load_model(sm, a.model);
  // work item t handles env t % n, column chunk t / n (consecutive threads: consecutive envs); the
  // envs are the launch's, or the range [*flo, *fhi) of the completed-env list
  const int lo = a.flo ? *a.flo : 0;
  const int n = a.fhi ? *a.fhi - lo : a.n_env;
  if (n <= 0) return;
  const long long total = (long long)n * a.nchunk;
  auto item = [&](long long t) {
    const int chunk = int(t / n), ti = int(t - (long long)chunk * n);
    const int e = DS_IX(a.fhi ? a.ws.dlist[lo + ti] : (a.env_list ? a.env_list[ti] : ti), a.B);
    if (a.model_id && a.model_id[e] != a.model_index) return;
    finish_env<NB, NV, NS, T>(sm, a, e, chunk, a.nchunk);
  };
  if (a.claim) {
    // dynamic split (CTAs that returned above leave their share to the others): a warp claims 32
    // consecutive items at a time
    const int lane = threadIdx.x & 31;
    for (;;) {
      int base = 0;
      if (lane == 0) base = atomicAdd(a.claim, 32);
      base = __shfl_sync(0xffffffffu, base, 0);
      if ((long long)base >= total) break;
      if ((long long)base + lane < total) item((long long)base + lane);
    }
    return;
  }
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x)
    item(t);
}

}  // namespace ds
