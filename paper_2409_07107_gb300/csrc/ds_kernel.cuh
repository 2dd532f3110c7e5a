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
__device__ __forceinline__ void proj_cone(const T* x, T mu, T* o) {
  const T nt = sqrt(x[0] * x[0] + x[1] * x[1]);
  if (nt <= mu * x[2]) { o[0] = x[0]; o[1] = x[1]; o[2] = x[2]; return; }
  if (mu * nt <= -x[2]) { o[0] = T(0); o[1] = T(0); o[2] = T(0); return; }
  const T s = (mu * nt + x[2]) / (T(1) + mu * mu);
  const T k = mu * s / nt;
  o[0] = k * x[0]; o[1] = k * x[1]; o[2] = s;
}

template <int NB, int NV, int NS, typename T>
struct Env {
  static constexpr int NC3 = 3 * NS;
  static constexpr bool kDouble = std::is_same<T, double>::value;
  double R[NB][9], P[NB][3];                 // world placement of every body (FP64)
  T S[NV][6];                                // world motion subspace of every dof
  T I[NB][10];                               // world spatial inertia of every body
  T V[NB][6], A[NB][6], VJ[NB][6], IV[NB][6], IA[NB][6], Fc[NB][6];
  T L[NV * (NV + 1) / 2];                    // Cholesky factor of M (packed lower)
  T v[NV], tau[NV], vdf[NV], vf[NV], vn[NV], astar[NV];
  int na;                                    // active contacts
  int slot[NS], body[NS];
  T x[NS][3], c[NS][3], f[NS][3];            // body point, contact point, contact force (world)
  T fr[3][3];                                // contact frame rows t1, t2, n
  double mu[NS];
  T Jc[NC3][NV];
  T Y[NC3][NV];                              // rows of M^-1 J_c^T
  T Gt[NC3][NC3];                            // Delassus matrix in the bulk type
  double Gd_[kDouble ? 1 : NC3][kDouble ? 1 : NC3];
  T gt[NC3];
  double gd[NC3], lam[NC3];
  int mode[NS];
  double margin;
  LUcp<NC3 + NS, NC3> lu;

  __device__ __forceinline__ double G(int i, int j) const {
    if constexpr (kDouble) return Gt[i][j]; else return Gd_[i][j];
  }
};

// ------------------------------------------------------------------------- NCP helpers (FP64)

template <class E>
__device__ double ncp_residual(const E& s, const double* lam) {
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

// Contact modes (breaking / sticking / sliding) from sigma = G lambda + g, lambda.
template <class E>
__device__ double classify(const E& s, const double* lam, double es_rel, double el_rel, int* mode) {
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
    const double ns = sqrt(sg[0] * sg[0] + sg[1] * sg[1] + sg[2] * sg[2]);
    const double nst = sqrt(sg[0] * sg[0] + sg[1] * sg[1]);
    if (ns <= es) {
      mode[i] = DS_MODE_STICKING;
      margin = fmin(margin, (es - ns) / es);
    } else if (sg[2] > es || lam[3 * i + 2] <= el) {
      mode[i] = DS_MODE_BREAKING;
      margin = fmin(margin, sg[2] > es ? (sg[2] - es) / gmax : 0.0);
    } else {
      mode[i] = DS_MODE_SLIDING;
      margin = fmin(margin, fmin(nst / gmax, lam[3 * i + 2] / lmax));
    }
  }
  return margin;
}

// Active-set update after a Newton solve that did not give an NCP solution (same rules as the
// oracle): breaking + penetrating -> sticking; sticking/sliding + pulling -> breaking; sticking
// with the impulse outside the cone -> sliding; sliding that stopped -> sticking.
template <class E>
__device__ bool reclassify(const E& s, const double* lam, int* mode, double es, double el, double delta) {
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
// FP64, basic-solution steps of a rank-revealing LU.
template <class E>
__device__ void newton_modes(E& s, double* lam, const int* mode, int iters, double sat_delta) {
  const int m = 3 * s.na;
  double scale = 1.0;
  for (int j = 0; j < m; ++j) scale = fmax(scale, fabs(s.gd[j]));
  int sat[E::NC3 / 3], nsat = 0;
  for (int i = 0; i < s.na; ++i) {
    const double* l = lam + 3 * i;
    const double nt = sqrt(l[0] * l[0] + l[1] * l[1]);
    if (mode[i] == DS_MODE_STICKING && nt > 0.0 && s.mu[i] * l[2] - nt <= sat_delta) sat[nsat++] = i;
  }
  const int rows = m + nsat;
  for (int it = 0; it < iters; ++it) {
    double sg[E::NC3], F[E::NC3 + E::NC3 / 3];
    for (int r = 0; r < m; ++r) {
      double t = s.gd[r];
      for (int j = 0; j < m; ++j) t += s.G(r, j) * lam[j];
      sg[r] = t;
    }
    s.lu.r = rows;
    s.lu.c = m;
    for (int r = 0; r < rows; ++r)
      for (int j = 0; j < m; ++j) s.lu.a[r][j] = 0.0;
    for (int i = 0; i < s.na; ++i) {
      const int r0 = 3 * i;
      if (mode[i] == DS_MODE_BREAKING) {
        for (int r = 0; r < 3; ++r) { F[r0 + r] = lam[r0 + r]; s.lu.a[r0 + r][r0 + r] = 1.0; }
      } else if (mode[i] == DS_MODE_STICKING) {
        for (int r = 0; r < 3; ++r) {
          F[r0 + r] = sg[r0 + r];
          for (int j = 0; j < m; ++j) s.lu.a[r0 + r][j] = s.G(r0 + r, j);
        }
      } else {
        const double ns = sqrt(sg[r0] * sg[r0] + sg[r0 + 1] * sg[r0 + 1]);
        const double u[2] = {sg[r0] / ns, sg[r0 + 1] / ns};
        const double mu = s.mu[i], ln = lam[r0 + 2];
        const double k = mu * ln / ns;
        for (int r = 0; r < 2; ++r) {
          F[r0 + r] = lam[r0 + r] + mu * ln * u[r];
          // k (I - u u^T) G_T, then [I2, mu u] on the contact's own columns
          for (int j = 0; j < m; ++j)
            s.lu.a[r0 + r][j] = k * (((r == 0) - u[r] * u[0]) * s.G(r0, j) + ((r == 1) - u[r] * u[1]) * s.G(r0 + 1, j));
          s.lu.a[r0 + r][r0 + r] += 1.0;
          s.lu.a[r0 + r][r0 + 2] += mu * u[r];
        }
        F[r0 + 2] = sg[r0 + 2];
        for (int j = 0; j < m; ++j) s.lu.a[r0 + 2][j] = s.G(r0 + 2, j);
      }
    }
    for (int q = 0; q < nsat; ++q) {
      const int i = sat[q], r0 = 3 * i;
      const double nt = sqrt(lam[r0] * lam[r0] + lam[r0 + 1] * lam[r0 + 1]);
      F[m + q] = s.mu[i] * lam[r0 + 2] - nt;
      s.lu.a[m + q][r0] = -lam[r0] / nt;
      s.lu.a[m + q][r0 + 1] = -lam[r0 + 1] / nt;
      s.lu.a[m + q][r0 + 2] = s.mu[i];
    }
    double fmaxv = 0.0;
    for (int r = 0; r < rows; ++r) fmaxv = fmax(fmaxv, fabs(F[r]));
    if (!(fmaxv > 1e-15 * scale)) break;
    s.lu.factor(1e-13);
    double dx[E::NC3];
    s.lu.solve(F, dx);
    for (int r = 0; r < m; ++r) lam[r] -= dx[r];
  }
}

// Staged NCP solve (same structure as the oracle's): each stage continues the over-relaxed ADMM
// (bulk type, rho = 0.3 mean diag G, De Saxce term at the latest primal iterate) to a tolerance,
// identifies the modes, and runs up to 4 active-set rounds of FP64 Newton on the mode equations;
// the first candidate whose FP64 NCP residual passes is accepted.
template <class E, typename T>
__device__ void solve_ncp(E& s, const KArgs& a, int& iters, uint32_t& st) {
  const int m = 3 * s.na;
  iters = 0;
  if (m == 0) return;
  T trace = T(0);
  for (int i = 0; i < m; ++i) trace += s.Gt[i][i];
  T rho = T(0.3) * trace / T(m);
  if (!(rho > T(1e-12))) rho = T(1e-12);
  const T relax = T(1.6);
  T Lg[E::NC3 * (E::NC3 + 1) / 2];
  for (int i = 0; i < m; ++i)
    for (int j = 0; j <= i; ++j) Lg[tri(i, j)] = s.Gt[i][j] + (i == j ? rho : T(0));
  if (!chol_packed(Lg, m)) { st |= DS_ENV_NONFINITE; }
  T x[E::NC3], z[E::NC3], y[E::NC3];
  for (int i = 0; i < m; ++i) { x[i] = T(0); z[i] = T(0); y[i] = T(0); }
  T gs = T(1);
  double scale = 1.0;
  for (int i = 0; i < m; ++i) { gs = fmax(gs, fabs(s.gt[i])); scale = fmax(scale, fabs(s.gd[i])); }
  double best[E::NC3], best_r = 1e300;
  double eps = a.admm_eps;
  const double shrink = E::kDouble ? 1e-2 : 0.1;
  const double floor_eps = E::kDouble ? 1e-13 : 1e-6;
  const int nstage = E::kDouble ? 4 : 3;
  const double tol = a.ncp_tol * scale;
  for (int stage = 0; stage < nstage; ++stage) {
    const T te = T(eps);
    while (iters < a.admm_max_iter) {
      ++iters;
      T rhs[E::NC3];
      for (int i = 0; i < s.na; ++i) {
        T sg[3];
        for (int k = 0; k < 3; ++k) {
          T t = s.gt[3 * i + k];
          for (int j = 0; j < m; ++j) t += s.Gt[3 * i + k][j] * x[j];
          sg[k] = t;
        }
        const T sd = T(s.mu[i]) * sqrt(sg[0] * sg[0] + sg[1] * sg[1]);
        for (int k = 0; k < 3; ++k)
          rhs[3 * i + k] = rho * z[3 * i + k] - y[3 * i + k] - s.gt[3 * i + k] - (k == 2 ? sd : T(0));
      }
      fwd_packed(Lg, rhs, m);
      bwd_packed(Lg, rhs, m);
      T rp = T(0), rd = T(0), zmax = T(1);
      for (int i = 0; i < s.na; ++i) {
        T w[3], p[3], xh[3];
        for (int k = 0; k < 3; ++k) {
          const int r = 3 * i + k;
          x[r] = rhs[r];
          xh[k] = relax * x[r] + (T(1) - relax) * z[r];
          w[k] = xh[k] + y[r] / rho;
        }
        proj_cone(w, T(s.mu[i]), p);
        for (int k = 0; k < 3; ++k) {
          const int r = 3 * i + k;
          rd = fmax(rd, fabs(p[k] - z[r]));
          z[r] = p[k];
          y[r] += rho * (xh[k] - z[r]);
          rp = fmax(rp, fabs(x[r] - z[r]));
          zmax = fmax(zmax, fabs(z[r]));
        }
      }
      rd *= rho;
      if (rp <= te * zmax && rd <= te * gs) break;
    }
    double lz[E::NC3], lp[E::NC3];
    double lscale = 1.0;
    for (int i = 0; i < m; ++i) { lz[i] = double(z[i]); lscale = fmax(lscale, fabs(lz[i])); }
    const double es = fmax(a.eps_sigma, 10.0 * eps), el = fmax(a.eps_lambda, 10.0 * eps);
    const double sat_delta = 10.0 * eps * lscale;
    int mode[E::NC3 / 3];
    classify(s, lz, es, el, mode);
    {
      const double r0 = ncp_residual(s, lz);
      if (r0 < best_r) { best_r = r0; for (int i = 0; i < m; ++i) best[i] = lz[i]; }
    }
    for (int i = 0; i < m; ++i) lp[i] = lz[i];
    for (int round = 0; round < 4 && best_r > tol; ++round) {
      newton_modes(s, lp, mode, a.polish_iters, sat_delta);
      const double rpol = ncp_residual(s, lp);
      if (rpol < best_r) { best_r = rpol; for (int i = 0; i < m; ++i) best[i] = lp[i]; }
      if (best_r <= tol) break;
      if (!reclassify(s, lp, mode, es * scale, el * lscale, sat_delta)) break;
      for (int i = 0; i < s.na; ++i) proj_cone(lp + 3 * i, s.mu[i], lp + 3 * i);
    }
    if (best_r <= tol || iters >= a.admm_max_iter) break;
    eps = fmax(eps * shrink, floor_eps);
  }
  for (int i = 0; i < m; ++i) s.lam[i] = best[i];
  if (!(best_r <= tol)) st |= DS_ENV_NOT_CONVERGED;
}

}  // namespace ds

namespace ds {

// Directional derivative of the contact-augmented inverse dynamics tau = RNEA(q, v, a*) - J_c^T f
// along one dof: kind 0 = tangent of q (the subtree of the dof's body moves by the rigid twist
// xi = S_d), kind 1 = unit change of the dof's velocity.  Uses the stored pass values V, A, VJ,
// IV, IA, Fc of the a* pass.  Writes dtau[NV].
template <int NB, int NV, int NS, typename T>
__device__ void rnea_tangent(const DevModel& m, const Env<NB, NV, NS, T>& s, int kind, int d, T* dtau) {
  const int j = m.dof_body[d];
  const int jend = m.sub_end[j];
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
        mcross(xi, s.S[dd], dS);
        for (int k = 0; k < 6; ++k) { dVJ[k] += dS[k] * s.v[dd]; dSa[k] += dS[k] * s.astar[dd]; }
      }
    } else if (i == j) {
      for (int k = 0; k < 6; ++k) dVJ[k] = xi[k];
    }
    T t1[6], t2[6];
    for (int k = 0; k < 6; ++k) dV[i][k] = (inside ? dV[par][k] : T(0)) + dVJ[k];
    mcross(dV[i], s.VJ[i], t1);
    mcross(s.V[i], dVJ, t2);
    for (int k = 0; k < 6; ++k) dA[i][k] = (inside ? dA[par][k] : T(0)) + dSa[k] + t1[k] + t2[k];
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
      T r = dot6(s.S[dd], dF[i]);
      if (kind == 0) {
        T dS[6];
        mcross(xi, s.S[dd], dS);
        r += dot6(dS, s.Fc[i]);
      }
      dtau[dd] = r;
    }
    if (i != j) {
      const int par = m.parent[i];
      for (int k = 0; k < 6; ++k) dF[par][k] += dF[i][k];
    }
  }
  for (int b = m.parent[j]; b >= 0; b = m.parent[b])
    for (int dd = m.iv[b]; dd < m.iv[b] + m.nd[b]; ++dd) dtau[dd] = dot6(s.S[dd], dF[j]);
}

// d(J_c v+)/dq_d for contact a at fixed v+ (App. D's FKV term, including the motion of the
// contact point with the body): Vp = body velocities under v+.
template <int NB, int NV, int NS, typename T>
__device__ __forceinline__ void fkv_tangent(const DevModel& m, const Env<NB, NV, NS, T>& s, const T (*Vp)[6],
                                            int a, int d, T* out) {
  const int j = m.dof_body[d];
  const int b = s.body[a];
  out[0] = out[1] = out[2] = T(0);
  if (b < j || b >= m.sub_end[j]) return;
  const T* xi = s.S[d];
  const int pj = m.parent[j];
  T rel[6], dVb[6], t[3], dc[3], dp[3];
  for (int k = 0; k < 6; ++k) rel[k] = Vp[b][k] - (pj >= 0 ? Vp[pj][k] : T(0));
  mcross(xi, rel, dVb);
  cross3(xi + 3, s.x[a], t);
  for (int k = 0; k < 3; ++k) dc[k] = xi[k] + t[k];
  cross3(dVb + 3, s.c[a], t);
  for (int k = 0; k < 3; ++k) dp[k] = dVb[k] + t[k];
  cross3(Vp[b] + 3, dc, t);
  for (int k = 0; k < 3; ++k) dp[k] += t[k];
  for (int r = 0; r < 3; ++r) out[r] = dot3(s.fr[r], dp);
}

template <int NB, int NV, int NS, typename T>
__device__ void run_env(const DevModel& m, const KArgs& a, const int e) {
  Env<NB, NV, NS, T> s;
  const int B = a.B;
  uint32_t st = 0;
  double q[NV + 1];
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
          R0[3 * r + c] = s.R[par][3 * r] * m.jrot[i][c] + s.R[par][3 * r + 1] * m.jrot[i][3 + c] + s.R[par][3 * r + 2] * m.jrot[i][6 + c];
        p0[r] = s.P[par][r] + s.R[par][3 * r] * m.jpos[i][0] + s.R[par][3 * r + 1] * m.jpos[i][1] + s.R[par][3 * r + 2] * m.jpos[i][2];
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
        for (int k = 0; k < 6; ++k) VJ[k] += s.S[dd][k] * s.v[dd];
      T t[6];
      for (int k = 0; k < 6; ++k) s.V[i][k] = (par >= 0 ? s.V[par][k] : T(0)) + VJ[k];
      mcross(s.V[i], VJ, t);
      for (int k = 0; k < 6; ++k)
        s.A[i][k] = (par >= 0 ? s.A[par][k] : (k < 3 ? -grav[k] : T(0))) + t[k];
      iapply(s.I[i], s.V[i], s.IV[i]);
      iapply(s.I[i], s.A[i], s.IA[i]);
      fcross(s.V[i], s.IV[i], t);
      for (int k = 0; k < 6; ++k) s.Fc[i][k] = s.IA[i][k] + t[k];
    }
    for (int i = NB - 1; i >= 0; --i) {
      for (int dd = m.iv[i]; dd < m.iv[i] + m.nd[i]; ++dd) bias[dd] = dot6(s.S[dd], s.Fc[i]);
      const int par = m.parent[i];
      if (par >= 0)
        for (int k = 0; k < 6; ++k) s.Fc[par][k] += s.Fc[i][k];
    }
  }

  // ---- F3 joint-space inertia by composite inertias (world frame: plain sums) + Cholesky
  {
    T IC[NB][10];
    for (int i = 0; i < NB; ++i)
      for (int k = 0; k < 10; ++k) IC[i][k] = s.I[i][k];
    for (int i = NB - 1; i > 0; --i) {
      const int par = m.parent[i];
      if (par >= 0)
        for (int k = 0; k < 10; ++k) IC[par][k] += IC[i][k];
    }
    for (int k = 0; k < NV * (NV + 1) / 2; ++k) s.L[k] = T(0);
    for (int i = 0; i < NB; ++i) {
      for (int dd = m.iv[i]; dd < m.iv[i] + m.nd[i]; ++dd) {
        T F[6];
        iapply(IC[i], s.S[dd], F);
        for (int d2 = m.iv[i]; d2 <= dd; ++d2) s.L[tri(dd, d2)] = dot6(s.S[d2], F);
        for (int b = m.parent[i]; b >= 0; b = m.parent[b])
          for (int d2 = m.iv[b]; d2 < m.iv[b] + m.nd[b]; ++d2) s.L[tri(dd, d2)] = dot6(s.S[d2], F);
      }
    }
    if (!chol_packed(s.L, NV)) st |= DS_ENV_NONFINITE;
    for (int k = 0; k < NV; ++k) s.vdf[k] = s.tau[k] - bias[k];
    fwd_packed(s.L, s.vdf, NV);
    bwd_packed(s.L, s.vdf, NV);
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
    for (int i = 0; i < 3; ++i) xw[i] = s.P[b][i] + s.R[b][3 * i] * pl[0] + s.R[b][3 * i + 1] * pl[1] + s.R[b][3 * i + 2] * pl[2];
    const double phi = pn[0] * xw[0] + pn[1] * xw[1] + pn[2] * xw[2] - pd - r;
    if (phi <= 0.0) {
      const int n = s.na++;
      s.slot[n] = k;
      s.body[n] = b;
      s.mu[n] = a.c_mu[k * B + e];
      for (int i = 0; i < 3; ++i) { s.x[n][i] = T(xw[i]); s.c[n][i] = T(xw[i] - r * pn[i]); }
    }
  }
  const int mdim = 3 * s.na;

  // ---- F5 contact Jacobian rows (t1, t2, n) . velocity of the body point at c
  for (int r = 0; r < mdim; ++r)
    for (int k = 0; k < NV; ++k) s.Jc[r][k] = T(0);
  for (int ac = 0; ac < s.na; ++ac) {
    for (int b = s.body[ac]; b >= 0; b = m.parent[b])
      for (int dd = m.iv[b]; dd < m.iv[b] + m.nd[b]; ++dd) {
        T pv[3], t[3];
        cross3(s.S[dd] + 3, s.c[ac], t);
        for (int k = 0; k < 3; ++k) pv[k] = s.S[dd][k] + t[k];
        for (int r = 0; r < 3; ++r) s.Jc[3 * ac + r][dd] = dot3(s.fr[r], pv);
      }
  }

  // ---- F6 Delassus matrix G = (L^-1 J^T)^T (L^-1 J^T), Y = M^-1 J^T, g = J v_f
  for (int r = 0; r < mdim; ++r) {
    for (int k = 0; k < NV; ++k) s.Y[r][k] = s.Jc[r][k];
    fwd_packed(s.L, s.Y[r], NV);
  }
  for (int r = 0; r < mdim; ++r)
    for (int c = 0; c <= r; ++c) {
      T t = T(0);
      for (int k = 0; k < NV; ++k) t += s.Y[r][k] * s.Y[c][k];
      s.Gt[r][c] = t;
      s.Gt[c][r] = t;
    }
  for (int r = 0; r < mdim; ++r) {
    bwd_packed(s.L, s.Y[r], NV);
    T t = T(0);
    for (int k = 0; k < NV; ++k) t += s.Jc[r][k] * s.vf[k];
    s.gt[r] = t;
    s.gd[r] = double(t);
  }
  if constexpr (!Env<NB, NV, NS, T>::kDouble)
    for (int r = 0; r < mdim; ++r)
      for (int c = 0; c < mdim; ++c) s.Gd_[r][c] = double(s.Gt[r][c]);

  // ---- F7/F8 NCP solve and residual check
  int iters = 0;
  for (int r = 0; r < mdim; ++r) s.lam[r] = 0.0;
  if (mdim > 0 && !(st & DS_ENV_NONFINITE)) solve_ncp<Env<NB, NV, NS, T>, T>(s, a, iters, st);
  s.margin = classify(s, s.lam, a.eps_sigma, a.eps_lambda, s.mode);
  if (mdim > 0 && s.margin < a.margin_delta) st |= DS_ENV_NEAR_SWITCH;

  // ---- F9 velocity update and symplectic-Euler position update
  for (int k = 0; k < NV; ++k) {
    T t = s.vf[k];
    for (int r = 0; r < mdim; ++r) t += s.Y[r][k] * T(s.lam[r]);
    s.vn[k] = t;
  }
  for (int k = 0; k < NV; ++k) {
    const double vv = double(s.vn[k]);
    if (!isfinite(vv)) st |= DS_ENV_NONFINITE;
    a.v_next[k * B + e] = vv;
  }
  if (a.q_next) {
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

  if (a.run != DS_RUN_STEP && !(st & DS_ENV_NONFINITE)) {
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
      for (int k = 0; k < 6; ++k) s.A[i][k] = (par >= 0 ? s.A[par][k] : (k < 3 ? -grav[k] : T(0))) + t[k];
      for (int dd = m.iv[i]; dd < m.iv[i] + m.nd[i]; ++dd)
        for (int k = 0; k < 6; ++k) s.A[i][k] += s.S[dd][k] * s.astar[dd];
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
        for (int k = 0; k < 6; ++k) s.Fc[par][k] += s.Fc[i][k];
    }
    // body velocities under v+ (for the FKV term)
    T Vp[NB][6];
    for (int i = 0; i < NB; ++i) {
      const int par = m.parent[i];
      for (int k = 0; k < 6; ++k) Vp[i][k] = (par >= 0 ? Vp[par][k] : T(0));
      for (int dd = m.iv[i]; dd < m.iv[i] + m.nd[i]; ++dd)
        for (int k = 0; k < 6; ++k) Vp[i][k] += s.S[dd][k] * s.vn[dd];
    }

    // ---- B3/B4 reduced implicit system A = B G C + blkdiag(0, Q) (App. B), FP64
    int off[NS], sz[NS];
    double Rm[NS][3][2], RP[NS][2][3];
    int md = 0;
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
      if (s.lu.rank < md) st |= DS_ENV_SINGULAR;
    }

    const T dt = T(a.dt);
    if (a.run == DS_RUN_JAC) {
      // ---- B1/B2/B5/B6 one Jacobian column at a time:
      // D = dv+/dtheta at fixed lambda, RHS = J_c D + F, X = -A^- B RHS, dv = D + Y C X
      for (int col = 0; col < 3 * NV; ++col) {
        const int blk = col / NV, d = col % NV;
        T Dc[NV];
        if (blk < 2) {
          T dtau[NV];
          rnea_tangent<NB, NV, NS, T>(m, s, blk, d, dtau);
          fwd_packed(s.L, dtau, NV);
          bwd_packed(s.L, dtau, NV);
          for (int k = 0; k < NV; ++k) Dc[k] = -dt * dtau[k] + (blk == 1 && k == d ? T(1) : T(0));
        } else {
          for (int k = 0; k < NV; ++k) Dc[k] = (k == d ? dt : T(0));
          fwd_packed(s.L, Dc, NV);
          bwd_packed(s.L, Dc, NV);
        }
        if (md > 0) {
          double rhs[3 * NS], X[3 * NS];
          for (int ac = 0; ac < s.na; ++ac) {
            if (sz[ac] == 0) continue;
            double r3[3];
            T fk[3] = {T(0), T(0), T(0)};
            if (blk == 0) fkv_tangent<NB, NV, NS, T>(m, s, Vp, ac, d, fk);
            for (int r = 0; r < 3; ++r) {
              T t = fk[r];
              for (int k = 0; k < NV; ++k) t += s.Jc[3 * ac + r][k] * Dc[k];
              r3[r] = double(t);
            }
            if (sz[ac] == 3) {
              for (int r = 0; r < 3; ++r) rhs[off[ac] + r] = -r3[r];
            } else {
              for (int r = 0; r < 2; ++r)
                rhs[off[ac] + r] = -(RP[ac][r][0] * r3[0] + RP[ac][r][1] * r3[1] + RP[ac][r][2] * r3[2]);
            }
          }
          s.lu.solve(rhs, X);
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
      T vb[NV], ub[NV], w2[NV];
      for (int k = 0; k < NV; ++k) { vb[k] = T(a.vbar[k * B + e]); ub[k] = vb[k]; }
      double zeta[3 * NS];
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
        s.lu.solve_t(wv, z);
        for (int ac = 0; ac < s.na; ++ac) {
          if (sz[ac] == 0) continue;
          if (sz[ac] == 3) { for (int r = 0; r < 3; ++r) zeta[3 * ac + r] = z[off[ac] + r]; }
          else { for (int r = 0; r < 3; ++r) zeta[3 * ac + r] = RP[ac][0][r] * z[off[ac]] + RP[ac][1][r] * z[off[ac] + 1]; }
        }
        for (int r = 0; r < mdim; ++r) {
          const T zr = T(zeta[r]);
          for (int k = 0; k < NV; ++k) ub[k] -= s.Jc[r][k] * zr;
        }
      }
      for (int k = 0; k < NV; ++k) w2[k] = ub[k];
      fwd_packed(s.L, w2, NV);
      bwd_packed(s.L, w2, NV);
      for (int blk = 0; blk < 2; ++blk)
        for (int d = 0; d < NV; ++d) {
          T dtau[NV];
          rnea_tangent<NB, NV, NS, T>(m, s, blk, d, dtau);
          T r = T(0);
          for (int k = 0; k < NV; ++k) r += dtau[k] * w2[k];
          r = -dt * r;
          if (blk == 1) r += ub[d];
          if (blk == 0) {
            for (int ac = 0; ac < s.na; ++ac) {
              if (sz[ac] == 0) continue;
              T fk[3];
              fkv_tangent<NB, NV, NS, T>(m, s, Vp, ac, d, fk);
              for (int rr = 0; rr < 3; ++rr) r -= fk[rr] * T(zeta[3 * ac + rr]);
            }
          }
          double* out = blk == 0 ? a.q_bar : a.v_bar;
          out[d * B + e] = double(r);
        }
      for (int k = 0; k < NV; ++k) a.tau_bar[k * B + e] = double(dt * w2[k]);
    }
  }
  if (a.status) a.status[e] = st;
}

template <int NB, int NV, int NS, typename T>
__global__ void __launch_bounds__(128) env_kernel(KArgs a) {
  __shared__ DevModel sm;
  {
    const int* src = reinterpret_cast<const int*>(a.model);
    int* dst = reinterpret_cast<int*>(&sm);
    for (int k = threadIdx.x; k < int(sizeof(DevModel) / sizeof(int)); k += blockDim.x) dst[k] = src[k];
  }
  __syncthreads();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= a.n_env) return;
  const int e = a.env_list ? a.env_list[t] : t;
  if (a.model_id && a.model_id[e] != a.model_index) return;
  run_env<NB, NV, NS, T>(sm, a, e);
}

template <int NB, int NV, int NS, typename T>
void launch_env(const KArgs& a, cudaStream_t s) {
  const int threads = 128;
  const int blocks = (a.n_env + threads - 1) / threads;
  if (blocks > 0) env_kernel<NB, NV, NS, T><<<blocks, threads, 0, s>>>(a);
}

}  // namespace ds
