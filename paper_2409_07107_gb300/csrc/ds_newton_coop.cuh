// Cooperative form of the Newton / active-set stage of the NCP solve (pipeline step 2b).
//
// One lane per equation row: L = 4 NS lanes per env (three rows per contact slot, then one
// saturation row per slot), 32 / L envs per warp.  The Delassus matrix of the env sits in shared
// memory; each lane builds its own row of the Newton matrix of the mode equations in registers and
// the rank-revealing LU with complete pivoting runs across the lanes (pivot = group arg-max, pivot
// row broadcast by shuffles, the right-hand side eliminated along).  The step is the same as the
// one-thread form's: the basic solution when the reduced system has full column rank, otherwise
// the minimum-norm solution of the pivot rows, x = U^T (U U^T)^-1 y with U the pivot rows of the
// eliminated matrix and y their eliminated right-hand side (the same solution set, so the same
// minimum-norm point).  Classification, residual and re-classification follow the one-thread
// rules line for line, with one lane per contact doing the per-contact arithmetic.
//
// Control flow is warp-uniform: loops run to bounds that every lane of the warp shares (or to an
// __any_sync of the per-env conditions), and per-env conditions only predicate work, so every
// shuffle and __syncwarp is reached by all 32 lanes.
#pragma once
#include "ds_kernel.cuh"

namespace ds {
namespace coop {

constexpr unsigned kFull = 0xffffffffu;

template <int NS>
struct Shape {
  static constexpr int NC3 = 3 * NS;
  static constexpr int L = 4 * NS;            // lanes per env
  static constexpr int EPW = 32 / L;          // envs per warp
  static constexpr int PS = NC3 | 1;          // odd row stride: rows of doubles hit distinct banks
  static constexpr int THREADS = NS >= 8 ? 64 : 128;
  static constexpr int MINB = NS >= 8 ? 1 : 5;  // blocks per SM the register budget is sized for
  static constexpr unsigned LMASK = L == 32 ? 0xffffffffu : ((1u << L) - 1u);
};

// Work space of the minimum-norm step in the LU's type LT: the pivot rows U (in pivot order),
// U U^T with its Cholesky factor, and a vector.
template <int NS, typename LT>
struct LUWork {
  LT U[Shape<NS>::NC3][Shape<NS>::PS];
  LT H[Shape<NS>::NC3][Shape<NS>::PS];
  LT w[Shape<NS>::NC3];
  LT rd[Shape<NS>::NC3];                     // reciprocals of the Cholesky diagonal
};

// Per-env shared memory: the Delassus matrix (FP64) and the step work spaces: FP64 always, FP32 as
// well in the mixed form (whose Newton steps factor in FP32 except in the last stage).
template <int NS, typename T>
struct Smem {
  double G[Shape<NS>::NC3][Shape<NS>::PS];
  LUWork<NS, double> d;
  typename std::conditional<std::is_same<T, float>::value, LUWork<NS, float>, char>::type f;
};

// Integer views of |x| for pivot comparisons (same order as the values for non-negative x).
template <typename LT>
struct LUBits;
template <>
struct LUBits<double> {
  using I = long long;
  static __device__ __forceinline__ I bits(double x) { return __double_as_longlong(fabs(x)); }
  static __device__ __forceinline__ double value(I b) { return __longlong_as_double(b); }
  static constexpr I kInf = 0x7FF0000000000000LL;
  static constexpr double kRankTol = 1e-13;
};
template <>
struct LUBits<float> {
  using I = int;
  static __device__ __forceinline__ I bits(float x) { return __float_as_int(fabsf(x)); }
  static __device__ __forceinline__ float value(I b) { return __int_as_float(b); }
  static constexpr I kInf = 0x7F800000;
  static constexpr float kRankTol = 1e-5f;
};

// What a lane is: its row li within the env's group, the contact ci it belongs to (row lanes:
// li / 3; saturation lanes: li - NC3) and the env-level data it needs.
template <int NS>
struct Lane {
  int li, base;        // row within the group; first lane of the group in the warp
  int ci, kc;          // contact and component (kc = 0, 1, 2 for row lanes)
  bool row;            // equation-row lane (li < NC3), else saturation lane
  int na;              // active contacts of the env (0 for an empty group)
  double mu, g;        // mu of contact ci; g[li] (row lanes of active contacts, else 0)
};

template <int L>
__device__ __forceinline__ double gmax(double v) {
#pragma unroll
  for (int o = L / 2; o >= 1; o >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

template <int L>
__device__ __forceinline__ double gmin(double v) {
#pragma unroll
  for (int o = L / 2; o >= 1; o >>= 1) v = fmin(v, __shfl_xor_sync(kFull, v, o));
  return v;
}

// The group's bits of a predicate (bit li = lane li of the env's group).
template <int NS>
__device__ __forceinline__ unsigned gbits(bool p, const Lane<NS>& ln) {
  return (__ballot_sync(kFull, p) >> ln.base) & Shape<NS>::LMASK;
}

template <int NS>
__device__ __forceinline__ bool gany(bool p, const Lane<NS>& ln) { return gbits<NS>(p, ln) != 0u; }

// sigma_li = g_li + sum_j G[li][j] lambda_j (row lanes; the sum runs over the padded width, where
// G and lambda are zero, in the same order as the one-thread form).
template <int NS, class SM>
__device__ __forceinline__ double sigma_row(const SM& S, const Lane<NS>& ln, double lam) {
  constexpr int NC3 = Shape<NS>::NC3;
  const int r = ln.row ? ln.li : 0;
  double t = ln.g;
#pragma unroll
  for (int j = 0; j < NC3; ++j) {
    const double lj = __shfl_sync(kFull, lam, ln.base + j);
    t += S.G[r][j] * lj;
  }
  return ln.row ? t : 0.0;
}

// The three components of the lane's contact of a row-lane quantity.
template <int NS>
__device__ __forceinline__ void contact3(double v, const Lane<NS>& ln, double* o) {
#pragma unroll
  for (int k = 0; k < 3; ++k) o[k] = __shfl_sync(kFull, v, ln.base + 3 * ln.ci + k);
}

// FP64 NCP residual of lambda (the max over contacts of the one-thread ncp_residual terms).
template <int NS, class SM>
__device__ double residual(const SM& S, const Lane<NS>& ln, double lam) {
  const double sg = sigma_row<NS>(S, ln, lam);
  double s[3], l[3];
  contact3<NS>(sg, ln, s);
  contact3<NS>(lam, ln, l);
  double r = 0.0;
  if (ln.row && ln.kc == 0 && ln.ci < ln.na) {
    const double w[3] = {s[0], s[1], s[2] + ln.mu * sqrt(s[0] * s[0] + s[1] * s[1])};
    double p[3];
    proj_cone(l, ln.mu, p);
    r = fmax(r, sqrt((l[0] - p[0]) * (l[0] - p[0]) + (l[1] - p[1]) * (l[1] - p[1]) + (l[2] - p[2]) * (l[2] - p[2])));
    proj_cone(w, 1.0 / ln.mu, p);
    r = fmax(r, sqrt((w[0] - p[0]) * (w[0] - p[0]) + (w[1] - p[1]) * (w[1] - p[1]) + (w[2] - p[2]) * (w[2] - p[2])));
    r = fmax(r, fabs(l[0] * w[0] + l[1] * w[1] + l[2] * w[2]));
  }
  return gmax<Shape<NS>::L>(r);
}

// Modes (same rules as the one-thread classify); every lane gets the mode of its contact.
// Returns the classification margin (group-uniform).
template <int NS, class SM>
__device__ double classify(const SM& S, const Lane<NS>& ln, double lam, double es_rel, double el_rel,
                           int& mode) {
  constexpr int L = Shape<NS>::L;
  const bool in = ln.row && ln.ci < ln.na;
  const double gm = fmax(1.0, gmax<L>(in ? fabs(ln.g) : 0.0));
  const double lm = fmax(1.0, gmax<L>(in ? fabs(lam) : 0.0));
  const double es = es_rel * gm, el = el_rel * lm;
  const double sg = sigma_row<NS>(S, ln, lam);
  double s[3], l[3];
  contact3<NS>(sg, ln, s);
  contact3<NS>(lam, ln, l);
  double margin = 1e300;
  mode = DS_MODE_BREAKING;
  if (ln.ci < ln.na) {
    const double ns = sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
    const double nst = sqrt(s[0] * s[0] + s[1] * s[1]);
    const double inside = ln.mu * l[2] - sqrt(l[0] * l[0] + l[1] * l[1]);
    if (ns <= es) {
      mode = DS_MODE_STICKING;
      margin = (es - ns) / es;
    } else if (s[2] > es || l[2] <= el) {
      mode = DS_MODE_BREAKING;
      margin = s[2] > es ? (s[2] - es) / gm : 0.0;
    } else if (inside > el) {
      mode = DS_MODE_STICKING;
      margin = inside / lm;
    } else {
      mode = DS_MODE_SLIDING;
      margin = fmin(nst / gm, l[2] / lm);
    }
  }
  return gmin<L>(margin);
}

// Active-set update (same rules as the one-thread reclassify); applied only where act.  Returns
// whether any mode of the env changed.
template <int NS, class SM>
__device__ bool reclassify(const SM& S, const Lane<NS>& ln, double lam, int& mode, double es, double el,
                           double delta, bool act) {
  const double sg = sigma_row<NS>(S, ln, lam);
  double s[3], l[3];
  contact3<NS>(sg, ln, s);
  contact3<NS>(lam, ln, l);
  int nm = mode;
  if (act && ln.ci < ln.na) {
    if (mode == DS_MODE_BREAKING) {
      if (s[2] < -es) nm = DS_MODE_STICKING;
    } else if (mode == DS_MODE_STICKING) {
      if (l[2] < -el) nm = DS_MODE_BREAKING;
      else if (ln.mu * l[2] - sqrt(l[0] * l[0] + l[1] * l[1]) < -delta) nm = DS_MODE_SLIDING;
    } else {
      if (l[2] < -el) nm = DS_MODE_BREAKING;
      else if (sqrt(s[0] * s[0] + s[1] * s[1]) < es) nm = DS_MODE_STICKING;
    }
  }
  const bool ch = nm != mode;
  mode = nm;
  return gany<NS>(ch, ln);
}

// The value of a[j] for a run-time column j (registers are indexed at compile time only).
template <int N>
__device__ __forceinline__ double pick(const double (&a)[N], int j) {
  double v = 0.0;
#pragma unroll
  for (int c = 0; c < N; ++c)
    if (c == j) v = a[c];
  return v;
}

// One Newton step of the reduced mode equations: the lane holds row li of the matrix (a, over the
// env's unknown columns um) and its residual F; rowact marks the rows of the reduced system.
// Returns dx of column li (0 for the columns that are not unknowns).
//
// The complete-pivot elimination swaps each pivot column into place (as the one-thread LU does), so
// that step k touches positions k .. NC3-1 only: with the step index unrolled those ranges are
// fixed at compile time and the FP64 work per step shrinks with k (the FP64 pipe is this kernel's
// bound; column moves are selects).  Columns that are not unknowns hold zeros and are never
// pivots.  mypos tracks where column li currently sits.
template <int NS, typename LT>
__device__ double solve_step(LUWork<NS, LT>& S, const Lane<NS>& ln, LT (&a)[Shape<NS>::NC3], LT F, unsigned um,
                             int nu, bool rowact, bool run) {
  using Bits = LUBits<LT>;
  constexpr int NC3 = Shape<NS>::NC3, L = Shape<NS>::L;
  int mypos = (ln.row && ((um >> ln.li) & 1u)) ? ln.li : -1;
  bool done = !(rowact && run);     // not (or no longer) a pivot candidate
  int kp = -1;                      // pivot step of this lane's row
  LT ipiv = LT(0);                  // 1 / its pivot
  int rank = 0;
  LT first = LT(0);
  bool go = run;
#pragma unroll
  for (int k = 0; k < NC3; ++k) {
    if (go && k >= nu) go = false;
    if (__any_sync(kFull, go)) {             // (once no env goes on, every later step is skipped)
      // Candidates are compared by the bit patterns of |a| as integers (the same order as the
      // values for non-negative doubles, and off the FP64 pipe); NaN entries are never candidates.
      typename Bits::I bk = -1;
      int bj = k;
      if (!done) {
#pragma unroll
        for (int j = k; j < NC3; ++j) {
          const typename Bits::I v = Bits::bits(a[j]);
          if (v <= Bits::kInf && v > bk) { bk = v; bj = j; }
        }
      }
      int key = (ln.li << 8) | bj;
#pragma unroll
      for (int o = L / 2; o >= 1; o >>= 1) {
        const typename Bits::I ov = __shfl_xor_sync(kFull, bk, o);
        const int ok = __shfl_xor_sync(kFull, key, o);
        if (ov > bk || (ov == bk && ok < key)) { bk = ov; key = ok; }
      }
      const LT bv = bk < 0 ? LT(-1) : Bits::value(bk);
      if (go) {
        if (k == 0) first = bv;
        if (!(bv > Bits::kRankTol * first) || bv == LT(0)) go = false;
      }
      const int bi = key >> 8, bjj = key & 255;
      if (go && bjj != k) {             // pivot column to position k, in every row of the env
        const LT t = a[k];
        LT nk = t;
#pragma unroll
        for (int j = k + 1; j < NC3; ++j) {
          const bool h = j == bjj;
          const LT aj = a[j];
          nk = h ? aj : nk;
          a[j] = h ? t : aj;
        }
        a[k] = nk;
        if (mypos == bjj) mypos = k;
        else if (mypos == k) mypos = bjj;
      }
      const int src = ln.base + (go ? bi : 0);
      const LT pv = __shfl_sync(kFull, a[k], src);
      const LT pf = __shfl_sync(kFull, F, src);
      const bool elim = go && !done && ln.li != bi;
      const LT inv = LT(1) / pv;
      const LT l = elim ? a[k] * inv : LT(0);
#pragma unroll
      for (int j = k + 1; j < NC3; ++j) {
        const LT pj = __shfl_sync(kFull, a[j], src);
        if (elim) a[j] -= l * pj;
      }
      if (elim) F -= l * pf;
      if (go) {
        if (ln.li == bi) { done = true; kp = k; ipiv = inv; }
        ++rank;
      }
    }
  }
  double dx = 0.0;
  const bool full = run && rank == nu;
  const bool mn = run && rank < nu;
  // full column rank: back substitution, one pivot at a time from the last
  LT s = F;
#pragma unroll
  for (int k = NC3 - 1; k >= 0; --k) {
    const bool stp = full && k < rank;
    if (__any_sync(kFull, stp)) {
      const unsigned ob = gbits<NS>(stp && kp == k, ln);
      const int own = ob ? __ffs(ob) - 1 : 0;
      LT xk = LT(0);
      if (stp && kp == k) xk = s * ipiv;
      xk = __shfl_sync(kFull, xk, ln.base + own);
      if (stp && kp >= 0 && kp < k) s -= a[k] * xk;
      if (stp && mypos == k) dx = double(xk);
    }
  }
  // rank deficient: x = U^T (U U^T)^-1 y over the positions, then back to the columns
  if (__any_sync(kFull, mn)) {
    const int maxrank = int(__reduce_max_sync(kFull, unsigned(mn ? rank : 0)));
    if (mn && kp >= 0) {
#pragma unroll
      for (int j = 0; j < NC3; ++j) S.U[kp][j] = j >= kp ? a[j] : LT(0);
    }
    __syncwarp();
    if (mn && kp >= 0) {
      for (int k2 = 0; k2 <= kp; ++k2) {
        LT t = LT(0);
#pragma unroll
        for (int j = 0; j < NC3; ++j) t += S.U[kp][j] * S.U[k2][j];
        S.H[kp][k2] = t;
      }
    }
    __syncwarp();
    // Cholesky of U U^T (rows in pivot order; lane kp owns row kp)
#pragma unroll 1
    for (int j = 0; j < maxrank; ++j) {
      const bool stp = mn && j < rank;
      if (stp && kp == j) {
        LT d = S.H[j][j];
        for (int c = 0; c < j; ++c) d -= S.H[j][c] * S.H[j][c];
        const LT sd = sqrt(fmax(d, LT(1e-30)));
        S.H[j][j] = sd;
        S.rd[j] = LT(1) / sd;
      }
      __syncwarp();
      if (stp && kp > j) {
        LT t = S.H[kp][j];
        for (int c = 0; c < j; ++c) t -= S.H[kp][c] * S.H[j][c];
        S.H[kp][j] = t * S.rd[j];
      }
      __syncwarp();
    }
    // forward (L w = y) and backward (L^T z = w) substitution, column sweeps
    LT acc = LT(0), wv = LT(0);
#pragma unroll 1
    for (int j = 0; j < maxrank; ++j) {
      const bool stp = mn && j < rank;
      const unsigned ob = gbits<NS>(stp && kp == j, ln);
      const int own = ob ? __ffs(ob) - 1 : 0;
      LT wj = LT(0);
      if (stp && kp == j) { wv = (s - acc) * S.rd[j]; wj = wv; }
      wj = __shfl_sync(kFull, wj, ln.base + own);
      if (stp && kp > j) acc += S.H[kp][j] * wj;
    }
    LT acc2 = LT(0), zv = LT(0);
#pragma unroll 1
    for (int j = maxrank - 1; j >= 0; --j) {
      const bool stp = mn && j < rank;
      const unsigned ob = gbits<NS>(stp && kp == j, ln);
      const int own = ob ? __ffs(ob) - 1 : 0;
      LT zj = LT(0);
      if (stp && kp == j) { zv = (wv - acc2) * S.rd[j]; zj = zv; }
      zj = __shfl_sync(kFull, zj, ln.base + own);
      if (stp && kp >= 0 && kp < j) acc2 += S.H[j][kp] * zj;
    }
    if (mn && kp >= 0) S.w[kp] = zv;
    __syncwarp();
    if (mn && mypos >= 0) {
      LT t = LT(0);
      for (int k = 0; k < rank; ++k) t += S.U[k][mypos] * S.w[k];
      dx = double(t);
    }
    __syncwarp();
  }
  return dx;
}

// Newton on the mode equations of the env (the one-thread newton_modes, one lane per row).
// lp is the lane's component of lambda (row lanes); act marks the envs that take part.
template <int NS, typename LT, class SM>
__device__ double newton_modes(const SM& S, LUWork<NS, LT>& W, const Lane<NS>& ln, double lp, int mode, int iters,
                               double sat_delta, bool act) {
  constexpr int NC3 = Shape<NS>::NC3, L = Shape<NS>::L;
  const bool inc = ln.ci < ln.na;
  const double scale = fmax(1.0, gmax<L>((ln.row && inc) ? fabs(ln.g) : 0.0));
  if (act && ln.row && inc && mode == DS_MODE_BREAKING) lp = 0.0;
  double l[3];
  contact3<NS>(lp, ln, l);
  const double nt0 = sqrt(l[0] * l[0] + l[1] * l[1]);
  const bool sat = act && inc && mode == DS_MODE_STICKING && nt0 > 0.0 && ln.mu * l[2] - nt0 <= sat_delta;
  const bool ucol = act && ln.row && inc && mode != DS_MODE_BREAKING;
  const unsigned um = gbits<NS>(ucol, ln);
  const int nu = __popc(um);
  const bool rowact = ln.row ? ucol : sat;
  bool run = act && nu > 0;
  double prev = 1e300;
#pragma unroll 1
  for (int it = 0; it < iters; ++it) {
    if (!__any_sync(kFull, run)) break;
    const double sg = sigma_row<NS>(S, ln, lp);
    double s[3];
    contact3<NS>(sg, ln, s);
    contact3<NS>(lp, ln, l);
    double a[NC3];
    double F = 0.0;
#pragma unroll
    for (int j = 0; j < NC3; ++j) a[j] = 0.0;
    if (rowact && ln.row) {
      const int r0 = 3 * ln.ci;
      if (mode == DS_MODE_STICKING || ln.kc == 2) {
#pragma unroll
        for (int j = 0; j < NC3; ++j) a[j] = ((um >> j) & 1u) ? S.G[ln.li][j] : 0.0;
        F = sg;
      } else {
        const double ns = sqrt(s[0] * s[0] + s[1] * s[1]);
        const double u0 = s[0] / ns, u1 = s[1] / ns;
        const double uk = ln.kc == 0 ? u0 : u1;
        const double k = ln.mu * l[2] / ns;
        F = lp + ln.mu * l[2] * uk;
        const double c0 = (ln.kc == 0 ? 1.0 : 0.0) - uk * u0;
        const double c1 = (ln.kc == 1 ? 1.0 : 0.0) - uk * u1;
#pragma unroll
        for (int j = 0; j < NC3; ++j)
          a[j] = ((um >> j) & 1u) ? k * (c0 * S.G[r0][j] + c1 * S.G[r0 + 1][j]) : 0.0;
#pragma unroll
        for (int j = 0; j < NC3; ++j) {
          if (j == ln.li) a[j] += 1.0;
          if (j == r0 + 2) a[j] += ln.mu * uk;
        }
      }
    } else if (rowact) {
      const int r0 = 3 * ln.ci;
      const double nt = sqrt(l[0] * l[0] + l[1] * l[1]);
      F = ln.mu * l[2] - nt;
#pragma unroll
      for (int j = 0; j < NC3; ++j)
        a[j] = j == r0 ? -l[0] / nt : (j == r0 + 1 ? -l[1] / nt : (j == r0 + 2 ? ln.mu : 0.0));
    }
    const double fmaxv = gmax<L>(rowact ? fabs(F) : 0.0);
    if (run) {
      if (!(fmaxv > 1e-15 * scale)) run = false;
      else if (it >= 2 && !(fmaxv < 0.5 * prev)) run = false;
      else prev = fmaxv;
    }
    if (!__any_sync(kFull, run)) break;
    LT al[NC3];
#pragma unroll
    for (int j = 0; j < NC3; ++j) al[j] = LT(a[j]);
    const double dx = solve_step<NS, LT>(W, ln, al, LT(F), um, nu, rowact, run);
    if (run && ucol) lp -= dx;
  }
  return lp;
}

// End of an ADMM stage (the one-thread newton_stage): classify z, up to four active-set rounds of
// Newton, keep the best candidate by FP64 NCP residual; with `enumerate`, a failure falls back to
// the contact-mode patterns of enum_mode (FP64 Newton from z on each, in order, until one passes).
// lz and best_l are the lane's components.
template <int NS, typename T>
__device__ bool newton_stage(Smem<NS, T>& S, const Lane<NS>& ln, double lz, double eps, const KArgs& a, double& best_l,
                             double& best_r, bool act, bool last, bool enumerate) {
  constexpr int L = Shape<NS>::L;
  const bool in = ln.row && ln.ci < ln.na;
  const double scale = fmax(1.0, gmax<L>(in ? fabs(ln.g) : 0.0));
  const double tol = a.ncp_tol * scale;
  const double lscale = fmax(1.0, gmax<L>(in ? fabs(lz) : 0.0));
  const double es = fmax(a.eps_sigma, 10.0 * eps), el = fmax(a.eps_lambda, 10.0 * eps);
  const double sat_delta = 10.0 * eps * lscale;
  int mode;
  classify<NS>(S, ln, lz, es, el, mode);
  const double r0 = residual<NS>(S, ln, lz);
  if (act && r0 < best_r) { best_r = r0; best_l = lz; }
  double lp = lz;
  bool go = act && best_r > tol;
#pragma unroll 1
  for (int round = 0; round < 4; ++round) {
    if (!__any_sync(kFull, go)) break;
    // mixed form: FP32 factorisations (FP64 residuals) except in an env's last chance
    if constexpr (std::is_same<T, float>::value)
      lp = newton_modes<NS, float>(S, S.f, ln, lp, mode, a.polish_iters, sat_delta, go && !last);
    lp = newton_modes<NS, double>(S, S.d, ln, lp, mode, a.polish_iters, sat_delta,
                                  go && (last || !std::is_same<T, float>::value));
    const double rpol = residual<NS>(S, ln, lp);
    if (go && rpol < best_r) { best_r = rpol; best_l = lp; }
    if (go && best_r <= tol) go = false;
    const double th = 10.0 * a.ncp_tol * lscale;
    const bool ch = reclassify<NS>(S, ln, lp, mode, 10.0 * tol, th, th, go);
    if (go && !ch) go = false;
    double l[3], p[3];
    contact3<NS>(lp, ln, l);
    if (go && in) {
      proj_cone(l, ln.mu, p);
      lp = p[ln.kc];
    }
  }
  // fallback: the enumerated contact-mode patterns, ranked by the normal impulses of z
  bool eg = enumerate && act && best_r > tol;
  if (__any_sync(kFull, eg)) {
    int rank = 0;
#pragma unroll
    for (int c = 0; c < NS; ++c) {
      const double lnc = __shfl_sync(kFull, lz, ln.base + 3 * c + 2);
      const double own = __shfl_sync(kFull, lz, ln.base + 3 * (ln.ci < NS ? ln.ci : 0) + 2);
      if (c < ln.na && (lnc > own || (lnc == own && c < ln.ci))) ++rank;
    }
    const int npat = 2 * ln.na * ln.na;
#pragma unroll 1
    for (int pat = 0; __any_sync(kFull, eg); ++pat) {
      if (pat >= npat) eg = false;
      const int pm = (ln.ci < ln.na && pat < npat) ? enum_mode(pat, rank, ln.na) : DS_MODE_BREAKING;
      const double lq = newton_modes<NS, double>(S, S.d, ln, lz, pm, DS_ENUM_NEWTON_ITERS, sat_delta, eg);
      const double rq = residual<NS>(S, ln, lq);
      if (eg && rq < best_r) { best_r = rq; best_l = lq; }
      if (eg && best_r <= tol) eg = false;
    }
  }
  return act && best_r <= tol;
}

}  // namespace coop

// 2b, cooperative: the Newton / active-set stage for the envs whose ADMM stage ended in this round
// (and the speculative attempts), 4 NS lanes per env.  Same bookkeeping as newton_env: accept
// (write lambda, modes, status), or queue the env for the next round (in the next stage unless the
// attempt was speculative).
template <int NS, typename T>
__global__ void __launch_bounds__(coop::Shape<NS>::THREADS, coop::Shape<NS>::MINB) newton_coop_kernel(KArgs a) {
  using Sh = coop::Shape<NS>;
  constexpr int NC3 = Sh::NC3, L = Sh::L, EPW = Sh::EPW;
  static_assert(32 % L == 0, "4 NS lanes per env must divide the warp");
  __shared__ coop::Smem<NS, T> smem[(Sh::THREADS / 32) * EPW];
  const WsView& w = a.ws;
  const int n = w.ncounts[a.round];
  const int B = a.B;
  const int lane = threadIdx.x & 31;
  const int grp = lane / L;
  coop::Smem<NS, T>& S = smem[DS_IX((threadIdx.x >> 5) * EPW + grp, (Sh::THREADS / 32) * EPW)];
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int t0 = warp * EPW; t0 < n; t0 += nwarps * EPW) {
    const int t = t0 + grp;
    const bool have = t < n;
    // entry e: the env's ADMM stage ended; ~e: a speculative attempt on an unconverged iterate
    const int entry = have ? w.nlist[t] : 0;
    const bool spec = entry < 0;
    const int e = have ? DS_IX(spec ? ~entry : entry, B) : 0;
    coop::Lane<NS> ln;
    ln.li = lane - grp * L;
    ln.base = grp * L;
    ln.row = ln.li < NC3;
    ln.ci = ln.row ? ln.li / 3 : ln.li - NC3;
    ln.kc = ln.row ? ln.li - 3 * ln.ci : 0;
    ln.na = have ? w.na[e] : 0;
    const int m = 3 * ln.na;
    const bool mine = ln.row && ln.li < m;
    ln.mu = ln.ci < ln.na ? w.mu[ln.ci * B + e] : 0.0;
    ln.g = mine ? w.g[ln.li * B + e] : 0.0;
    if (ln.row) {
#pragma unroll
      for (int j = 0; j < NC3; ++j) {
        double v = 0.0;
        if (mine && j < m) v = j <= ln.li ? w.G[tri(ln.li, j) * B + e] : w.G[tri(j, ln.li) * B + e];
        S.G[ln.li][j] = v;
      }
    }
    __syncwarp();
    const double lz = mine ? double(T(w.az[ln.li * B + e])) : 0.0;
    double best_l = mine ? w.lam[ln.li * B + e] : 0.0;
    double best_r = have ? w.best_r[e] : 1e300;
    const int stage = have ? w.stage[e] : 0;
    const int iters = have ? w.iters[e] : 0;
    uint32_t st = have ? w.st[e] : 0u;
    const double eps = stage_eps<T>(a, stage);
    const bool last = !spec && (iters >= a.admm_max_iter || stage + 1 >= num_stages<T>() || a.final_round);
    const bool ok = coop::newton_stage<NS, T>(S, ln, lz, eps, a, best_l, best_r, have && m > 0, last,
                                              a.round == a.sched.spec_from);
    if (mine) w.lam[ln.li * B + e] = best_l;
    const bool fin = ok || last;
    int mode;
    const double margin = coop::classify<NS>(S, ln, best_l, a.eps_sigma, a.eps_lambda, mode);
    if (have && fin) {
      if (ln.row && ln.kc == 0 && ln.ci < ln.na) w.mode[ln.ci * B + e] = int8_t(mode);
      if (ln.li == 0) {
        if (!ok) st |= DS_ENV_NOT_CONVERGED;
        if (margin < a.margin_delta) st |= DS_ENV_NEAR_SWITCH;
        w.st[e] = st;
        const int k = atomicAdd(&w.dcount[0], 1);
        w.dlist[k] = e;
      }
    } else if (have && ln.li == 0) {
      if (!spec) w.stage[e] = stage + 1;
      w.best_r[e] = best_r;
      const int k = atomicAdd(&w.counts[a.round + 1], 1);
      w.list[(a.round + 1) & 1][k] = e;
    }
    __syncwarp();
  }
}

}  // namespace ds
