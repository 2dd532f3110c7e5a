// Shared device-side definitions of the batched contact-step kernels (sm_103a).
#pragma once
#include <cstdint>
#include <cstring>
#include <type_traits>

#include <cuda_runtime.h>

#include "diffsim.h"

// Device functions are also host-callable so that the same templates can be run on the CPU.
#define DS_HD __host__ __device__
#define DS_HDI __host__ __device__ __forceinline__

// Checked build (compiled with -DDS_CHECK, a debugging aid): the tree indices (bodies, parents,
// dofs, subtrees), the env indices read from the work lists and the shared-memory group indices go
// through DS_IX, which counts an index outside [0, n) in this translation unit's counter (read by
// ds_check_bad_indices) and uses 0 instead, so a bad index shows up as a count, not a memory fault.
// In the normal build DS_IX is the index itself.
#ifdef DS_CHECK
static __device__ unsigned int ds_check_bad;
DS_HDI int ds_ix(int i, int n) {
  if (static_cast<unsigned>(i) < static_cast<unsigned>(n)) return i;
#ifdef __CUDA_ARCH__
  atomicAdd(&ds_check_bad, 1u);
#endif
  return 0;
}
#define DS_IX(i, n) ds_ix((i), (n))
#else
#define DS_IX(i, n) (i)
#endif

#define DS_MAXB 32       // bodies per model
#define DS_MAXNV 36      // velocity dofs per model
#define DS_MAXSLOTS 16   // contact slots per env

// Device copy of a model.  Bodies are in depth-first preorder: the subtree of body i is the index
// range [i, sub_end[i]).  A dof is a column of a joint's motion subspace; the dofs of body i are
// iv[i] .. iv[i] + nd[i] - 1.
struct DevModel {
  int nb, nq, nv, pad;
  int parent[DS_MAXB], jtype[DS_MAXB], iq[DS_MAXB], iv[DS_MAXB], nd[DS_MAXB], sub_end[DS_MAXB];
  int dof_body[DS_MAXNV];
  int dof_parent[DS_MAXNV];   // the dof before each dof on its path to the root (-1 at the root)
  double axis[DS_MAXB][3], jrot[DS_MAXB][9], jpos[DS_MAXB][3];
  double mass[DS_MAXB], com[DS_MAXB][3], inertia[DS_MAXB][6];
};

enum { DS_RUN_STEP = 0, DS_RUN_JAC = 1, DS_RUN_VJP = 2 };

// Workspace of the three-kernel pipeline (setup -> compacted ADMM rounds -> finish), structure of
// arrays over the batch.  Carved out of one caller-provided buffer by ds_workspace_layout().
#define DS_ROUNDS 9

// Newton steps per pattern of the fallback enumeration (a pattern that is the solution converges
// quadratically from a nearby iterate; the others are dropped early).
#define DS_ENUM_NEWTON_ITERS 5

// Mode of the contact of rank `rank` (0 = the largest normal impulse in the iterate) in pattern p
// of the fallback enumeration: first the 2 na patterns with one contact in contact (sticking, then
// sliding), then for each pair of ranks (ra < rb, in order) its four sticking / sliding
// combinations; every other contact breaks.  2 na^2 patterns in all.
DS_HDI int enum_mode(int p, int rank, int na) {
  if (p < 2 * na) return rank == p / 2 ? ((p & 1) ? 2 : 1) : 0;
  p -= 2 * na;
  int pair = p >> 2;
  const int combo = p & 3;
  int ra = 0, cnt = na - 1;
  while (cnt > 0 && pair >= cnt) { pair -= cnt; ++ra; --cnt; }
  const int rb = ra + 1 + pair;
  if (rank == ra) return (combo & 1) ? 2 : 1;
  if (rank == rb) return (combo & 2) ? 2 : 1;
  return 0;
}

// ADMM iterations an env may run in round r before the lists are regrouped (and before its iterate
// is tried by the Newton stage, in the rounds with speculative attempts), for the three tables:
// {32, 32, 64, ..., 4096} (0), halved (1), doubled with 4096 kept as the last cap (2).  The last
// round runs to the iteration limit whatever its cap.
DS_HDI int ds_round_cap(int table, int r) {
  const int base = table == 1 ? 16 : (table == 2 ? 64 : 32);
  const int c = r == 0 ? base : base << (r - 1);
  return c > 4096 ? 4096 : c;
}
// Rows (of B doubles) of the forward state that a pipeline step keeps per env from its setup for
// its finish, for a model of nb bodies, nv dofs and ns contact slots (order: FwLayout).
DS_HDI int ds_forward_rows(int nb, int nv, int ns) {
  return 8 * nv + 28 * nb + nv * (nv + 1) / 2 + 6 * ns * nv + 9 * ns;
}

// Rows (of B doubles) of the split finish's per-env column state (order: ColState::visit), for
// a model of nb bodies, nv dofs and ns contact slots; stored in the forward-state rows, which
// are sized for the larger of the two.
DS_HDI constexpr int ds_colstate_rows(int nb, int nv, int ns) {
  return 6 * nv + 2 * nv + 10 * nb + 7 * 6 * nb + nv * (nv + 1) / 2 + 9 * ns + 9 + 3 * ns * nv + nv * 3 * ns +
         2 * nv + 3 * ns + ns + nv + ns + ns + 2;
}

struct WsView {
  int32_t* counts;        // [DS_ROUNDS + 1] envs queued for each round
  int32_t* list[2];       // [B] ping-pong work lists of env indices
  int32_t* na;            // [B] active contacts
  int32_t* stage;         // [B] current ADMM stage
  int32_t* iters;         // [B] ADMM iterations so far
  uint32_t* st;           // [B] status bits
  int8_t* mode;           // [NS][B] modes of the active contacts
  double* mu;             // [NS][B]
  double* G;              // [NC3 (NC3 + 1) / 2][B] Delassus matrix, packed lower, FP64
  double* g;              // [NC3][B]
  double* lam;            // [NC3][B] best impulse so far / result
  double* best_r;         // [B] its NCP residual
  double *ax, *az, *ay, *asx;  // [NC3][B] ADMM state
  double* K;              // [NC3 NC3][B] (G + rho I)^-1, row-major
  double* rho;            // [B]
  double* fw;             // [forward rows][B] the setup's forward state, read by the finish
  int32_t* nlist;         // [B] envs whose ADMM stage ended in a round (Newton queue)
  int32_t* ncounts;       // [DS_ROUNDS]
  int32_t* fetch;         // [DS_ROUNDS] next unclaimed entry of each round's list (follows ncounts)
  int32_t* dlist;         // [B] envs whose NCP solve is complete, in completion order
  int32_t* dcount;        // [2] entries of dlist; a snapshot of it (follows fetch)
  int32_t* claim;         // [1] next unclaimed work item of the overlapped finish (follows dcount)
  int32_t* queue;         // [DS_Q_COUNT + DS_PERSIST_MAXMODELS] persistent launch: queue words, then
                          // the length of each model's env list
  int32_t* qlists;        // [nmodels][B] persistent launch: env indices of each model
};

// Persistent launch (ds_schedule.persistent): at most this many models in a batch, and the words
// at the head of WsView.queue.
#define DS_PERSIST_MAXMODELS 4
enum { DS_Q_PARTED = 0, DS_Q_ABANDON = 1, DS_Q_NEXT = 2, DS_Q_TIMEOUTS = 3, DS_Q_COUNT = 4 };

// Lays out the workspace for ns contact slots, B envs, nmodels models and fw_rows rows of forward
// state per env starting at base (may be NULL to size it), and returns its size.  The per-env arrays are shared; every model has its own
// work lists and counters (its pipeline may run concurrently with the others'), and *v gets those
// of model `model`.
inline size_t ds_workspace_layout(int ns, int B, void* base, WsView* v, int nmodels = 1, int model = 0,
                                  int fw_rows = 0) {
  const int nc3 = 3 * ns;
  size_t off = 0;
  char* b = static_cast<char*>(base);
  auto take = [&](size_t bytes) -> void* {
    void* p = b ? b + off : nullptr;
    off += (bytes + 255) & ~size_t(255);
    return p;
  };
  WsView w;
  w.na = static_cast<int32_t*>(take(sizeof(int32_t) * B));
  w.stage = static_cast<int32_t*>(take(sizeof(int32_t) * B));
  w.iters = static_cast<int32_t*>(take(sizeof(int32_t) * B));
  w.st = static_cast<uint32_t*>(take(sizeof(uint32_t) * B));
  w.mode = static_cast<int8_t*>(take(size_t(ns) * B));
  w.mu = static_cast<double*>(take(sizeof(double) * ns * size_t(B)));
  w.G = static_cast<double*>(take(sizeof(double) * (nc3 * (nc3 + 1) / 2) * size_t(B)));
  w.g = static_cast<double*>(take(sizeof(double) * nc3 * size_t(B)));
  w.lam = static_cast<double*>(take(sizeof(double) * nc3 * size_t(B)));
  w.best_r = static_cast<double*>(take(sizeof(double) * size_t(B)));
  w.ax = static_cast<double*>(take(sizeof(double) * nc3 * size_t(B)));
  w.az = static_cast<double*>(take(sizeof(double) * nc3 * size_t(B)));
  w.ay = static_cast<double*>(take(sizeof(double) * nc3 * size_t(B)));
  w.asx = static_cast<double*>(take(sizeof(double) * nc3 * size_t(B)));
  w.K = static_cast<double*>(take(sizeof(double) * nc3 * nc3 * size_t(B)));
  w.rho = static_cast<double*>(take(sizeof(double) * size_t(B)));
  w.fw = static_cast<double*>(take(sizeof(double) * size_t(fw_rows) * size_t(B)));
  w.queue = static_cast<int32_t*>(take(sizeof(int32_t) * (DS_Q_COUNT + DS_PERSIST_MAXMODELS)));
  w.qlists = static_cast<int32_t*>(take(sizeof(int32_t) * size_t(nmodels) * size_t(B)));
  for (int k = 0; k < nmodels; ++k) {
    int32_t* counts = static_cast<int32_t*>(take(sizeof(int32_t) * (DS_ROUNDS + 1)));
    int32_t* l0 = static_cast<int32_t*>(take(sizeof(int32_t) * B));
    int32_t* l1 = static_cast<int32_t*>(take(sizeof(int32_t) * B));
    int32_t* nl = static_cast<int32_t*>(take(sizeof(int32_t) * B));
    int32_t* nc = static_cast<int32_t*>(take(sizeof(int32_t) * (2 * DS_ROUNDS + 3)));
    int32_t* dl = static_cast<int32_t*>(take(sizeof(int32_t) * B));
    if (k == model) {
      w.counts = counts;
      w.list[0] = l0;
      w.list[1] = l1;
      w.nlist = nl;
      w.ncounts = nc;
      w.fetch = nc + DS_ROUNDS;
      w.dcount = nc + 2 * DS_ROUNDS;
      w.claim = nc + 2 * DS_ROUNDS + 2;
      w.dlist = dl;
    }
  }
  if (v) *v = w;
  return off;
}

// How the pipeline divides the work: ADMM round-cap table, the first round run by the
// row-per-lane ADMM kernel (DS_ROUNDS = never), finish-kernel target CTAs per SM for splitting
// Jacobian columns (0 = one thread per env), Newton kernel form, and the round after which the
// envs already solved are finished on a side stream while the slow ones still iterate; whether
// the Newton stage is also tried on unconverged ADMM iterates.  It changes how the work is divided;
// what an env computes changes only by rounding (the two Newton forms) or, through the round caps
// and the speculative Newton attempts, by where the ADMM iteration is stopped: the accepted
// impulse always passes the same NCP residual test.
struct ds_schedule {
  int caps, wide_from, finish_ctas, newton_thread;
  int overlap_from;   // after this round, finish the completed envs on a side stream (DS_ROUNDS = never)
  int pair_from;      // first round of the two-warp ADMM kernel (FP64, 3 NS <= 32; DS_ROUNDS = never)
  int reserve;        // overlapped finish: keep off the SMs with smid % reserve == 0 (0 = use all)
  int spec_from;      // from the end of this round on, every env still iterating gets a Newton /
                      // active-set attempt (also when its stage tolerance was not met: it keeps
                      // its stage if the attempt fails); in this round a failed attempt falls
                      // back to enumerating the contact-mode patterns with one or two contacts in
                      // contact (DS_ROUNDS = never)
  int presolve;       // 1: the setup solves Eq. 1 exactly for the envs whose solution has a single
                      // contact in contact (the others breaking), which then skip the ADMM rounds
  int persistent;     // 1: the whole step as one persistent launch over an atomic work queue (one
                      // env per lane, every model of the batch in the same kernel), where a kernel
                      // with the batch's shapes is compiled; 0: the workspace pipeline
  int finish_split;   // 1: the finish as a prep kernel (one thread per env) and a column kernel
                      // (one warp per env, its state in shared memory); 0: one kernel, an env's
                      // columns over finish_ctas-derived threads
};

// Everything a launch needs; passed by value.
struct KArgs {
  const DevModel* model;
  const int32_t* env_list;   // envs handled by this launch (NULL: 0 .. n_env-1)
  const int32_t* model_id;   // [B] or NULL; a launch only handles envs with model_id == model_index
  int model_index;
  int n_env;
  int B, ncmax;
  const double *q, *v, *tau;
  const int32_t* c_link;
  const double *c_point, *c_radius, *c_mu, *plane;
  double dt, gx, gy, gz;
  double bkp, bkd;         // Baumgarte gains (App. D); 1, 0 (and no margin): no term
  double cmargin;          // activation distance: a slot is active when phi <= cmargin
  int solver;              // ds_solver: the NCP iteration (ADMM or projected Gauss-Seidel)
  int rho_adapt;           // ADMM penalty updated between rounds by residual balancing
  int admm_max_iter, polish_iters;
  double admm_eps, ncp_tol, eps_sigma, eps_lambda, margin_delta;
  double *v_next, *q_next, *lambda;
  uint8_t* modes;
  uint32_t* status;
  int32_t* iters;
  double *dv_dq, *dv_dv, *dv_dtau;
  const double* vbar;
  // tape of a preceding sim_step on the same inputs (per slot impulses and modes, status): the
  // finish reads the NCP solution from it instead of solving (NULL = no tape)
  const double* tlam;
  const uint8_t* tmodes;
  const uint32_t* tstat;
  const double* qnbar;     // [nv][B] cotangent of q+ (tangent coordinates) or NULL
  double *q_bar, *v_bar, *tau_bar;
  int run;
  WsView ws;               // pipeline workspace (unused by the fused kernel)
  int round, round_cap, final_round;
  int nchunk;              // finish kernel: threads per env (Jacobian columns split between them)
  int fin_reserve;         // finish kernel: CTAs on SMs with smid % fin_reserve == 0 return at once
  int32_t* claim;          // finish kernel: work items claimed a warp at a time from *claim (NULL:
                           // a static grid-stride split)
  ds_schedule sched;
  // finish kernel over a device-side range of ws.dlist: entries [*flo, *fhi) (flo NULL = from 0);
  // fhi NULL = every env of the launch
  const int32_t* flo;
  const int32_t* fhi;
  cudaStream_t side;       // pipeline: stream for the overlapped finish (NULL = no overlap)
  cudaEvent_t ev_fork, ev_join;
};

typedef void (*ds_launch_fn)(const KArgs& a, cudaStream_t s);

// Stage tracing: when enabled, the launchers bracket every kernel with events on its stream.
enum { DS_STAGE_SETUP = 0, DS_STAGE_ADMM = 1, DS_STAGE_NEWTON = 2, DS_STAGE_FINISH = 3, DS_STAGE_FUSED = 4,
       DS_NSTAGES = 5 };
void ds_trace_mark(int stage, int begin, cudaStream_t s);   // no-op unless tracing is on

// Registry of compiled shapes: (bodies, dofs, contact slots, precision) -> launchers of the fused
// kernel and of the workspace pipeline.
struct ds_kernel_entry {
  int nb, nv, ns, precision;
  ds_launch_fn fn;
  ds_launch_fn pipeline;
  ds_launch_fn tape;       // finish only, from a tape (KArgs.tlam / tmodes / tstat)
  unsigned (*check)();     // checked build: reads and clears the shape's bad-index count (else 0)
};
// Persistent launch: the models of the batch (device copies), each one's index in the kernel's
// shape list, the order in which their chunks of envs are numbered, and the queue.
struct PArgs {
  const DevModel* model[DS_PERSIST_MAXMODELS];
  int shape[DS_PERSIST_MAXMODELS];   // index of each model's shape in the kernel's shape list
  int order[DS_PERSIST_MAXMODELS];   // models in the order their chunks are numbered
  int nv[DS_PERSIST_MAXMODELS];      // velocity dofs of each model (the NaN preset of v+)
  int nmodels;
  int poll_limit;                    // polls of the partition count before a CTA gives up
  int32_t* queue;                    // WsView.queue
  int32_t* lists;                    // WsView.qlists
};
typedef void (*ds_persist_fn)(const KArgs& a, const PArgs& p, cudaStream_t s);
struct ds_persist_entry {
  int precision, nshapes;
  int shape[DS_PERSIST_MAXMODELS][3];   // {bodies, dofs, contact slots} per shape index
  ds_persist_fn launch;
  unsigned (*check)();
};
// The persistent kernel of a precision (NULL if none is compiled).
extern "C++" const ds_persist_entry* ds_persist_kernel(int precision);

// Sum over the compiled shapes of their bad-index counts, cleared (0 in the normal build).
extern "C++" unsigned long long ds_check_sum();
extern "C++" const ds_kernel_entry* ds_find_kernel(int nb, int nv, int ns, int precision);
extern "C++" const ds_kernel_entry* ds_fit_kernel(int nb, int nv, int slots, int ncmax, int precision);
// Whether calls of this host thread may use the library's helper streams (on by default).
extern "C++" void ds_allow_helper_streams(bool on);

// ------------------------------------------------------------------------------ small algebra

template <typename T>
DS_HDI void cross3(const T* a, const T* b, T* o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

template <typename T>
DS_HDI T dot3(const T* a, const T* b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

template <typename T>
DS_HDI T dot6(const T* a, const T* b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2] + a[3] * b[3] + a[4] * b[4] + a[5] * b[5];
}

// Spatial vectors are (linear, angular), expressed in world axes at the world origin.
// o = a x b (motion cross product); o must not alias a or b.
template <typename T>
DS_HDI void mcross(const T* a, const T* b, T* o) {
  T t1[3], t2[3];
  cross3(a + 3, b, t1);
  cross3(a, b + 3, t2);
  o[0] = t1[0] + t2[0];
  o[1] = t1[1] + t2[1];
  o[2] = t1[2] + t2[2];
  cross3(a + 3, b + 3, o + 3);
}

// o = a x* f (force cross product); o must not alias a or f.
template <typename T>
DS_HDI void fcross(const T* a, const T* f, T* o) {
  T t1[3], t2[3];
  cross3(a + 3, f, o);
  cross3(a + 3, f + 3, t1);
  cross3(a, f, t2);
  o[3] = t1[0] + t2[0];
  o[4] = t1[1] + t2[1];
  o[5] = t1[2] + t2[2];
}

// Spatial inertia about the world origin, 10 numbers: mass m, first moment h = m c, rotational
// inertia about the origin (xx, yy, zz, xy, xz, yz).  o = I x; o must not alias x.
template <typename T>
DS_HDI void iapply(const T* I, const T* x, T* o) {
  const T m = I[0];
  const T* h = I + 1;
  const T* J = I + 4;
  T t[3];
  cross3(x + 3, h, t);
  o[0] = m * x[0] + t[0];
  o[1] = m * x[1] + t[1];
  o[2] = m * x[2] + t[2];
  cross3(h, x, t);
  o[3] = t[0] + J[0] * x[3] + J[3] * x[4] + J[4] * x[5];
  o[4] = t[1] + J[3] * x[3] + J[1] * x[4] + J[5] * x[5];
  o[5] = t[2] + J[4] * x[3] + J[5] * x[4] + J[2] * x[5];
}

DS_HDI int tri(int i, int j) { return i * (i + 1) / 2 + j; }  // i >= j

// In-place Cholesky of a packed lower-triangular n x n matrix; returns false if not positive.
template <typename T>
DS_HD bool chol_packed(T* L, int n) {
  for (int j = 0; j < n; ++j) {
    T s = L[tri(j, j)];
    for (int k = 0; k < j; ++k) s -= L[tri(j, k)] * L[tri(j, k)];
    if (!(s > T(0))) return false;
    const T d = sqrt(s);
    L[tri(j, j)] = d;
    const T inv = T(1) / d;
    for (int i = j + 1; i < n; ++i) {
      T t = L[tri(i, j)];
      for (int k = 0; k < j; ++k) t -= L[tri(i, k)] * L[tri(j, k)];
      L[tri(i, j)] = t * inv;
    }
  }
  return true;
}

// x <- L^-1 x
template <typename T>
DS_HDI void fwd_packed(const T* L, T* x, int n) {
  for (int i = 0; i < n; ++i) {
    T s = x[i];
    for (int k = 0; k < i; ++k) s -= L[tri(i, k)] * x[k];
    x[i] = s / L[tri(i, i)];
  }
}

// x <- L^-T x
template <typename T>
DS_HDI void bwd_packed(const T* L, T* x, int n) {
  for (int i = n - 1; i >= 0; --i) {
    T s = x[i];
    for (int k = i + 1; k < n; ++k) s -= L[tri(k, i)] * x[k];
    x[i] = s / L[tri(i, i)];
  }
}

// Factorisation M = L^T L of the joint-space inertia matrix, whose nonzeros lie on pairs of dofs one
// of which is an ancestor of the other (par[k] < k is the dof before k on its path to the root, -1
// at the root; packed lower storage, entries of other pairs zero).  The elimination runs from the
// leaves to the root, so the factor keeps the tree's sparsity (no fill-in): the factorisation, and
// the solves below, touch only ancestor pairs -- the kinematic-tree sparsity of Sec. 3.3 (for a
// chain, every pair).  Returns false if M is not positive definite.
template <typename T>
DS_HD bool ltl_factor(T* L, int n, const int* par) {
  for (int k = n - 1; k >= 0; --k) {
    const T d = L[tri(k, k)];
    if (!(d > T(0))) return false;
    const T s = sqrt(d);
    L[tri(k, k)] = s;
    const T inv = T(1) / s;
    for (int i = par[k]; i >= 0; i = par[DS_IX(i, n)]) L[tri(k, i)] *= inv;
    for (int i = par[k]; i >= 0; i = par[DS_IX(i, n)]) {
      const T a = L[tri(k, i)];
      for (int j = i; j >= 0; j = par[DS_IX(j, n)]) L[tri(i, j)] -= a * L[tri(k, j)];
    }
  }
  return true;
}

// x <- L^-T x (from the leaves to the root)
template <typename T>
DS_HDI void ltl_solve_t(const T* L, T* x, int n, const int* par) {
  for (int k = n - 1; k >= 0; --k) {
    const T xk = x[k] / L[tri(k, k)];
    x[k] = xk;
    for (int i = par[k]; i >= 0; i = par[DS_IX(i, n)]) x[i] -= L[tri(k, i)] * xk;
  }
}

// x <- L^-1 x (from the root to the leaves); M^-1 b = L^-1 L^-T b
template <typename T>
DS_HDI void ltl_solve(const T* L, T* x, int n, const int* par) {
  for (int k = 0; k < n; ++k) {
    T s = x[k];
    for (int i = par[k]; i >= 0; i = par[DS_IX(i, n)]) s -= L[tri(k, i)] * x[i];
    x[k] = s / L[tri(k, k)];
  }
}

// LU factorisation with complete pivoting, P A Q = L U, in FP64, for an r x c matrix (r <= MR,
// c <= MC).  Rank-revealing: pivots below rel_tol * |first pivot| are treated as zero and the
// corresponding unknowns are set to 0 (basic solution), which solves consistent singular or
// over-determined systems exactly.
template <int MR, int MC>
struct LUcp {
  double a[MR][MC];
  int pr[MR], pc[MC];
  int r, c, rank;

  DS_HD void factor(double rel_tol) {
    for (int i = 0; i < r; ++i) pr[i] = i;
    for (int j = 0; j < c; ++j) pc[j] = j;
    double first = 0.0;
    const int kmax = r < c ? r : c;
    rank = kmax;
    for (int k = 0; k < kmax; ++k) {
      double best = -1.0;
      int bi = k, bj = k;
      for (int i = k; i < r; ++i)
        for (int j = k; j < c; ++j) {
          const double v = fabs(a[i][j]);
          if (v > best) { best = v; bi = i; bj = j; }
        }
      if (k == 0) first = best;
      if (!(best > rel_tol * first) || best == 0.0) { rank = k; return; }
      if (bi != k) {
        for (int j = 0; j < c; ++j) { double t = a[k][j]; a[k][j] = a[bi][j]; a[bi][j] = t; }
        int t = pr[k]; pr[k] = pr[bi]; pr[bi] = t;
      }
      if (bj != k) {
        for (int i = 0; i < r; ++i) { double t = a[i][k]; a[i][k] = a[i][bj]; a[i][bj] = t; }
        int t = pc[k]; pc[k] = pc[bj]; pc[bj] = t;
      }
      const double inv = 1.0 / a[k][k];
      for (int i = k + 1; i < r; ++i) {
        const double l = a[i][k] * inv;
        a[i][k] = l;
        for (int j = k + 1; j < c; ++j) a[i][j] -= l * a[k][j];
      }
    }
  }

  // Null-space basis of the factored matrix (c - rank columns, stored as rows of nb[][]) and the
  // Cholesky factor of its Gram matrix, for minimum-norm solutions.
  double nb[MC][MC];
  double ng[MC * (MC + 1) / 2];
  int nk;

  DS_HD void nullspace() {
    nk = c - rank;
    for (int j = 0; j < nk; ++j) {
      double w[MC];
      for (int i = rank - 1; i >= 0; --i) {       // w = -U11^-1 U12[:, j]
        double s = -a[i][rank + j];
        for (int k = i + 1; k < rank; ++k) s -= a[i][k] * w[k];
        w[i] = s / a[i][i];
      }
      for (int i = 0; i < c; ++i) nb[j][pc[i]] = i < rank ? w[i] : (i - rank == j ? 1.0 : 0.0);
    }
    for (int i = 0; i < nk; ++i)
      for (int j = 0; j <= i; ++j) {
        double t = 0.0;
        for (int k = 0; k < c; ++k) t += nb[i][k] * nb[j][k];
        ng[tri(i, j)] = t;
      }
    chol_packed(ng, nk);
  }

  // x <- x - N (N^T N)^-1 N^T x  (orthogonal projection onto the row space)
  DS_HD void project_out_null(double* x) const {
    if (nk <= 0) return;
    double t[MC];
    for (int j = 0; j < nk; ++j) {
      double s = 0.0;
      for (int k = 0; k < c; ++k) s += nb[j][k] * x[k];
      t[j] = s;
    }
    fwd_packed(ng, t, nk);
    bwd_packed(ng, t, nk);
    for (int k = 0; k < c; ++k) {
      double s = 0.0;
      for (int j = 0; j < nk; ++j) s += nb[j][k] * t[j];
      x[k] -= s;
    }
  }

  // x[c] = A^- b[r] (basic solution)
  DS_HD void solve(const double* b, double* x) const {
    double y[MR];
    for (int i = 0; i < r; ++i) y[i] = b[pr[i]];
    for (int i = 0; i < rank; ++i) {
      double s = y[i];
      for (int j = 0; j < i; ++j) s -= a[i][j] * y[j];
      y[i] = s;
    }
    for (int i = rank - 1; i >= 0; --i) {
      double s = y[i];
      for (int j = i + 1; j < rank; ++j) s -= a[i][j] * y[j];
      y[i] = s / a[i][i];
    }
    for (int j = 0; j < c; ++j) x[pc[j]] = j < rank ? y[j] : 0.0;
  }

  // minimum-norm solution of a consistent system (call nullspace() after factor())
  DS_HD void solve_mn(const double* b, double* x) const {
    solve(b, x);
    project_out_null(x);
  }

  // z[r] = (A^-)^T w[c], the transpose of the basic-solution map (square systems)
  DS_HD void solve_t(const double* w, double* z) const {
    double t[MR];
    for (int j = 0; j < c; ++j) t[j] = w[pc[j]];
    for (int i = 0; i < rank; ++i) {
      double s = t[i];
      for (int j = 0; j < i; ++j) s -= a[j][i] * t[j];
      t[i] = s / a[i][i];
    }
    for (int i = rank - 1; i >= 0; --i) {
      double s = t[i];
      for (int j = i + 1; j < rank; ++j) s -= a[j][i] * t[j];
      t[i] = s;
    }
    for (int i = 0; i < r; ++i) z[pr[i]] = i < rank ? t[i] : 0.0;
  }

  // transpose of the minimum-norm map x = P_row A^- b:  z = A^-T (P_row w)
  DS_HD void solve_t_mn(const double* w, double* z) const {
    double p[MC];
    for (int j = 0; j < c; ++j) p[j] = w[j];
    project_out_null(p);
    solve_t(p, z);
  }
};
