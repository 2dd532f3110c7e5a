// C ABI of the batched contact step: argument checks, model upload, kernel dispatch.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "ds_common.cuh"

struct ds_model {
  DevModel host;       // host copy (dims, preorder data)
  DevModel* dev;       // device copy
  int device;
};

extern "C" void ds_options_default(ds_options* o) {
  if (!o) return;
  o->dt = 1e-3;
  o->gravity[0] = 0.0; o->gravity[1] = 0.0; o->gravity[2] = -9.81;
  o->admm_max_iter = 5000;
  o->admm_eps = 1e-4;
  o->polish_iters = 10;
  o->ncp_tol = 1e-12;
  o->eps_sigma = 1e-8;
  o->eps_lambda = 1e-8;
  o->margin_delta = 1e-3;
  o->precision = DS_FP64;
  o->baumgarte_kp = 1.0;
  o->baumgarte_kd = 0.0;
  o->contact_margin = 0.0;
  o->ncp_solver = DS_ADMM;
  o->queue_poll_limit = 1 << 22;
  o->admm_rho_adapt = 0;
}

extern "C" const char* ds_status_string(ds_status s) {
  switch (s) {
    case DS_OK: return "ok";
    case DS_EINVAL: return "invalid argument";
    case DS_ECUDA: return "CUDA error";
    case DS_ENOMEM: return "out of device memory";
    case DS_EUNSUPPORTED: return "no compiled kernel for this model shape";
    case DS_ETOOLARGE: return "batch too large for the fixed scratch of sim_step_jac_noalloc";
  }
  return "unknown status";
}

extern "C" ds_status ds_model_create(const ds_model_desc* d, ds_model** out) {
  if (!d || !out) return DS_EINVAL;
  *out = nullptr;
  const int nb = d->nbodies;
  if (nb <= 0 || nb > DS_MAXB || !d->parent || !d->joint_type || !d->axis || !d->joint_rot ||
      !d->joint_pos || !d->mass || !d->com || !d->inertia)
    return DS_EINVAL;
  DevModel h;
  std::memset(&h, 0, sizeof(h));
  h.nb = nb;
  int nq = 0, nv = 0;
  for (int i = 0; i < nb; ++i) {
    const int p = d->parent[i];
    const int jt = d->joint_type[i];
    if (p >= i || p < -1) return DS_EINVAL;                 // topological order
    if (jt != 0 && jt != 1) return DS_EINVAL;
    if (jt == 1 && p != -1) return DS_EINVAL;                // free-flyer only at a root
    if (!(d->mass[i] > 0.0) || !std::isfinite(d->mass[i])) return DS_EINVAL;
    h.parent[i] = p;
    h.jtype[i] = jt;
    h.iq[i] = nq;
    h.iv[i] = nv;
    h.nd[i] = jt == 1 ? 6 : 1;
    nq += jt == 1 ? 7 : 1;
    nv += h.nd[i];
    if (nv > DS_MAXNV) return DS_EINVAL;
    for (int k = 0; k < 3; ++k) {
      h.axis[i][k] = d->axis[3 * i + k];
      h.jpos[i][k] = d->joint_pos[3 * i + k];
      h.com[i][k] = d->com[3 * i + k];
    }
    for (int k = 0; k < 9; ++k) h.jrot[i][k] = d->joint_rot[9 * i + k];
    for (int k = 0; k < 6; ++k) h.inertia[i][k] = d->inertia[6 * i + k];
    h.mass[i] = d->mass[i];
    if (jt == 0) {
      const double n2 = h.axis[i][0] * h.axis[i][0] + h.axis[i][1] * h.axis[i][1] + h.axis[i][2] * h.axis[i][2];
      if (!(std::fabs(n2 - 1.0) < 1e-9)) return DS_EINVAL;   // unit axis
    }
  }
  h.nq = nq;
  h.nv = nv;
  // subtree ranges; preorder means every subtree is a contiguous index range
  for (int i = 0; i < nb; ++i) {
    int e = i + 1;
    while (e < nb) {
      int b = e;
      while (b > i) b = h.parent[b];
      if (b != i) break;
      ++e;
    }
    h.sub_end[i] = e;
    for (int k = e; k < nb; ++k) {
      int b = k;
      while (b > i) b = h.parent[b];
      if (b == i) return DS_EINVAL;                          // not depth-first preorder
    }
    for (int dd = h.iv[i]; dd < h.iv[i] + h.nd[i]; ++dd) {
      h.dof_body[dd] = i;
      h.dof_parent[dd] = dd > h.iv[i] ? dd - 1 : (h.parent[i] >= 0 ? h.iv[h.parent[i]] + h.nd[h.parent[i]] - 1 : -1);
    }
  }
  ds_model* m = new (std::nothrow) ds_model;
  if (!m) return DS_ENOMEM;
  m->host = h;
  if (cudaGetDevice(&m->device) != cudaSuccess) { delete m; return DS_ECUDA; }
  if (cudaMalloc(&m->dev, sizeof(DevModel)) != cudaSuccess) { delete m; return DS_ENOMEM; }
  if (cudaMemcpy(m->dev, &h, sizeof(DevModel), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(m->dev);
    delete m;
    return DS_ECUDA;
  }
  *out = m;
  return DS_OK;
}

extern "C" ds_status ds_model_destroy(ds_model* m) {
  if (!m) return DS_EINVAL;
  cudaFree(m->dev);
  delete m;
  return DS_OK;
}

extern "C" ds_status ds_model_dims(const ds_model* m, int32_t* nb, int32_t* nq, int32_t* nv) {
  if (!m) return DS_EINVAL;
  if (nb) *nb = m->host.nb;
  if (nq) *nq = m->host.nq;
  if (nv) *nv = m->host.nv;
  return DS_OK;
}

// Rows of forward state per env in the workspace: the most any model of the batch needs (each env
// uses its own model's rows).  -1 when a model is missing or has no kernel for its slots.
static int forward_rows(const ds_model* const* models, int32_t nmodels, const ds_batch* b, const ds_options* o) {
  int rows = 0;
  for (int k = 0; k < nmodels; ++k) {
    if (!models[k]) return -1;
    const int slots = b->model_slots ? b->model_slots[k] : b->ncmax;
    if (slots < 0 || slots > b->ncmax) return -1;
    const ds_kernel_entry* ke = ds_fit_kernel(models[k]->host.nb, models[k]->host.nv, slots, b->ncmax, o->precision);
    if (!ke) return -1;
    const int r = std::max(ds_forward_rows(ke->nb, ke->nv, ke->ns), ds_colstate_rows(ke->nb, ke->nv, ke->ns));
    if (r > rows) rows = r;
  }
  return rows;
}

extern "C" ds_status ds_workspace_size(const ds_model* const* models, int32_t nmodels, const ds_batch* b,
                                       const ds_options* o, size_t* bytes) {
  if (!models || nmodels <= 0 || !b || !o || !bytes) return DS_EINVAL;
  if (b->B < 0 || b->ncmax < 0 || b->ncmax > DS_MAXSLOTS) return DS_EINVAL;
  const int fw = forward_rows(models, nmodels, b, o);
  if (fw < 0) return DS_EINVAL;
  *bytes = ds_workspace_layout(b->ncmax, b->B, nullptr, nullptr, nmodels, 0, fw);
  return DS_OK;
}

// Set only while ds_autotune times a candidate, for the calls of its own thread.
static thread_local const ds_schedule* g_force_sched = nullptr;

// Helper streams, created on first use per device and kept until exit: streams 0-3 run the
// pipelines of a mixed-model batch, streams 4-7 their overlapped finish (side streams).
static constexpr int kHelperStreams = 4;
struct HelperStreams {
  cudaStream_t s[2 * kHelperStreams];
  cudaEvent_t fork, join[kHelperStreams];
  cudaEvent_t side_fork[kHelperStreams], side_join[kHelperStreams];
};

// Cleared by sim_step_jac_noalloc around its call: it creates no streams or events.
static thread_local bool g_allow_helpers = true;
void ds_allow_helper_streams(bool on) { g_allow_helpers = on; }

static ds_status helper_streams(HelperStreams** out) {
  static std::mutex mu;
  static HelperStreams* per_dev[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return DS_ECUDA;
  std::lock_guard<std::mutex> lock(mu);
  if (!per_dev[dev]) {
    HelperStreams* h = new (std::nothrow) HelperStreams;
    if (!h) return DS_ENOMEM;
    bool ok = cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming) == cudaSuccess;
    for (int j = 0; j < 2 * kHelperStreams && ok; ++j)
      ok = cudaStreamCreateWithFlags(&h->s[j], cudaStreamNonBlocking) == cudaSuccess;
    for (int j = 0; j < kHelperStreams && ok; ++j)
      ok = cudaEventCreateWithFlags(&h->join[j], cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&h->side_fork[j], cudaEventDisableTiming) == cudaSuccess &&
           cudaEventCreateWithFlags(&h->side_join[j], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) { delete h; return DS_ECUDA; }
    per_dev[dev] = h;
  }
  *out = per_dev[dev];
  return DS_OK;
}

// Schedules chosen by ds_autotune, per batch signature; calls without an entry use the default.
static const ds_schedule kDefaultSchedule = {0, 5, 4, 0, 5, 5, 8, DS_ROUNDS, 1, 0, 0};
struct SchedKey {
  int nmodels, nb0, nv0, ncmax, precision, mode, bbucket;
  bool operator<(const SchedKey& o) const {
    const int x[7] = {nmodels, nb0, nv0, ncmax, precision, mode, bbucket};
    const int y[7] = {o.nmodels, o.nb0, o.nv0, o.ncmax, o.precision, o.mode, o.bbucket};
    for (int i = 0; i < 7; ++i)
      if (x[i] != y[i]) return x[i] < y[i];
    return false;
  }
};
static std::mutex g_sched_mu;
static std::map<SchedKey, ds_schedule> g_sched;

static SchedKey sched_key(const ds_model* const* models, int nmodels, const ds_batch* b, const ds_options* o,
                          int mode) {
  int bb = 0;
  while ((1 << bb) < b->B && bb < 30) ++bb;
  return SchedKey{nmodels, models[0]->host.nb, models[0]->host.nv, b->ncmax, o->precision, mode, bb};
}

static ds_schedule find_schedule(const SchedKey& k) {
  std::lock_guard<std::mutex> lock(g_sched_mu);
  auto it = g_sched.find(k);
  return it == g_sched.end() ? kDefaultSchedule : it->second;
}

// The whole step as one persistent launch (ds_schedule.persistent) when a persistent kernel with
// the shape of every model's fitted kernel is compiled; DS_EUNSUPPORTED (nothing launched) when not.
static ds_status run_persistent(const ds_model* const* models, int32_t nmodels, const ds_batch* b,
                                const ds_options* o, const ds_kernel_entry* const* kern, int fw_rows, void* ws,
                                KArgs a, cudaStream_t s) {
  const ds_persist_entry* pe = nmodels <= DS_PERSIST_MAXMODELS ? ds_persist_kernel(o->precision) : nullptr;
  if (!pe) return DS_EUNSUPPORTED;
  PArgs p;
  std::memset(&p, 0, sizeof(p));
  long long cost[DS_PERSIST_MAXMODELS];
  for (int k = 0; k < nmodels; ++k) {
    int found = -1;
    for (int i = 0; i < pe->nshapes && found < 0; ++i)
      if (pe->shape[i][0] == kern[k]->nb && pe->shape[i][1] == kern[k]->nv && pe->shape[i][2] == kern[k]->ns)
        found = i;
    if (found < 0) return DS_EUNSUPPORTED;
    p.model[k] = models[k]->dev;
    p.shape[k] = found;
    p.nv[k] = models[k]->host.nv;
    p.order[k] = k;
    cost[k] = (long long)kern[k]->nv * kern[k]->nv * (kern[k]->ns + 1);   // rough per-env cost
  }
  // the costliest model's chunks first, so that the cheap ones fill in at the end
  std::sort(p.order, p.order + nmodels, [&](int x, int y) { return cost[x] > cost[y] || (cost[x] == cost[y] && x < y); });
  ds_workspace_layout(b->ncmax, b->B, ws, &a.ws, nmodels, 0, fw_rows);
  p.nmodels = nmodels;
  p.poll_limit = o->queue_poll_limit;
  p.queue = a.ws.queue;
  p.lists = a.ws.qlists;
  a.model = nullptr;
  a.model_index = 0;
  a.model_id = b->model_id;
  a.env_list = nullptr;
  a.n_env = b->B;
  if (cudaMemsetAsync(p.queue, 0, sizeof(int32_t) * (DS_Q_COUNT + DS_PERSIST_MAXMODELS), s) != cudaSuccess)
    return DS_ECUDA;
  pe->launch(a, p, s);
  return cudaGetLastError() == cudaSuccess ? DS_OK : DS_ECUDA;
}

static ds_status run(const ds_model* const* models, int32_t nmodels, const ds_batch* b, const ds_options* o,
                     const ds_step_out* out, int mode, double* dq, double* dv, double* dtau, const double* vbar,
                     const double* qnbar, double* qb, double* vb, double* tb, void* ws, size_t ws_bytes,
                     void* stream, const ds_step_out* tape = nullptr) {
  if (!models || nmodels <= 0 || nmodels > 64 || !b || !o || !out) return DS_EINVAL;
  if (b->B < 0 || b->ncmax < 0 || b->ncmax > DS_MAXSLOTS) return DS_EINVAL;
  if (b->B == 0) return DS_OK;
  if (!out->v_next) return DS_EINVAL;
  if (!b->q || !b->v || !b->tau || !b->plane) return DS_EINVAL;
  if (b->ncmax > 0 && (!b->c_link || !b->c_point || !b->c_radius || !b->c_mu)) return DS_EINVAL;
  if (nmodels > 1 && !b->model_id) return DS_EINVAL;
  if (!(o->dt > 0.0) || o->admm_max_iter < 1 || o->polish_iters < 0 || !(o->admm_eps > 0.0) || !(o->ncp_tol > 0.0))
    return DS_EINVAL;
  if (o->precision != DS_FP64 && o->precision != DS_MIXED) return DS_EINVAL;
  if (!std::isfinite(o->baumgarte_kp) || !std::isfinite(o->baumgarte_kd)) return DS_EINVAL;
  if (!(o->contact_margin >= 0.0) || !std::isfinite(o->contact_margin)) return DS_EINVAL;
  if (o->ncp_solver != DS_ADMM && o->ncp_solver != DS_PGS) return DS_EINVAL;
  if (o->queue_poll_limit < 0) return DS_EINVAL;
  if (o->admm_rho_adapt != 0 && o->admm_rho_adapt != 1) return DS_EINVAL;
  if (mode == DS_RUN_JAC && (!dq || !dv || !dtau)) return DS_EINVAL;
  if (mode == DS_RUN_VJP && (!vbar || !qb || !vb || !tb)) return DS_EINVAL;
  const ds_kernel_entry* kern[64];
  int fw_rows = 0;
  for (int k = 0; k < nmodels; ++k) {
    if (!models[k]) return DS_EINVAL;
    const int slots = b->model_slots ? b->model_slots[k] : b->ncmax;
    if (slots < 0 || slots > b->ncmax) return DS_EINVAL;
    kern[k] = ds_fit_kernel(models[k]->host.nb, models[k]->host.nv, slots, b->ncmax, o->precision);
    if (!kern[k]) return DS_EUNSUPPORTED;
    const int r = std::max(ds_forward_rows(kern[k]->nb, kern[k]->nv, kern[k]->ns),
                           ds_colstate_rows(kern[k]->nb, kern[k]->nv, kern[k]->ns));
    if (r > fw_rows) fw_rows = r;
  }
  if (ws && (ws_bytes < ds_workspace_layout(b->ncmax, b->B, nullptr, nullptr, nmodels, 0, fw_rows) ||
             (reinterpret_cast<uintptr_t>(ws) & 255) != 0))
    return DS_EINVAL;
  KArgs a;
  std::memset(&a, 0, sizeof(a));
  a.B = b->B; a.ncmax = b->ncmax;
  a.q = b->q; a.v = b->v; a.tau = b->tau;
  a.c_link = b->c_link; a.c_point = b->c_point; a.c_radius = b->c_radius; a.c_mu = b->c_mu; a.plane = b->plane;
  a.dt = o->dt; a.gx = o->gravity[0]; a.gy = o->gravity[1]; a.gz = o->gravity[2];
  a.bkp = o->baumgarte_kp; a.bkd = o->baumgarte_kd; a.cmargin = o->contact_margin;
  a.solver = o->ncp_solver;
  a.rho_adapt = o->ncp_solver == DS_ADMM && o->admm_rho_adapt;
  a.admm_max_iter = o->admm_max_iter; a.polish_iters = o->polish_iters;
  a.admm_eps = o->admm_eps; a.ncp_tol = o->ncp_tol;
  a.eps_sigma = o->eps_sigma; a.eps_lambda = o->eps_lambda; a.margin_delta = o->margin_delta;
  a.v_next = out->v_next; a.q_next = out->q_next; a.lambda = out->lambda; a.modes = out->modes;
  a.status = out->env_status; a.iters = out->iters;
  a.dv_dq = dq; a.dv_dv = dv; a.dv_dtau = dtau;
  a.vbar = vbar; a.qnbar = qnbar; a.q_bar = qb; a.v_bar = vb; a.tau_bar = tb;
  a.run = mode;
  a.env_list = nullptr;
  a.n_env = b->B;
  a.model_id = nmodels > 1 ? b->model_id : nullptr;
  if (tape) {
    if ((b->ncmax > 0 && (!tape->lambda || !tape->modes)) || !tape->env_status) return DS_EINVAL;
    a.tlam = tape->lambda;
    a.tmodes = tape->modes;
    a.tstat = tape->env_status;
    cudaStream_t ts = static_cast<cudaStream_t>(stream);
    for (int k = 0; k < nmodels; ++k) {
      a.model = models[k]->dev;
      a.model_index = k;
      kern[k]->tape(a, ts);
      if (cudaGetLastError() != cudaSuccess) return DS_ECUDA;
    }
    return DS_OK;
  }
  a.sched = g_force_sched ? *g_force_sched : find_schedule(sched_key(models, nmodels, b, o, mode));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (ws && a.sched.persistent) {
    const ds_status r = run_persistent(models, nmodels, b, o, kern, fw_rows, ws, a, s);
    if (r != DS_EUNSUPPORTED) return r;
  }
  HelperStreams* hs = nullptr;
  if (ws && g_allow_helpers && helper_streams(&hs) != DS_OK) return DS_ECUDA;
  a.side = nullptr;
  if (ws && hs && nmodels > 1) {
    // Each model's pipeline on a helper stream of its own (fork / join with events on the caller's
    // stream): the models' kernels are small and overlap on the GPU.
    if (cudaEventRecord(hs->fork, s) != cudaSuccess) return DS_ECUDA;
    for (int k = 0; k < nmodels; ++k) {
      cudaStream_t sk = hs->s[k % kHelperStreams];
      if (cudaStreamWaitEvent(sk, hs->fork, 0) != cudaSuccess) return DS_ECUDA;
      ds_workspace_layout(b->ncmax, b->B, ws, &a.ws, nmodels, k, fw_rows);
      a.model = models[k]->dev;
      a.model_index = k;
      a.side = hs->s[kHelperStreams + k % kHelperStreams];
      a.ev_fork = hs->side_fork[k % kHelperStreams];
      a.ev_join = hs->side_join[k % kHelperStreams];
      kern[k]->pipeline(a, sk);
      if (cudaGetLastError() != cudaSuccess) return DS_ECUDA;
    }
    for (int j = 0; j < kHelperStreams && j < nmodels; ++j) {
      if (cudaEventRecord(hs->join[j], hs->s[j]) != cudaSuccess) return DS_ECUDA;
      if (cudaStreamWaitEvent(s, hs->join[j], 0) != cudaSuccess) return DS_ECUDA;
    }
    return DS_OK;
  }
  if (hs) {
    a.side = hs->s[kHelperStreams];
    a.ev_fork = hs->side_fork[0];
    a.ev_join = hs->side_join[0];
  }
  for (int k = 0; k < nmodels; ++k) {
    const ds_kernel_entry* ke = kern[k];
    if (ws) ds_workspace_layout(b->ncmax, b->B, ws, &a.ws, nmodels, k, fw_rows);
    a.model = models[k]->dev;
    a.model_index = k;
    if (ws) ke->pipeline(a, s);
    else ke->fn(a, s);
    if (cudaGetLastError() != cudaSuccess) return DS_ECUDA;
  }
  return DS_OK;
}

extern "C" ds_status sim_step(const ds_model* const* models, int32_t nmodels, const ds_batch* batch,
                              const ds_options* opt, const ds_step_out* out, void* ws, size_t ws_bytes,
                              void* stream) {
  return run(models, nmodels, batch, opt, out, DS_RUN_STEP, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
             nullptr, nullptr, ws, ws_bytes, stream);
}

extern "C" ds_status sim_step_jac(const ds_model* const* models, int32_t nmodels, const ds_batch* batch,
                                  const ds_options* opt, const ds_step_out* out, double* dv_dq, double* dv_dv,
                                  double* dv_dtau, void* ws, size_t ws_bytes, void* stream) {
  return run(models, nmodels, batch, opt, out, DS_RUN_JAC, dv_dq, dv_dv, dv_dtau, nullptr, nullptr, nullptr,
             nullptr, nullptr, ws, ws_bytes, stream);
}

extern "C" ds_status sim_step_vjp_tape(const ds_model* const* models, int32_t nmodels, const ds_batch* batch,
                                       const ds_options* opt, const double* v_next_bar, const double* q_next_bar,
                                       const ds_step_out* tape, const ds_step_out* out, double* q_bar, double* v_bar,
                                       double* tau_bar, void* stream) {
  if (!tape) return DS_EINVAL;
  return run(models, nmodels, batch, opt, out, DS_RUN_VJP, nullptr, nullptr, nullptr, v_next_bar, q_next_bar, q_bar,
             v_bar, tau_bar, nullptr, 0, stream, tape);
}

extern "C" ds_status sim_step_vjp(const ds_model* const* models, int32_t nmodels, const ds_batch* batch,
                                  const ds_options* opt, const double* v_next_bar, const double* q_next_bar,
                                  const ds_step_out* out, double* q_bar, double* v_bar, double* tau_bar, void* ws,
                                  size_t ws_bytes, void* stream) {
  return run(models, nmodels, batch, opt, out, DS_RUN_VJP, nullptr, nullptr, nullptr, v_next_bar, q_next_bar, q_bar,
             v_bar, tau_bar, ws, ws_bytes, stream);
}

// ------------------------------------------------------------------ cotangent coordinate maps
// Between a cotangent of the raw configuration vector (nq numbers per env: the free-flyer's
// position and quaternion) and one of its tangent coordinates at q (nv numbers), for the
// perturbation q (+) eta used by the derivatives (position += R eta_lin, quaternion <- quaternion
// * exp(eta_ang / 2)).  With Q(quat) the matrix of left quaternion multiplication and c1, c2, c3
// its last three columns, d q_raw / d eta = [R, 0; 0, Q(quat)[:, 1:4] / 2] and (unit quaternion)
// d eta / d q_raw = [R^T, 0; 0, 2 Q(quat)^T[1:4, :]]; revolute rows are the identity.
// to_tangent: out = (d q_raw / d eta)^T in; to_raw: out = (d eta / d q_raw)^T in.
__global__ void cotangent_kernel(const DevModel* __restrict__ m, int model_index, const int32_t* model_id, int B,
                                 const double* __restrict__ q, const double* __restrict__ in,
                                 double* __restrict__ out, int to_raw) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= B) return;
  if (model_id && model_id[e] != model_index) return;
  const int nb = m->nb;
  for (int i = 0; i < nb; ++i) {
    const int k0 = m->iq[i], d0 = m->iv[i];
    if (m->jtype[i] == 0) {
      if (to_raw) out[k0 * B + e] = in[d0 * B + e];
      else out[d0 * B + e] = in[k0 * B + e];
      continue;
    }
    double w = q[(k0 + 3) * B + e], x = q[(k0 + 4) * B + e], y = q[(k0 + 5) * B + e], z = q[(k0 + 6) * B + e];
    const double inv = 1.0 / sqrt(w * w + x * x + y * y + z * z);
    w *= inv; x *= inv; y *= inv; z *= inv;
    const double R[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                         2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                         2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)};
    const double c[3][4] = {{-x, w, z, -y}, {-y, -z, w, x}, {-z, y, -x, w}};
    if (to_raw) {
      const double el[3] = {in[d0 * B + e], in[(d0 + 1) * B + e], in[(d0 + 2) * B + e]};
      const double ea[3] = {in[(d0 + 3) * B + e], in[(d0 + 4) * B + e], in[(d0 + 5) * B + e]};
      for (int r = 0; r < 3; ++r) out[(k0 + r) * B + e] = R[3 * r] * el[0] + R[3 * r + 1] * el[1] + R[3 * r + 2] * el[2];
      for (int r = 0; r < 4; ++r) out[(k0 + 3 + r) * B + e] = 2.0 * (c[0][r] * ea[0] + c[1][r] * ea[1] + c[2][r] * ea[2]);
    } else {
      const double pb[3] = {in[k0 * B + e], in[(k0 + 1) * B + e], in[(k0 + 2) * B + e]};
      const double qb[4] = {in[(k0 + 3) * B + e], in[(k0 + 4) * B + e], in[(k0 + 5) * B + e], in[(k0 + 6) * B + e]};
      for (int r = 0; r < 3; ++r) out[(d0 + r) * B + e] = R[r] * pb[0] + R[3 + r] * pb[1] + R[6 + r] * pb[2];
      for (int r = 0; r < 3; ++r)
        out[(d0 + 3 + r) * B + e] = 0.5 * (c[r][0] * qb[0] + c[r][1] * qb[1] + c[r][2] * qb[2] + c[r][3] * qb[3]);
    }
  }
}

static ds_status cotangent(const ds_model* const* models, int32_t nmodels, int32_t B, const int32_t* model_id,
                           const double* q, const double* in, double* out, int to_raw, void* stream) {
  if (!models || nmodels <= 0 || nmodels > 64 || B < 0) return DS_EINVAL;
  if (B == 0) return DS_OK;
  if (!q || !in || !out || (nmodels > 1 && !model_id)) return DS_EINVAL;
  for (int k = 0; k < nmodels; ++k)
    if (!models[k]) return DS_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int k = 0; k < nmodels; ++k) {
    cotangent_kernel<<<(B + 127) / 128, 128, 0, s>>>(models[k]->dev, k, nmodels > 1 ? model_id : nullptr, B, q, in,
                                                     out, to_raw);
    if (cudaGetLastError() != cudaSuccess) return DS_ECUDA;
  }
  return DS_OK;
}

extern "C" ds_status ds_cotangent_to_tangent(const ds_model* const* models, int32_t nmodels, int32_t B,
                                             const int32_t* model_id, const double* q, const double* q_bar_raw,
                                             double* q_bar_tangent, void* stream) {
  return cotangent(models, nmodels, B, model_id, q, q_bar_raw, q_bar_tangent, 0, stream);
}

// Schedule knobs and their options.  The index of ds_autotune / ds_set_schedule is the mixed-radix
// number of the chosen option positions, knob 0 the lowest digit.
static const int kKnobs = 11, kNumSchedules = 3 * 3 * 3 * 2 * 5 * 3 * 3 * 3 * 2 * 2 * 2;
static const int kNopt[kKnobs] = {3, 3, 3, 2, 5, 3, 3, 3, 2, 2, 2};
static const int kOpt[kKnobs][5] = {{0, 1, 2, 0},          // round-cap table
                                    {3, 5, DS_ROUNDS, 0},  // first row-per-lane ADMM round
                                    {0, 4, 8, 0},          // finish: target CTAs per SM
                                    {0, 1, 0, 0},          // Newton: cooperative / one thread per env
                                    {-1, 2, 4, 5, DS_ROUNDS},  // overlapped finish after this round (-1: setup)
                                    {3, 5, DS_ROUNDS, 0},  // first two-warp ADMM round
                                    {0, 8, 4, 0},          // overlapped finish: SM stride kept free
                                    {3, 5, DS_ROUNDS, 0},  // speculative Newton attempts from round
                                    {1, 0, 0, 0},          // single-contact presolve: on / off
                                    {0, 1, 0, 0},          // workspace pipeline / persistent launch
                                    {0, 1, 0, 0}};         // finish: one kernel / prep + column kernels
static int* knob(ds_schedule& c, int d) {
  switch (d) {
    case 0: return &c.caps;
    case 1: return &c.wide_from;
    case 2: return &c.finish_ctas;
    case 3: return &c.newton_thread;
    case 4: return &c.overlap_from;
    case 5: return &c.pair_from;
    case 6: return &c.reserve;
    case 7: return &c.spec_from;
    case 8: return &c.presolve;
    case 9: return &c.persistent;
    default: return &c.finish_split;
  }
}
static int schedule_index(ds_schedule c) {
  int idx = 0, mul = 1;
  for (int d = 0; d < kKnobs; ++d) {
    int pos = 0;
    for (int o = 0; o < kNopt[d]; ++o)
      if (kOpt[d][o] == *knob(c, d)) { pos = o; break; }
    idx += pos * mul;
    mul *= kNopt[d];
  }
  return idx;
}
static ds_schedule schedule_from_index(int i) {
  ds_schedule c;
  for (int d = 0; d < kKnobs; ++d) {
    *knob(c, d) = kOpt[d][i % kNopt[d]];
    i /= kNopt[d];
  }
  return c;
}

extern "C" ds_status ds_set_schedule(const ds_model* const* models, int32_t nmodels, const ds_batch* batch,
                                     const ds_options* opt, int32_t mode, int32_t index) {
  if (!models || nmodels <= 0 || nmodels > 64 || !batch || !opt || batch->B <= 0) return DS_EINVAL;
  if (mode < DS_RUN_STEP || mode > DS_RUN_VJP || index < -1 || index >= kNumSchedules) return DS_EINVAL;
  for (int k = 0; k < nmodels; ++k)
    if (!models[k]) return DS_EINVAL;
  const SchedKey key = sched_key(models, nmodels, batch, opt, mode);
  std::lock_guard<std::mutex> lock(g_sched_mu);
  if (index < 0) g_sched.erase(key);
  else g_sched[key] = schedule_from_index(index);
  return DS_OK;
}

extern "C" ds_status ds_cotangent_to_raw(const ds_model* const* models, int32_t nmodels, int32_t B,
                                         const int32_t* model_id, const double* q, const double* q_bar_tangent,
                                         double* q_bar_raw, void* stream) {
  return cotangent(models, nmodels, B, model_id, q, q_bar_tangent, q_bar_raw, 1, stream);
}

// ------------------------------------------------------------------------------ autotuning
extern "C" ds_status ds_autotune(const ds_model* const* models, int32_t nmodels, const ds_batch* batch,
                                 const ds_options* opt, int32_t mode, const double* v_next_bar,
                                 const ds_step_out* out, double* o0, double* o1, double* o2, void* ws,
                                 size_t ws_bytes, void* stream, int32_t* chosen) {
  if (!models || nmodels <= 0 || nmodels > 64 || !batch || !opt || !out || !ws) return DS_EINVAL;
  if (mode < DS_RUN_STEP || mode > DS_RUN_VJP) return DS_EINVAL;
  for (int k = 0; k < nmodels; ++k)
    if (!models[k]) return DS_EINVAL;
  if (batch->B <= 0) return DS_EINVAL;
  static std::mutex tune_mu;
  std::lock_guard<std::mutex> lock(tune_mu);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  auto call = [&]() -> ds_status {
    if (mode == DS_RUN_STEP) return sim_step(models, nmodels, batch, opt, out, ws, ws_bytes, stream);
    if (mode == DS_RUN_JAC) return sim_step_jac(models, nmodels, batch, opt, out, o0, o1, o2, ws, ws_bytes, stream);
    return sim_step_vjp(models, nmodels, batch, opt, v_next_bar, nullptr, out, o0, o1, o2, ws, ws_bytes, stream);
  };
  // Coordinate search from the default: each knob in turn over its options, the others held at
  // the best found so far; two passes, since some knobs pay only together (the two-warp ADMM
  // rounds and the SMs kept free of the overlapped finish).
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return DS_ECUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return DS_ECUDA; }
  ds_schedule best = kDefaultSchedule;
  ds_status st = DS_OK;
  // Each timed run starts with a cold L2 (a 256 MB scratch buffer is written before it, outside
  // the timed region), as a step of a real loop would.  A candidate's time is the second slowest
  // of five runs: some schedules (an overlapped finish on a batch with no ADMM tail) run fast or
  // slow from one step to the next, and a schedule has to be fast in most steps to be chosen.
  void* flush = nullptr;
  const size_t flush_bytes = size_t(256) << 20;
  if (cudaMalloc(&flush, flush_bytes) != cudaSuccess) {
    flush = nullptr;
    cudaGetLastError();
  }
  auto timed = [&](const ds_schedule& c, float* ms_out) -> ds_status {
    g_force_sched = &c;
    ds_status r = call();                                 // untimed
    float ms5[5];
    int n = 0;
    for (int k = 0; k < 5 && r == DS_OK; ++k) {
      if (flush) cudaMemsetAsync(flush, k, flush_bytes, s);
      cudaEventRecord(e0, s);
      r = call();
      cudaEventRecord(e1, s);
      float ms = 0.f;
      if (r == DS_OK && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
        r = DS_ECUDA;
      if (r == DS_OK) ms5[n++] = ms;
    }
    g_force_sched = nullptr;
    std::sort(ms5, ms5 + n);
    *ms_out = n > 0 ? ms5[n >= 2 ? n - 2 : 0] : 1e30f;
    return r;
  };
  float best_ms = 0.f;
  st = timed(best, &best_ms);
  for (int pass = 0; pass < 2 && st == DS_OK; ++pass)
    for (int d = 0; d < kKnobs && st == DS_OK; ++d)
      for (int o = 0; o < kNopt[d] && st == DS_OK; ++o) {
        ds_schedule c = best;
        int* field = knob(c, d);
        if (*field == kOpt[d][o]) continue;
        *field = kOpt[d][o];
        float ms = 0.f;
        st = timed(c, &ms);
        if (st == DS_OK && ms < 0.98f * best_ms) { best_ms = ms; best = c; }   // 2 % to switch: noise
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (flush) {
    cudaStreamSynchronize(s);
    cudaFree(flush);
  }
  if (st != DS_OK) return st;
  {
    std::lock_guard<std::mutex> l2(g_sched_mu);
    g_sched[sched_key(models, nmodels, batch, opt, mode)] = best;
  }
  if (chosen) *chosen = schedule_index(best);
  return call();                                          // leave the outputs of the chosen schedule
}

// ---------------------------------------------------------------------------- checked build
#ifdef DS_CHECK
static __global__ void ds_check_probe_kernel(int i, int n) { (void)DS_IX(i, n); }
#endif

extern "C" ds_status ds_check_bad_indices(uint64_t* count) {
  if (!count) return DS_EINVAL;
#ifdef DS_CHECK
  if (cudaDeviceSynchronize() != cudaSuccess) return DS_ECUDA;
  *count = ds_check_sum();
  return DS_OK;
#else
  *count = 0;
  return DS_EUNSUPPORTED;
#endif
}

extern "C" ds_status ds_check_self_test(int32_t index, int32_t n, uint64_t* count) {
  if (!count || n <= 0) return DS_EINVAL;
#ifdef DS_CHECK
  unsigned z = 0, v = 0;
  if (cudaMemcpyToSymbol(ds_check_bad, &z, sizeof z) != cudaSuccess) return DS_ECUDA;
  ds_check_probe_kernel<<<1, 1>>>(index, n);
  if (cudaDeviceSynchronize() != cudaSuccess) return DS_ECUDA;
  if (cudaMemcpyFromSymbol(&v, ds_check_bad, sizeof v) != cudaSuccess) return DS_ECUDA;
  *count = v;
  return DS_OK;
#else
  (void)index;
  *count = 0;
  return DS_EUNSUPPORTED;
#endif
}
