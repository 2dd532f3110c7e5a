// Persistent launch over a batch that mixes models: one kernel for the whole step, its envs pulled
// from an atomic work queue.
//
// The grid is sized to the CTAs the GPU keeps resident at once.  Every CTA first files its slice
// of the env indices into one list per model (warp-aggregated atomics), presets those envs'
// status to DS_ENV_QUEUE_TIMEOUT and their v+ to NaN, and counts itself done.  Work items are
// chunks of 32 envs of one model, numbered model after model in the order the host gives (the
// costliest first, so that the cheap chunks fill the gaps at the end); a chunk can only be
// decoded once every list is complete, so each CTA then polls the done count.  That poll is
// bounded: after queue_poll_limit polls the CTA gives up, raises the queue's abandon flag and
// counts a timeout; every CTA stops claiming work once the flag is up, and the envs nobody
// processed keep the preset status and NaN.  A warp claims one chunk at a time and runs one env
// per lane: F1-F9 and the requested derivatives of the fused per-env path, with the model's own
// compiled shape, so that an env's results are those of the fused kernel for its model.
#pragma once
#include "ds_launch.cuh"

namespace ds {

template <int NB_, int NV_, int NS_>
struct PShape {
  static constexpr int NB = NB_, NV = NV_, NS = NS_;
};

DS_HDI int ld_acquire(const int32_t* p) {
#ifdef __CUDA_ARCH__
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
#else
  return *p;
#endif
}

// One env on this thread: the fused per-env path for one shape, in three out-of-line steps
// (forward pass; NCP solve and classification; finish), so that the kernel's stack is the largest
// shape's frame rather than the sum of all of them.  The steps are defined only in the units that
// define DS_PERSIST_PART (relocatable device code, one shape or one step per unit, so that they
// compile in parallel: each shape's path is a large function) and explicitly instantiated there;
// the kernel's unit sees declarations, and the device link resolves the calls.
template <int NB, int NV, int NS, typename T>
__device__ uint32_t persist_forward(const DevModel& m, const KArgs& a, int e, Env<NB, NV, NS, T>& s);
template <int NB, int NV, int NS, typename T>
__device__ int persist_solve(const KArgs& a, Env<NB, NV, NS, T>& s, uint32_t& st);
template <int NB, int NV, int NS, typename T>
__device__ void persist_finish(const DevModel& m, const KArgs& a, int e, Env<NB, NV, NS, T>& s, uint32_t st,
                               int iters);

#ifdef DS_PERSIST_PART
template <int NB, int NV, int NS, typename T>
__device__ __noinline__ uint32_t persist_forward(const DevModel& m, const KArgs& a, int e, Env<NB, NV, NS, T>& s) {
  return env_forward<NB, NV, NS, T>(m, a, e, s);
}

template <int NB, int NV, int NS, typename T>
__device__ __noinline__ int persist_solve(const KArgs& a, Env<NB, NV, NS, T>& s, uint32_t& st) {
  const int mdim = 3 * s.na;
  int iters = 0;
  for (int r = 0; r < mdim; ++r) s.lam[r] = 0.0;
  if (mdim > 0 && !(st & DS_ENV_NONFINITE)) solve_ncp<Env<NB, NV, NS, T>, T>(s, a, iters, st);
  s.margin = classify(s, s.lam, a.eps_sigma, a.eps_lambda, s.mode);
  if (mdim > 0 && s.margin < a.margin_delta) st |= DS_ENV_NEAR_SWITCH;
  return iters;
}

template <int NB, int NV, int NS, typename T>
__device__ __noinline__ void persist_finish(const DevModel& m, const KArgs& a, int e, Env<NB, NV, NS, T>& s,
                                            uint32_t st, int iters) {
  env_finish<NB, NV, NS, T>(m, a, e, s, st, iters);
}

#define DS_PERSIST_FORWARD(NB, NV, NS, T) \
  template __device__ uint32_t persist_forward<NB, NV, NS, T>(const DevModel&, const KArgs&, int, Env<NB, NV, NS, T>&);
#define DS_PERSIST_SOLVE(NB, NV, NS, T) \
  template __device__ int persist_solve<NB, NV, NS, T>(const KArgs&, Env<NB, NV, NS, T>&, uint32_t&);
#define DS_PERSIST_FINISH(NB, NV, NS, T)                                                                   \
  template __device__ void persist_finish<NB, NV, NS, T>(const DevModel&, const KArgs&, int, Env<NB, NV, NS, T>&, \
                                                         uint32_t, int);
#endif

// The steps of run_env, in its order.
template <int NB, int NV, int NS, typename T>
__device__ __noinline__ void persist_run(const DevModel& m, const KArgs& a, int e) {
  Env<NB, NV, NS, T> s;
  uint32_t st = persist_forward<NB, NV, NS, T>(m, a, e, s);
  const int iters = persist_solve<NB, NV, NS, T>(a, s, st);
  persist_finish<NB, NV, NS, T>(m, a, e, s, st, iters);
}

// Dispatch to shape index sh of the list S...
template <typename T, int I>
__device__ __forceinline__ void persist_env_at(const DevModel&, const KArgs&, int, int) {}

template <typename T, int I, class S, class... Rest>
__device__ __forceinline__ void persist_env_at(const DevModel& m, const KArgs& a, int e, int sh) {
  if (sh == I) persist_run<S::NB, S::NV, S::NS, T>(m, a, e);
  else persist_env_at<T, I + 1, Rest...>(m, a, e, sh);
}

template <typename T, class... S>
__global__ void __launch_bounds__(128, 4) persist_kernel(KArgs a, PArgs p) {
#ifdef __CUDA_ARCH__
  __shared__ DevModel sm[DS_PERSIST_MAXMODELS];
  __shared__ int go;
  for (int k = 0; k < p.nmodels; ++k) {
    const int* src = reinterpret_cast<const int*>(p.model[k]);
    int* dst = reinterpret_cast<int*>(&sm[k]);
    for (int i = threadIdx.x; i < int(sizeof(DevModel) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
  }
  int32_t* q = p.queue;
  int32_t* cnt = q + DS_Q_COUNT;
  const int B = a.B;
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  // ---- partition: this CTA's slice of the env indices into the per-model lists
  const int per = (B + gridDim.x - 1) / gridDim.x;
  const int lo = blockIdx.x * per;
  const int hi = min(B, lo + per);
  for (int base = lo; base < hi; base += blockDim.x) {   // every warp of the CTA runs the same trips
    const int e = base + int(threadIdx.x);
    int k = -1;
    if (e < hi) {
      const int id = a.model_id ? a.model_id[e] : 0;
      if (id >= 0 && id < p.nmodels) {
        k = id;
        if (a.status) a.status[e] = DS_ENV_QUEUE_TIMEOUT;
        a.v_next[e] = __longlong_as_double(0x7ff8000000000000LL);
        for (int i = 1; i < p.nv[k]; ++i) a.v_next[i * B + e] = __longlong_as_double(0x7ff8000000000000LL);
      }
    }
    for (int j = 0; j < p.nmodels; ++j) {
      const unsigned mask = __ballot_sync(0xffffffffu, k == j);
      if (!mask) continue;
      const int leader = __ffs(mask) - 1;
      int pos = 0;
      if (lane == leader) pos = atomicAdd(&cnt[j], __popc(mask));
      pos = __shfl_sync(0xffffffffu, pos, leader);
      if (k == j) p.lists[size_t(j) * B + pos + __popc(mask & lt)] = e;
    }
  }
  __threadfence();
  __syncthreads();
  // ---- wait until every CTA has filed its slice (bounded)
  if (threadIdx.x == 0) {
    atomicAdd(&q[DS_Q_PARTED], 1);
    int ok = 0;
    for (int it = 0;; ++it) {
      if (ld_acquire(&q[DS_Q_PARTED]) >= int(gridDim.x)) { ok = 1; break; }
      if (ld_acquire(&q[DS_Q_ABANDON])) break;
      if (it >= p.poll_limit) {
        atomicExch(&q[DS_Q_ABANDON], 1);
        atomicAdd(&q[DS_Q_TIMEOUTS], 1);
        break;
      }
      __nanosleep(256);
    }
    __threadfence();
    go = ok;
  }
  __syncthreads();
  if (!go) return;
  // ---- chunks of 32 envs, model after model in p.order
  int nch[DS_PERSIST_MAXMODELS], len[DS_PERSIST_MAXMODELS];
  int total = 0;
  for (int j = 0; j < p.nmodels; ++j) {
    len[j] = ld_acquire(&cnt[p.order[j]]);
    nch[j] = (len[j] + 31) / 32;
    total += nch[j];
  }
  for (;;) {
    int t = 0;
    if (lane == 0) t = ld_acquire(&q[DS_Q_ABANDON]) ? total : atomicAdd(&q[DS_Q_NEXT], 1);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= total) break;
    int j = 0;
    while (t >= nch[j]) { t -= nch[j]; ++j; }
    const int k = p.order[j];
    const int i = t * 32 + lane;
    if (i < len[j]) {
      const int e = DS_IX(p.lists[size_t(k) * B + i], B);
      persist_env_at<T, 0, S...>(sm[k], a, e, p.shape[k]);
    }
  }
#endif
}

// Launcher of the persistent kernel over shapes S...: grid = the CTAs resident at once on this GPU
// (at most one per 128 envs).
template <typename T, class... S>
void launch_persist(const KArgs& a, const PArgs& p, cudaStream_t s) {
  static_assert(sizeof...(S) <= DS_PERSIST_MAXMODELS, "too many shapes");
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persist_kernel<T, S...>, 128, 0);
  if (per_sm <= 0) per_sm = 1;
  int g = per_sm * ds_sm_count();
  const int need = (a.B + 127) / 128;
  if (g > need) g = need;
  if (g < 1) g = 1;
  ds_trace_mark(DS_STAGE_FUSED, 1, s);
  persist_kernel<T, S...><<<g, 128, 0, s>>>(a, p);
  ds_trace_mark(DS_STAGE_FUSED, 0, s);
}

template <typename T, class... S>
ds_persist_entry persist_entry(int precision, ds_persist_fn fn, unsigned (*check)()) {
  ds_persist_entry r;
  r.precision = precision;
  r.nshapes = int(sizeof...(S));
  const int nb[] = {S::NB...}, nv[] = {S::NV...}, ns[] = {S::NS...};
  for (int i = 0; i < r.nshapes; ++i) { r.shape[i][0] = nb[i]; r.shape[i][1] = nv[i]; r.shape[i][2] = ns[i]; }
  r.launch = fn;
  r.check = check;
  return r;
}

}  // namespace ds
