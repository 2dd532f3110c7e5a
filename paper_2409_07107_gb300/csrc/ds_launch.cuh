// Host launchers of the fused kernel and of the workspace pipeline (setup, compacted ADMM rounds
// with their Newton stages, finish).
#pragma once
#include "ds_newton_coop.cuh"

namespace ds {

// Reads and clears this translation unit's bad-index count (the checked build; 0 otherwise).
inline unsigned check_read() {
#ifdef DS_CHECK
  unsigned v = 0, z = 0;
  if (cudaMemcpyFromSymbol(&v, ds_check_bad, sizeof v) != cudaSuccess) return 0xffffffffu;
  cudaMemcpyToSymbol(ds_check_bad, &z, sizeof z);
  return v;
#else
  return 0;
#endif
}

inline int ds_sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

template <int NB, int NV, int NS, typename T>
void launch_env(const KArgs& a, cudaStream_t s) {
  const int threads = 128;
  const int blocks = (a.n_env + threads - 1) / threads;
  if (blocks <= 0) return;
  ds_trace_mark(DS_STAGE_FUSED, 1, s);
  env_kernel<NB, NV, NS, T><<<blocks, threads, 0, s>>>(a);
  ds_trace_mark(DS_STAGE_FUSED, 0, s);
}

// Blocks for n envs x nchunk work items (the finish kernel loops over the rest).
inline int finish_blocks(int n, int nchunk, int threads) {
  const long long b = ((long long)n * nchunk + threads - 1) / threads;
  return int(b < (1 << 20) ? (b > 0 ? b : 1) : (1 << 20));
}

// The split finish (schedule finish_split) over the envs of fa (its range flo/fhi, or all): the
// prep kernel (CTAs of one warp), then the column kernel with up to 4 envs per CTA as fit in
// 200 KB of shared memory (at least one), ColsShape::WPE warps per env, CTAs for the SMs'
// resident capacity.
template <int NB, int NV, int NS, typename T>
void launch_finish_split(const KArgs& fa, cudaStream_t s) {
  // prep threads per env (Jacobians): enough to fill the SMs' 16 resident warps (128 registers a
  // thread), a power of two with at least 8 rows of P each (every thread holds its own copy of the
  // env's state, so more of them cost local-memory traffic: measured, 8 threads per env slowed the
  // quadruped's prep at 8192 envs and sped the humanoid's at 4096)
  KArgs pa = fa;
  pa.nchunk = 1;
  if (fa.run == DS_RUN_JAC) {
    const int want = fa.n_env > 0 ? (ds_sm_count() * 16 * 32) / fa.n_env : 1;
    int cap = 1;
    while (cap * 2 * 8 <= NV && cap < 8) cap *= 2;
    int c = want >= 8 ? 8 : (want >= 4 ? 4 : (want >= 2 ? 2 : 1));
    pa.nchunk = c < cap ? c : cap;
  }
  const long long items = (long long)fa.n_env * pa.nchunk;
  const int pblocks = int((items + 31) / 32);
  if (pblocks <= 0) return;
  ds_trace_mark(DS_STAGE_FINISH, 1, s);
  finish_prep_kernel<NB, NV, NS, T><<<pblocks, 32, 0, s>>>(pa);
  constexpr size_t cs_bytes = sizeof(ColState<NB, NV, NS, T>);
  constexpr int epb = cs_bytes * 4 <= 200 * 1024 ? 4 : (cs_bytes * 2 <= 200 * 1024 ? 2 : 1);
  constexpr int cthreads = 32 * ColsShape<NV>::WPE * epb;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(finish_cols_kernel<NB, NV, NS, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         int(epb * cs_bytes));
    attr = true;
  }
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, finish_cols_kernel<NB, NV, NS, T>, cthreads, epb * cs_bytes);
  if (per_sm <= 0) per_sm = 1;
  int cblocks = ds_sm_count() * per_sm;
  const int need = (fa.n_env + epb - 1) / epb;
  if (cblocks > need) cblocks = need;
  finish_cols_kernel<NB, NV, NS, T><<<cblocks, cthreads, epb * cs_bytes, s>>>(fa);
  ds_trace_mark(DS_STAGE_FINISH, 0, s);
}

template <int NB, int NV, int NS, typename T>
void launch_pipeline(const KArgs& a0, cudaStream_t s) {
  const int threads = 128;
  const int blocks = (a0.n_env + threads - 1) / threads;
  if (blocks <= 0) return;
  cudaMemsetAsync(a0.ws.counts, 0, sizeof(int32_t) * (DS_ROUNDS + 1), s);
  cudaMemsetAsync(a0.ws.ncounts, 0, sizeof(int32_t) * (2 * DS_ROUNDS + 3), s);   // ncounts, fetch, dcount, claim
  ds_trace_mark(DS_STAGE_SETUP, 1, s);
  setup_kernel<NB, NV, NS, T><<<blocks, threads, 0, s>>>(a0);
  ds_trace_mark(DS_STAGE_SETUP, 0, s);
  // Round caps (ADMM iterations an env may run per round before regrouping and, with speculative
  // attempts, before the Newton stage tries its iterate); the last round runs to the iteration limit.
  const ds_schedule sc = a0.sched;
  const int table = (sc.caps >= 0 && sc.caps < 3) ? sc.caps : 0;
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, admm_round_kernel<NS, T>, threads, 0);
  if (per_sm <= 0) per_sm = 1;
  const int envs_per_block = threads / NS;
  int rblocks = ds_sm_count() * per_sm;
  const int need = (a0.n_env + envs_per_block - 1) / envs_per_block;
  if (rblocks > need) rblocks = need;
  // the PGS round kernel (ncp_solver = DS_PGS): one thread per env
  int gper = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&gper, pgs_round_kernel<NS, T>, threads, 0);
  if (gper <= 0) gper = 1;
  int gblocks = ds_sm_count() * gper;
  if (gblocks > blocks) gblocks = blocks;
  // the row-per-lane ADMM kernel for the late rounds (where the schedule says so and 3 NS <= 32)
  constexpr bool kWideOk = WideShape<NS>::kOk;
  int wblocks = 1;
  if constexpr (kWideOk) {
    int wper = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&wper, admm_round_wide_kernel<NS, T>, threads, 0);
    if (wper <= 0) wper = 1;
    const int wenvs = threads / WideShape<NS>::L;
    wblocks = ds_sm_count() * wper;
    const int wneed = (a0.n_env + wenvs - 1) / wenvs;
    if (wblocks > wneed) wblocks = wneed;
  }
  // the two-warp ADMM kernel (FP64; 64-thread CTAs, 32 / L envs each) from the schedule's round
  constexpr bool kPairOk = kWideOk && std::is_same<T, double>::value;
  int pblocks = 1;
  if constexpr (kPairOk) {
    int pper = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pper, admm_round_pair_kernel<NS, T>, 64, 0);
    if (pper <= 0) pper = 1;
    const int penvs = PairShape<NS>::EPW;
    pblocks = ds_sm_count() * pper;
    const int pneed = (a0.n_env + penvs - 1) / penvs;
    if (pblocks > pneed) pblocks = pneed;
  }
  // Newton stage: the cooperative kernel (4 NS lanes per env) where 4 NS divides the warp, else
  // one thread per env.
  // (the schedule may ask for the one-thread form instead).
  constexpr bool kCoopOk = 32 % (4 * NS) == 0;
  const bool coop = kCoopOk && !sc.newton_thread;
  const int nthreads = coop ? coop::Shape<kCoopOk ? NS : 1>::THREADS : threads;
  const int envs_per_nblock = coop ? nthreads / (4 * NS) : nthreads;
  int nper = 0;
  if constexpr (kCoopOk) {
    if (coop) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nper, newton_coop_kernel<NS, T>, nthreads, 0);
  }
  if (!coop) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nper, newton_kernel<NS, T>, nthreads, 0);
  if (nper <= 0) nper = 1;
  int nblocks = ds_sm_count() * nper;
  const int nneed = (a0.n_env + envs_per_nblock - 1) / envs_per_nblock;
  if (nblocks > nneed) nblocks = nneed;
  // Finish: with a small batch the Jacobian columns (VJP dof passes) of an env are split over
  // several threads, each recomputing the env's forward pass, so that the launch still fills the
  // GPU (by default about 4 CTAs of 128 threads per SM); large batches keep one thread per env.
  KArgs af = a0;
  af.nchunk = 1;
  const int maxc = a0.run == DS_RUN_JAC ? 3 * NV : 2 * NV;
  if (a0.run != DS_RUN_STEP && sc.finish_ctas > 0) {
    const int target = ds_sm_count() * sc.finish_ctas * threads;
    int c = target / (a0.n_env > 0 ? a0.n_env : 1);
    af.nchunk = c < 1 ? 1 : (c > maxc ? maxc : c);
  }
  // With a side stream and an overlap round, the envs solved by then are finished on the side
  // stream while the later ADMM rounds run; the rest are finished at the end.  Overlap round -1:
  // right after the setup (the envs it solved: no contact, separating, presolved).
  const bool overlap = a0.side && sc.overlap_from < DS_ROUNDS - 1;
  const bool split = sc.finish_split && a0.run != DS_RUN_STEP;
  auto fork_finish = [&]() {
    ds_trace_mark(DS_STAGE_FINISH, 1, s);
    dcount_snapshot_kernel<<<1, 1, 0, s>>>(a0.ws.dcount);
    ds_trace_mark(DS_STAGE_FINISH, 0, s);
    cudaEventRecord(a0.ev_fork, s);
    cudaStreamWaitEvent(a0.side, a0.ev_fork, 0);
    KArgs fa = af;
    fa.flo = nullptr;
    fa.fhi = a0.ws.dcount + 1;
    int fb = finish_blocks(a0.n_env, fa.nchunk, threads);
    if (sc.reserve > 0) {
      // one CTA per resident slot of every SM (those on reserved SMs return at once), items
      // claimed dynamically, so the other SMs stay full until the work runs out
      int fper = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fper, finish_kernel<NB, NV, NS, T>, threads, 0);
      fb = ds_sm_count() * (fper > 0 ? fper : 1);
      fa.fin_reserve = sc.reserve;
      fa.claim = a0.ws.claim;
    }
    if (split) {
      fa.fin_reserve = 0;
      fa.claim = nullptr;
      launch_finish_split<NB, NV, NS, T>(fa, a0.side);
    } else {
      ds_trace_mark(DS_STAGE_FINISH, 1, a0.side);
      finish_kernel<NB, NV, NS, T><<<fb, threads, 0, a0.side>>>(fa);
      ds_trace_mark(DS_STAGE_FINISH, 0, a0.side);
    }
    cudaEventRecord(a0.ev_join, a0.side);
  };
  if (overlap && sc.overlap_from < 0) fork_finish();
  for (int r = 0; r < DS_ROUNDS; ++r) {
    KArgs a = a0;
    a.round = r;
    a.final_round = r == DS_ROUNDS - 1;
    const int cap = ds_round_cap(table, r);
    a.round_cap = a.final_round ? (a0.admm_max_iter > cap ? a0.admm_max_iter : cap) : cap;
    ds_trace_mark(DS_STAGE_ADMM, 1, s);
    bool done = a0.solver == DS_PGS;
    if (done) pgs_round_kernel<NS, T><<<gblocks, threads, 0, s>>>(a);
    if constexpr (kPairOk) {
      if (!done && r >= sc.pair_from) { admm_round_pair_kernel<NS, T><<<pblocks, 64, 0, s>>>(a); done = true; }
    }
    if constexpr (kWideOk) {
      if (!done && r >= sc.wide_from) {
        admm_round_wide_kernel<NS, T><<<wblocks, threads, 0, s>>>(a);
        done = true;
      }
    }
    if (!done) admm_round_kernel<NS, T><<<rblocks, threads, 0, s>>>(a);
    ds_trace_mark(DS_STAGE_ADMM, 0, s);
    ds_trace_mark(DS_STAGE_NEWTON, 1, s);
    bool launched = false;
    if constexpr (kCoopOk) {
      if (coop) { newton_coop_kernel<NS, T><<<nblocks, nthreads, 0, s>>>(a); launched = true; }
    }
    if (!launched) newton_kernel<NS, T><<<nblocks, nthreads, 0, s>>>(a);
    ds_trace_mark(DS_STAGE_NEWTON, 0, s);
    if (a0.rho_adapt && !a.final_round) {
      ds_trace_mark(DS_STAGE_ADMM, 1, s);
      rho_adapt_kernel<NS, T><<<blocks < ds_sm_count() * 8 ? blocks : ds_sm_count() * 8, threads, 0, s>>>(a);
      ds_trace_mark(DS_STAGE_ADMM, 0, s);
    }
    if (overlap && r == sc.overlap_from) fork_finish();
  }
  if (overlap) {
    // the envs completed after the split: few, so every column gets its own thread
    KArgs fb_args = af;
    fb_args.nchunk = a0.run == DS_RUN_STEP ? 1 : maxc;
    fb_args.flo = a0.ws.dcount + 1;
    fb_args.fhi = a0.ws.dcount;
    const int fb = finish_blocks(a0.n_env, fb_args.nchunk, threads);
    if (split) {
      launch_finish_split<NB, NV, NS, T>(fb_args, s);
    } else {
      ds_trace_mark(DS_STAGE_FINISH, 1, s);
      finish_kernel<NB, NV, NS, T><<<fb, threads, 0, s>>>(fb_args);
      ds_trace_mark(DS_STAGE_FINISH, 0, s);
    }
    cudaStreamWaitEvent(s, a0.ev_join, 0);
    return;
  }
  if (split) {
    launch_finish_split<NB, NV, NS, T>(af, s);
    return;
  }
  const int fblocks = finish_blocks(a0.n_env, af.nchunk, threads);
  ds_trace_mark(DS_STAGE_FINISH, 1, s);
  finish_kernel<NB, NV, NS, T><<<fblocks, threads, 0, s>>>(af);
  ds_trace_mark(DS_STAGE_FINISH, 0, s);
}

// Finish only, from a tape (KArgs.tlam / tmodes / tstat); columns split as in the pipeline.
template <int NB, int NV, int NS, typename T>
void launch_tape(const KArgs& a0, cudaStream_t s) {
  const int threads = 128;
  if (a0.n_env <= 0) return;
  KArgs a = a0;
  a.nchunk = 1;
  if (a0.run != DS_RUN_STEP) {
    const int maxc = a0.run == DS_RUN_JAC ? 3 * NV : 2 * NV;
    const int c = ds_sm_count() * 4 * threads / a0.n_env;
    a.nchunk = c < 1 ? 1 : (c > maxc ? maxc : c);
  }
  ds_trace_mark(DS_STAGE_FINISH, 1, s);
  finish_tape_kernel<NB, NV, NS, T><<<finish_blocks(a0.n_env, a.nchunk, threads), threads, 0, s>>>(a);
  ds_trace_mark(DS_STAGE_FINISH, 0, s);
}

}  // namespace ds
