#!/usr/bin/env python3
"""Throughput of one batched simulation step with its full Jacobians dv+/d(q, v, tau).

Workload (default): 65536 envs of a 7-dof fixed-base arm with a 0.05 m cube at the tip, 4 corner
contacts on a plane, mu ~ U(0.2, 1.0), half the envs set up to stick and half to slide, dt = 1e-3.
One "step" = one sim_step_jac call over the whole batch (forward step, NCP solve, implicit
derivatives, all three Jacobians written); with --workload uneven (a batch that mixes the arm, the
quadruped and the humanoid) one sim_step_vjp call.  The headline value is the plain FP64 method; the same
line carries the mixed-precision form (FP32 bulk, FP64 polish / residual / reduced system).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2409_07107_gb300 import replicas, scenes  # noqa: E402

WORKLOAD_B = 65536

# DRAM bytes (read + write) per env and launch of the FP64 ADMM round kernels on the arm + cube
# workload, from one ncu capture of a default-schedule step at 16384 envs (nine launches,
# 103.1 MB); the workspace traffic grows with the envs.  Valid only while the kernel sources hash
# as recorded here (the ADMM kernels in them are the captured ones).
ADMM_TRAFFIC = {"bytes_per_env_launch": 103.136512e6 / 9 / 16384,
                "sources_sha256_16": {"ds_kernel.cuh": "36baa06f3c62c6ff", "ds_common.cuh": "d9ed443c0376b110"}}


def _admm_traffic_valid():
    import hashlib
    csrc = os.path.join(ROOT, "paper_2409_07107_gb300", "csrc")
    for f, h in ADMM_TRAFFIC["sources_sha256_16"].items():
        with open(os.path.join(csrc, f), "rb") as fh:
            if hashlib.sha256(fh.read()).hexdigest()[:16] != h:
                return False
    return True
METRIC = "env-steps/s with full dv'/d(q,v,tau) at 1 GB300"
METRIC_VJP = "env-steps/s with the VJP of the step at 1 GB300"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# ---------------------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 8:
                continue
            try:
                sm.append(float(p[0]))
                mx = max(mx, float(p[1]))
            except ValueError:
                continue
            for n, v in zip(names, p[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------- algorithmic work model
# Floating-point operations the method has to perform per env-step (an FMA counts 2), by stage, as
# functions of the model's shape and of the env's contact state; the derivation and the per-item
# counts are in the design notes.  It counts what the algorithm requires once (no recomputation,
# no explicit inverse, dense Cholesky of M, one tangent pass per derivative column), so
# (flops / time) / peak is the fraction of the CUDA-core roofline a stage reaches.
C_FK_BODY, C_S_DOF, C_I_BODY, C_RNEA_BODY = 100, 24, 140, 270
C_CRBA_DOF, C_CRBA_PAIR, C_CONTACT, C_JC_DOF, C_FKV_DOF = 72, 12, 24, 25, 30


def _dof_depths(model):
    """Number of dofs on the path from each body to the root (its own included), and the sum over
    dofs of the number of ancestor dofs (the nonzero lower triangle of M)."""
    w = np.array([6 if t == scenes.FREEFLYER else 1 for t in model.jtype])
    depth = np.zeros(model.nb, np.int64)
    for i in range(model.nb):
        depth[i] = w[i] + (depth[model.parent[i]] if model.parent[i] >= 0 else 0)
    pairs = 0
    for i in range(model.nb):
        base = depth[model.parent[i]] if model.parent[i] >= 0 else 0
        for k in range(w[i]):
            pairs += base + k + 1
    return depth, pairs


def algorithmic_flops(model, c_link, modes, iters, kind="jac", mixed=False):
    """Per-stage (fp32, fp64) flop totals over the envs given by c_link / modes [nc][B] (mode 3 =
    inactive slot) and ADMM iteration counts [B].  kind "jac": full Jacobians; "vjp": the VJP."""
    nb, nv = model.nb, model.nv
    depth, pairs = _dof_depths(model)
    act = modes != 3
    na = act.sum(0).astype(float)
    nstk = (modes == 1).sum(0).astype(float)
    nsld = (modes == 2).sum(0).astype(float)
    m, mu = 3.0 * na, 3.0 * (nstk + nsld)
    mr = 3.0 * nstk + 2.0 * nsld
    cdep = np.where(act, depth[np.clip(c_link, 0, nb - 1)], 0).sum(0).astype(float)
    solved = (na > 0) & (iters > 0)
    B = modes.shape[1]
    # setup: F1-F6 (kinematics, bias, M and its factor, contacts, J_c, M^-1 J_c^T, G, g), G + rho I factor
    kin = (C_FK_BODY + C_I_BODY) * nb + C_S_DOF * nv + C_CONTACT * na + C_JC_DOF * cdep
    bulk = C_RNEA_BODY * nb + 10 * nb + C_CRBA_DOF * nv + C_CRBA_PAIR * pairs + 2 * nv ** 3 / 3 + 2 * nv ** 2
    dl = 6 * na * nv ** 2 + m * (m + 1) * nv + 2 * m * nv
    setup64 = kin + dl + bulk * (not mixed) * np.ones(B)
    setup32 = bulk * mixed * np.ones(B)
    admm_f = np.where(solved, 2 * m ** 3 / 3, 0.0)
    setup32, setup64 = (setup32 + admm_f, setup64) if mixed else (setup32, setup64 + admm_f)
    admm = iters * (2 * m ** 2 + 30 * m)
    # Newton polish on the identified modes: one step (factor + solve) and the residual check
    newt_fac = np.where(solved, 2 * mu ** 3 / 3 + 2 * mu ** 2, 0.0)
    newt_res = np.where(solved, 2 * m ** 2 + 30 * na, 0.0)
    # finish: F9, then the derivatives (B1-B6) or the adjoint (B7)
    f9 = 2 * nv * m + nv
    if kind == "jac":
        tang = 2 * nv * (C_RNEA_BODY * nb + 2 * nv ** 2) + nv * 2 * nv ** 2 + nv * C_FKV_DOF * na
        red = 20 * mr ** 2 + 2 * mr ** 3 / 3 + 3 * nv * 2 * mr ** 2 + 18 * na * nv ** 2 + 18 * mr * nv
        asm = 12 * na * nv + 18 * na * nv ** 2
    else:
        tang = 2 * C_RNEA_BODY * nb + 4 * nv ** 2 + nv * C_FKV_DOF * na
        red = 20 * mr ** 2 + 2 * mr ** 3 / 3 + 2 * mr ** 2 + 12 * mr
        asm = 12 * na * nv
    fin_bulk = f9 + tang + asm
    out = {"setup": (setup32, setup64),
           "admm": (admm, 0.0 * admm) if mixed else (0.0 * admm, admm),
           "newton": (newt_fac, newt_res) if mixed else (0.0 * newt_fac, newt_fac + newt_res),
           "finish": (fin_bulk, red) if mixed else (0.0 * red, fin_bulk + red)}
    return {k: (float(np.sum(a)), float(np.sum(b))) for k, (a, b) in out.items()}


def stage_rooflines(flops, stage_ms, step_ms, peak32, peak64):
    """Per stage and for the whole step: achieved TFLOP/s and the fraction of the roofline time
    (F32 / peak32 + F64 / peak64) in the measured time."""
    res = {}
    tot32 = tot64 = 0.0
    for k, (f32, f64) in flops.items():
        tot32 += f32
        tot64 += f64
        t = stage_ms.get(k)
        if not t:
            continue
        bound = (f32 / (peak32 * 1e12) + f64 / (peak64 * 1e12)) * 1e3
        res[k] = {"gflop": (f32 + f64) / 1e9, "fp32_share": f32 / max(f32 + f64, 1.0),
                  "achieved_tflops": (f32 + f64) / (t * 1e-3) / 1e12, "roofline_ms": bound, "frac": bound / t}
    bound = (tot32 / (peak32 * 1e12) + tot64 / (peak64 * 1e12)) * 1e3
    res["step"] = {"gflop": (tot32 + tot64) / 1e9, "achieved_tflops": (tot32 + tot64) / (step_ms * 1e-3) / 1e12,
                   "roofline_ms": bound, "frac": bound / step_ms}
    return res


def dominant_roofline(dominant, roof_stages, stage_launches, admm):
    """The roofline object of the step's dominant stage (the one with the most kernel time): the
    ADMM round kernels' own object when the ADMM stage dominates (the arm), else the dominant
    stage's kernels against the measured FP32 and FP64 FMA peaks weighted by the stage's
    algorithmic FP32 / FP64 flop split (the humanoid's and quadruped's finish); the ADMM object is
    kept under "admm" either way."""
    if dominant in (None, "admm") or dominant not in roof_stages:
        return admm
    r = roof_stages[dominant]
    peak = r["gflop"] / r["roofline_ms"] if r["roofline_ms"] > 0 else None
    return {"bound": "alu", "kernel": "%s stage kernels" % dominant, "achieved": r["achieved_tflops"],
            "peak": peak, "unit": "TFLOP/s", "frac": r["frac"], "traffic": None,
            "peak_source": "measured FMA probes (FP32 and FP64 CUDA cores) in this run, weighted by the "
                           "stage's algorithmic FP32 / FP64 flops (FP32 share %.2f)" % r["fp32_share"],
            "algorithmic_gflop_per_step": r["gflop"], "launches_per_step": stage_launches.get(dominant),
            "admm": admm}


# ------------------------------------------------------------------------------------- CPU oracle
def _model_of(wl, e):
    return wl.models[0 if wl.batch.model_id is None else int(wl.batch.model_id[e])]


def _oracle_rec(args):
    """One env through the oracle: step + full Jacobian (the VJP of the uneven workload is a product
    with it); returns what the error statistics need.  A fourth argument names the oracle's NCP
    route (default its ADMM route; "pgs" the projected Gauss-Seidel one)."""
    model, env, opt = args[:3]
    from oracle import step as S
    if len(args) > 3:
        import types
        opt = types.SimpleNamespace(**dict(vars(opt), ncp_route=args[3]))
    st = S.step_jac(model, env, opt)
    return {k: st[k] for k in ("v_next", "modes", "margin", "slots", "dv_dq", "dv_dv", "dv_dtau", "G", "g", "mu")}


def oracle_alternatives(wl, snaps, recs, processes=None):
    """Eq. 1 can have several solutions (redundant contacts): for the envs where a GPU form's v+ is
    farther from the oracle's ADMM-route solution than its tolerance (1e-6 FP64, 1e-4 mixed), the
    oracle's second route (projected
    Gauss-Seidel), so that the error statistics compare with the nearer oracle solution, as the
    parity tests do.  Returns {env: record}."""
    import multiprocessing as mp
    tol = {"fp64": 1e-6, "mixed": 1e-4}
    envs = sorted({e for prec, snap in snaps.items() for e, r in enumerate(recs)
                   if _rel(snap["v_next"][:_model_of(wl, e).nv, e], r["v_next"]) > tol[prec]})
    if not envs:
        return {}
    args = [(_model_of(wl, e), wl.batch.env(e, _model_of(wl, e)), wl.options, "pgs") for e in envs]
    with mp.get_context("spawn").Pool(min(len(args), processes or os.cpu_count() or 1)) as pool:
        alt = pool.map(_oracle_rec, args)
    return dict(zip(envs, alt))


def cpu_model_name():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_single_thread(wl, seconds=3.0, max_envs=64):
    """Microseconds per env-step (step + full Jacobian) of the oracle on one core, envs in order."""
    t0 = time.perf_counter()
    n = 0
    while n < max_envs and (n < 2 or time.perf_counter() - t0 < seconds):
        m = _model_of(wl, n)
        _oracle_rec((m, wl.batch.env(n, m), wl.options))
        n += 1
    return 1e6 * (time.perf_counter() - t0) / n, n


def collision_pairs_device(n, seed):
    """Seeded random sphere / capsule / box pairs generated on the device (inputs only): types
    uniform over the three, sizes uniform (sphere r in [0.03, 0.1]; capsule half length in
    [0.03, 0.12], r in [0.02, 0.06]; box half extents in [0.03, 0.12]), rotations from normalised
    Gaussian quaternions, positions uniform in a 0.24 m cube (about half the pairs overlap)."""
    import torch
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    f64 = dict(device="cuda", dtype=torch.float64)
    types = torch.randint(0, 3, (2, n), generator=g, device="cuda", dtype=torch.int64)
    lo = torch.tensor([[0.03, 0.0, 0.0], [0.03, 0.02, 0.0], [0.03, 0.03, 0.03]], **f64)
    hi = torch.tensor([[0.1, 0.0, 0.0], [0.12, 0.06, 0.0], [0.12, 0.12, 0.12]], **f64)
    size = lo[types] + (hi - lo)[types] * torch.rand((2, n, 3), generator=g, **f64)
    qt = torch.randn((2, n, 4), generator=g, **f64)
    w, x, y, z = (qt / qt.norm(dim=-1, keepdim=True)).unbind(-1)
    R = torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                     2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                     2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], dim=-1)
    pos = (torch.rand((2, n, 3), generator=g, **f64) * 2.0 - 1.0) * 0.12
    pose = torch.cat([R, pos], dim=-1)
    t32 = types.to(torch.int32)
    return [t32[0].contiguous(), size[0].contiguous(), pose[0].contiguous(),
            t32[1].contiguous(), size[1].contiguous(), pose[1].contiguous()]


def hull_pairs_device(n, seed, n_hulls=4096, verts=16):
    """Seeded random hull pairs generated on the device (inputs only): a pool of n_hulls hulls of
    verts points on ellipsoids with semi-axes in [0.03, 0.1], radius in [0, 0.02]; side A a random
    hull, side B a random hull (even k) or box (odd k); rotations and positions as in
    collision_pairs_device."""
    import torch
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    f64 = dict(device="cuda", dtype=torch.float64)
    x = torch.randn((n_hulls, verts, 3), generator=g, **f64)
    axes = 0.03 + 0.07 * torch.rand((n_hulls, 1, 3), generator=g, **f64)
    pool = (x / x.norm(dim=-1, keepdim=True) * axes).reshape(-1, 3).contiguous()
    pick = torch.randint(0, n_hulls, (2, n), generator=g, device="cuda")
    hull_size = torch.stack([(pick * verts).double(), torch.full((2, n), float(verts), **f64),
                             0.02 * torch.rand((2, n), generator=g, **f64)], dim=-1)
    ta, sa, pa, tb, sb, pb = collision_pairs_device(n, seed + 1)
    box = (torch.arange(n, device="cuda") % 2) == 1
    ta = torch.full_like(ta, 3)
    tb = torch.where(box, torch.full_like(tb, 2), torch.full_like(tb, 3))
    box_size = 0.03 + 0.09 * torch.rand((n, 3), generator=g, **f64)
    sa = hull_size[0].contiguous()
    sb = torch.where(box[:, None], box_size, hull_size[1]).contiguous()
    return [ta.contiguous(), sa, pa, tb.contiguous(), sb, pb], pool


def _time_launches(fn, steps, warmup, flush):
    import torch
    stream = torch.cuda.current_stream()
    ms = []
    for i in range(warmup + steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn(stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if i >= warmup:
            ms.append(e0.elapsed_time(e1))
    return float(np.mean(ms))


def collision_bench(n, steps, warmup, flush):
    """Time ds_collide (one pair per thread) on n random pairs: CUDA events on the launching
    stream around each launch, the L2 flushed before each."""
    import torch

    import paper_2409_07107_gb300 as ds
    args = collision_pairs_device(n, seed=2409)
    out = torch.empty((n, ds.COLLIDE_OUT), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    ms = []
    for i in range(warmup + steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ds.collide(*args, out=out, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if i >= warmup:
            ms.append(e0.elapsed_time(e1))
    overlap = float((out[:, 0] < 0).double().mean())
    bytes_per_pair = 2 * (4 + 3 * 8 + 12 * 8) + ds.COLLIDE_OUT * 8
    t = float(np.mean(ms))
    # convex hulls (16 vertices) against hulls and boxes: GJK, and EPA for overlapping cores
    nh = 65536
    hargs, pool = hull_pairs_device(nh, seed=2410)
    hout = torch.empty((nh, ds.COLLIDE_OUT), dtype=torch.float64, device="cuda")
    th = _time_launches(lambda st: ds.collide(*hargs, hull_vertices=pool, out=hout, stream=st), steps, warmup, flush)
    hulls = {"pairs": nh, "ms_per_launch": th, "pairs_per_s": nh / (th * 1e-3),
             "overlap_fraction": float((hout[:, 0] < 0).double().mean()),
             "nonfinite_pairs": int((~torch.isfinite(hout).all(dim=1)).sum()),
             "note": "hull (16 vertices) against hull or box, every other pair; pool of 4096 hulls"}
    # App. C's randomized-smoothing derivative, 8 antithetic samples (16 collision detections a pair)
    ns, S, sigma = 65536, 8, 1e-3
    sargs = [a[:ns].contiguous() for a in args]
    gen = torch.Generator(device="cuda")
    gen.manual_seed(2411)
    eps = sigma * torch.randn((S, 12), generator=gen, device="cuda", dtype=torch.float64)
    jac = torch.empty((ns, 7, 12), dtype=torch.float64, device="cuda")
    tsm = _time_launches(lambda st: ds.collide_smoothed(*sargs, eps, sigma, out=jac, stream=st), steps, warmup, flush)
    smoothed = {"pairs": ns, "samples": S, "sigma": sigma, "ms_per_launch": tsm, "pairs_per_s": ns / (tsm * 1e-3),
                "nonfinite_pairs": int((~torch.isfinite(jac.reshape(ns, -1)).all(dim=1)).sum())}
    return {"pairs": n, "ms_per_launch": t, "pairs_per_s": n / (t * 1e-3),
            "hbm_gbs": n * bytes_per_pair / (t * 1e-3) / 1e9, "bytes_per_pair": bytes_per_pair,
            "overlap_fraction": overlap, "launches": steps, "hulls": hulls, "smoothing_derivative": smoothed,
            "note": "sphere / capsule / box pairs, FP64; GJK for separated cores, the nearest facet of "
                    "the Minkowski difference (separating axes) for overlapping ones; bound by FP64 "
                    "arithmetic, not HBM; not part of the step (its contacts are primitive versus plane)"}


def oracle_sample(wl, seconds=15.0, cap=1024, processes=None):
    """The oracle on the first n envs of the workload (n: what the host cores do in about
    `seconds`, at most `cap`), in a spawn-started pool.  Returns (records, seconds, cores)."""
    import multiprocessing as mp
    procs = processes or os.cpu_count() or 1
    t0 = time.perf_counter()
    k = min(len(wl.models), wl.batch.B)
    for e in range(k):
        _oracle_rec((_model_of(wl, e), wl.batch.env(e, _model_of(wl, e)), wl.options))
    per = max((time.perf_counter() - t0) / k, 1e-3)
    n = int(max(procs, min(wl.batch.B, cap, seconds * procs / per)))
    args = [(_model_of(wl, e), wl.batch.env(e, _model_of(wl, e)), wl.options) for e in range(n)]
    with mp.get_context("spawn").Pool(procs) as pool:
        pool.map(_oracle_rec, args[:procs])        # warm the workers
        t0 = time.perf_counter()
        recs = pool.map(_oracle_rec, args, chunksize=max(1, n // (4 * procs)))
        dt = time.perf_counter() - t0
    return recs, dt, procs


def _rel(x, ref, floor=1e-6):
    x, ref = np.asarray(x, float), np.asarray(ref, float)
    return float(np.max(np.abs(x - ref)) / max(float(np.max(np.abs(ref))) if ref.size else 0.0, floor)) if ref.size else 0.0


def error_stats(wl, snap, recs, vbar=None, delta=1e-3, alt=None):
    """Per-env relative error (||x - x_ref||_inf / max(||x_ref||_inf, 1e-6)) of v+ and of each
    Jacobian (or each VJP output) against the FP64 oracle, on the envs the oracle ran: max, p99
    and median; Jacobians, VJPs and modes on envs whose oracle classification margin is >= delta;
    counts of mode disagreements, of envs near a mode switch (oracle margin < delta) and of envs
    whose v+ differs from the oracle's by more than 1e-6 (an error).  The reference of an env is
    the nearer (in v+) of the oracle's ADMM-route solution and, where given in ``alt``, its PGS-route
    one (Eq. 1 can have several solutions); envs that took the second are counted.  An env whose v+
    is beyond the form's tolerance (1e-6 FP64, 1e-4 mixed) from both but whose impulse satisfies
    Eq. 1 for the oracle's G, g, mu (NCP residual <= 1e-9 max(1, |g|)) reached yet another solution:
    it is counted, with its v+ difference, under other_solution_of_eq1 and left out of the
    statistics (as the parity tests accept it)."""
    from oracle.ncp import ncp_residual
    keys = ("q_bar", "v_bar", "tau_bar") if vbar is not None else ("dv_dq", "dv_dv", "dv_dtau")
    err = {k: [] for k in ("v_next",) + keys}
    mode_dis = near = far = second = 0
    other = []
    tol = 1e-4 if snap.get("_form") == "mixed" else 1e-6
    for e, r in enumerate(recs):
        nv = _model_of(wl, e).nv
        ev = _rel(snap["v_next"][:nv, e], r["v_next"])
        if alt and e in alt:
            ea = _rel(snap["v_next"][:nv, e], alt[e]["v_next"])
            if ea < ev:
                r, ev = alt[e], ea
                second += 1
        if ev > tol and len(r["slots"]) and "lambda" in snap:
            # neither oracle route's solution: does the GPU impulse solve Eq. 1 for the oracle's
            # problem data (another member of the solution set)?
            lam = np.concatenate([snap["lambda"][3 * k:3 * k + 3, e] for k in r["slots"]])
            scale = max(1.0, float(np.max(np.abs(r["g"]))))
            if ncp_residual(r["G"], r["g"], r["mu"], lam) <= 1e-9 * scale:
                other.append(ev)
                continue
        err["v_next"].append(ev)
        far += ev > 1e-6
        if r["margin"] < delta:
            near += 1
            continue
        if [int(snap["modes"][k, e]) for k in r["slots"]] != [int(x) for x in r["modes"]]:
            mode_dis += 1
            continue
        for k, jk in zip(keys, ("dv_dq", "dv_dv", "dv_dtau")):
            if vbar is None:
                err[k].append(_rel(snap[k][:nv, :nv, e], r[jk]))
            else:
                err[k].append(_rel(snap[k][:nv, e], r[jk].T @ vbar[:nv, e]))

    def q(v):
        return ({"max": float(np.max(v)), "p99": float(np.percentile(v, 99)), "median": float(np.median(v)),
                 "envs": len(v)} if len(v) else None)
    return dict({k: q(v) for k, v in err.items()}, envs=len(recs), mode_disagreements=mode_dis,
                near_switch=near, v_next_off_by_1e6=int(far), second_route_solution=int(second),
                other_solution_of_eq1={"envs": len(other), "v_next_max_diff": float(max(other)) if other else None})


# -------------------------------------------------------------------------------------- rollout
def bench_rollout(args, rank, world):
    """Gradient of a T-step rollout loss w.r.t. all joint torques (forward + reverse pass), the
    quadruped standing on the ground; with segment recomputation every 20 steps and with every
    step's inputs kept.  One timed step = one full rollout forward + backward."""
    import torch
    import paper_2409_07107_gb300 as ds
    from paper_2409_07107_gb300 import build, rollout as R
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    build.build()
    ds.lib()
    B, T, every = args.envs or 4096, args.horizon, 20
    wl = scenes.quadruped_feet(B, seed=replicas.rank_seed(1004, rank))
    rng = np.random.default_rng(21 + rank)
    dev = dict(dtype=torch.float64, device="cuda")
    nv = wl.batch.v.shape[0]
    mask = torch.ones(1, nv, 1, **dev)
    mask[:, :6] = 0.0                                    # no actuation of the floating base
    tau0 = torch.tensor(rng.normal(size=(T, nv, B)) * 2.0, **dev) * mask
    q0, v0 = torch.tensor(wl.batch.q, **dev), torch.tensor(wl.batch.v, **dev)
    sc = R.StepContext(wl, precision="fp64")
    schedule = None if args.no_autotune else sc.autotune(q0, v0, tau0[0].contiguous())
    with torch.no_grad():                                 # reachable goal: a perturbed-torque rollout
        goal, _ = R.rollout(sc, q0, v0, list(tau0 + torch.tensor(rng.normal(size=(T, nv, B)) * 0.5, **dev) * mask), 0)

    def one(ev):
        tau = tau0.clone().requires_grad_(True)
        qT, _ = R.rollout(sc, q0, v0, list(tau * mask), ev)
        loss = ((qT - goal) ** 2).sum()
        loss.backward()
        return tau.grad

    res = {}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for ev in (every, 0):
        for _ in range(args.warmup):
            one(ev)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.reset_peak_memory_stats()
        base = torch.cuda.memory_allocated()
        times = []
        ds.profile(True)
        ds.profile_read()
        with ClockSampler(torch.cuda.current_device()) as clk:
            for _ in range(args.steps):
                flush.fill_(1.0)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                one(ev)
                e1.record()
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
        # library kernels counted by the stage tracer, plus the two cotangent-map kernels per reverse step
        launches = sum(n for _, n in ds.profile_read().values()) + 2 * T * args.steps
        ds.profile(False)
        ms = replicas.slowest_ms(float(np.mean(times)))
        res[ev] = {"ms_per_rollout": ms, "value": replicas.job_throughput(B * T, world, ms),
                   "peak_extra_mib": (torch.cuda.max_memory_allocated() - base) / 2 ** 20, "clocks": clk.summary(),
                   "launches": launches}
    r = res[every]
    line = {"metric": "rollout env-steps/s, forward + reverse pass (d loss / d tau_t) at 1 GB300", "value": r["value"],
            "unit": "env-steps/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": r["ms_per_rollout"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": "quadruped18-rollout: 18-dof quadruped, 4 point feet, %d envs, T=%d steps, "
                                   "loss = sum |q_T - q_goal|^2 (raw q), checkpoint every %d steps" % (B, T, every),
                       "envs_per_gpu": B, "horizon": T, "l2": "flushed between timed rollouts (256 MiB write)"},
            "clocks": r["clocks"], "peak_extra_mib": r["peak_extra_mib"],
            "no_recompute": {"value": res[0]["value"], "ms_per_step": res[0]["ms_per_rollout"],
                             "peak_extra_mib": res[0]["peak_extra_mib"]},
            "gpu_launches": r["launches"], "schedule": schedule}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


# ----------------------------------------------------------------------------- reference arm
def _oracle_count(args):
    _oracle_rec(args)
    return 1


def reference_arm(args, wl, gains, metric, cfg, B):
    """The FP64 oracle on the host cores: W + K steps, each a bounded sample of the workload (the
    next consecutive envs, as many as the cores do in about 0.6 s), timed one by one."""
    import multiprocessing as mp
    for k, val in gains.items():                  # the oracle reads the same gains
        setattr(wl.options, k, val)
    procs = os.cpu_count() or 1
    per, _ = oracle_single_thread(wl, seconds=1.0, max_envs=4)
    n = int(max(procs, min(B // max(1, args.steps + args.warmup), 0.6 * procs / (per * 1e-6))))
    times = []
    with mp.get_context("spawn").Pool(procs) as pool:
        pool.map(_oracle_count, [(_model_of(wl, e), wl.batch.env(e, _model_of(wl, e)), wl.options)
                                 for e in range(procs)])
        for i in range(args.warmup + args.steps):
            lo = (i * n) % max(1, B - n + 1)
            chunk = [(_model_of(wl, e), wl.batch.env(e, _model_of(wl, e)), wl.options) for e in range(lo, lo + n)]
            t0 = time.perf_counter()
            pool.map(_oracle_count, chunk, chunksize=max(1, n // (4 * procs)))
            if i >= args.warmup:
                times.append(time.perf_counter() - t0)
    sec = float(np.mean(times))
    rate = n / sec
    c = dict(cfg, reference_step="%d consecutive envs of the %d-env workload per step (the oracle's "
                                  "bounded sample), step + full Jacobian" % (n, B))
    line = {"impl": "reference", "metric": metric, "value": rate, "unit": "env-steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": c,
            "cpu_baseline": {"value": rate, "unit": "env-steps/s", "cores": procs, "kind": "oracle",
                             "cpu_model": cpu_model_name(),
                             "sample": "%d steps of %d envs each, %.2f s per step" % (args.steps, n, sec)},
            "e2e": {"value": rate, "unit": "env-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------------ main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--envs", type=int, default=None)
    ap.add_argument("--workload", default="arm7-cube", choices=["arm7-cube", "humanoid36-feet", "quadruped18-feet", "uneven",
                                                         "quadruped18-rollout"])
    ap.add_argument("--horizon", type=int, default=200, help="rollout length (quadruped18-rollout)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default pipeline schedule")
    ap.add_argument("--baumgarte", default=None, metavar="KP,KD",
                    help="Baumgarte stabilisation gains (App. D); default: none (1,0)")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus)))
    if args.workload == "quadruped18-rollout":
        if args.impl != "reference":
            return bench_rollout(args, rank, world)
        if rank == 0:
            print(json.dumps({"impl": "reference", "unavailable": "the oracle arm times single steps; the rollout "
                              "workload has no CPU arm"}), flush=True)
        return 0
    wl_name = args.workload
    B = args.envs or {"arm7-cube": WORKLOAD_B, "humanoid36-feet": 16384, "quadruped18-feet": 32768,
                      "uneven": 32768}[wl_name]
    vjp = wl_name == "uneven"          # the mixed-robot batch is timed with sim_step_vjp
    metric = METRIC_VJP if vjp else METRIC
    desc = {"arm7-cube": "7-dof arm + 0.05 m cube, 4 corner contacts",
            "humanoid36-feet": "36-dof humanoid (free-flyer + 30 joints), 2 box feet, 0-8 corner contacts",
            "quadruped18-feet": "18-dof quadruped (free-flyer + 12 joints), 4 point feet",
            "uneven": "mixed batch, envs interleaved: 7-dof arm + cube (8 slots), 18-dof quadruped (4 feet), "
                      "36-dof humanoid (8 foot + 8 hand corners); 16 slots per env; step + VJP with "
                      "v_bar ~ N(0, 1)"}[wl_name]
    cfg = {"workload": "%s: %s, %d envs per GPU, dt=1e-3" % (wl_name, desc, B),
           "envs_per_gpu": B, "l2": "flushed between timed steps (256 MiB write)"}
    gains = {}
    if args.baumgarte:
        kp, kd = (float(x) for x in args.baumgarte.split(","))
        gains = dict(baumgarte_kp=kp, baumgarte_kd=kd)
        cfg["baumgarte"] = {"kp": kp, "kd": kd}
    make = {"arm7-cube": lambda n, r: scenes.arm_cube(n, seed=replicas.rank_seed(1001, r)),
            "humanoid36-feet": lambda n, r: scenes.humanoid_feet(n, seed=replicas.rank_seed(1002, r)),
            "quadruped18-feet": lambda n, r: scenes.quadruped_feet(n, seed=replicas.rank_seed(1004, r)),
            "uneven": lambda n, r: scenes.uneven(n, seed=replicas.rank_seed(1003, r))}[wl_name]

    if args.impl == "reference":
        if rank != 0:
            return 0
        return reference_arm(args, make(B, 0), gains, metric, cfg, B)

    import torch
    import paper_2409_07107_gb300 as ds
    from paper_2409_07107_gb300 import build
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    build.build()
    ds.lib()
    dev = torch.cuda.current_device()
    wl = make(B, rank)
    for k, val in gains.items():                      # the oracle (cpu_baseline) reads the same gains
        setattr(wl.options, k, val)
    peaks = _peaks()

    # measured CUDA-core FMA peaks (the path is bound by plain FP64 / FP32 arithmetic)
    probe = torch.zeros(152 * 16 * 256, dtype=torch.float64, device="cuda")
    fma = {}
    for fp64, iters in ((1, 4096), (0, 32768)):
        ds.fma_peak(probe, 152 * 16, 256, fp64)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        ds.fma_peak(probe, 152 * 16, iters, fp64)
        e1.record()
        torch.cuda.synchronize()
        fma["fp64" if fp64 else "fp32"] = 2 * 8 * iters * 152 * 16 * 256 / (e0.elapsed_time(e1) * 1e-3) / 1e12

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    results, snaps = {}, {}
    vbar = torch.as_tensor(np.random.default_rng(17 + rank).normal(size=wl.batch.v.shape), dtype=torch.float64,
                           device="cuda")

    def one_step(sim):
        return sim.step_vjp(vbar) if vjp else sim.step_jac()

    for prec in ("fp64", "mixed"):
        sim = ds.Simulator(wl, precision=prec, **gains)
        stream = torch.cuda.current_stream()
        # pick the pipeline schedule for this batch (ds_autotune; untimed, part of the set-up)
        schedule = None
        if not args.no_autotune:
            schedule = sim.autotune("vjp", vbar) if vjp else sim.autotune("jac")
        for _ in range(args.warmup):
            one_step(sim)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        times = []
        with ClockSampler(dev) as clk:
            for _ in range(args.steps):
                flush.fill_(1.0)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                one_step(sim)
                e1.record(stream)
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
        # a separate traced pass (CUDA events around every library kernel) for the stage split and
        # the ADMM kernels' time; tracing itself costs time, so it stays out of the timed loop
        traced = max(1, min(args.steps, 5))
        ds.profile(True)
        ds.profile_read()
        for _ in range(traced):
            flush.fill_(1.0)
            one_out = one_step(sim)
        torch.cuda.synchronize()
        stages = ds.profile_read()
        ds.profile(False)
        # the same step replayed from a CUDA graph (launch overhead removed)
        replay = sim.capture("vjp", vbar) if vjp else sim.capture("jac")
        gtimes = []
        for _ in range(args.steps):
            flush.fill_(1.0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            replay()
            e1.record(stream)
            torch.cuda.synchronize()
            gtimes.append(e0.elapsed_time(e1))
        total_ms = replicas.slowest_ms(sum(times))      # max over ranks (replicas; no data exchange)
        ms = total_ms / args.steps
        out = sim.out
        iters = out["iters"].cpu().numpy().astype(np.int64)
        modes = out["modes"].cpu().numpy()
        status = out["status"].cpu().numpy()
        na = (modes != 3).sum(0)
        m = 3 * na
        # algorithmic flops of the ADMM rounds: per env-iteration, the x-step (K times rhs, 2 m^2)
        # plus the right-hand side, De Saxce term, relaxation, projection and dual step (30 m)
        admm_flops = float(np.sum(iters * (2.0 * m * m + 30.0 * m)))
        stage_ms = {k: v[0] / traced for k, v in stages.items() if v[1]}
        stage_launches = {k: v[1] // traced for k, v in stages.items() if v[1]}
        t_admm = stage_ms.get("admm", float("nan"))
        peak = fma["fp64"] if prec == "fp64" else fma["fp32"]
        achieved = admm_flops / (t_admm * 1e-3) / 1e12
        dominant = max(stage_ms, key=stage_ms.get) if stage_ms else None
        # algorithmic work of every stage (per model, summed) and the rooflines of stages and step
        kind = "vjp" if vjp else "jac"
        fl = {}
        c_link = wl.batch.c_link
        for mi, mdl in enumerate(wl.models):
            sel = slice(None) if wl.batch.model_id is None else (wl.batch.model_id == mi)
            part = algorithmic_flops(mdl, c_link[:, sel], modes[:, sel], iters[sel], kind, mixed=(prec == "mixed"))
            for k, (a32, a64) in part.items():
                b32, b64 = fl.get(k, (0.0, 0.0))
                fl[k] = (a32 + b32, a64 + b64)
        roof_stages = stage_rooflines(fl, stage_ms, ms, fma["fp32"], fma["fp64"])
        # contact-mode pattern of every env (sorted modes of its active contacts)
        pat = {}
        for e in range(modes.shape[1]):
            key = "".join("bks"[int(x)] for x in sorted(modes[:, e]) if x != 3) or "-"
            pat[key] = pat.get(key, 0) + 1
        snaps[prec] = {k: v[..., :1024].cpu().numpy() for k, v in one_out.items()}
        snaps[prec]["_form"] = prec
        traffic = None
        if prec == "fp64" and wl_name == "arm7-cube" and _admm_traffic_valid():
            traffic = ADMM_TRAFFIC["bytes_per_env_launch"] * B
        results[prec] = dict(
            ms=ms, value=replicas.job_throughput(B, world, ms), clocks=clk.summary(), schedule=schedule,
            graph={"value": B * world / (float(np.mean(gtimes)) * 1e-3), "ms_per_step": float(np.mean(gtimes))},
            roofline=dominant_roofline(dominant, roof_stages, stage_launches, {
                      "bound": "alu", "kernel": "admm_round_kernel (ADMM rounds, one lane per contact)",
                      "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                      "traffic": traffic,
                      "traffic_note": "DRAM read + write bytes per ADMM launch, from an ncu capture at "
                                      "16384 envs scaled to this batch (null unless the kernels are "
                                      "the captured ones)",
                      "peak_source": "measured FMA probe (%s CUDA cores) in this run" % ("FP64" if prec == "fp64" else "FP32"),
                      "algorithmic_gflop_per_step": admm_flops / 1e9,
                      "launches_per_step": stage_launches.get("admm"),
                      "avg_launch_ms": t_admm / max(stage_launches.get("admm", 1), 1)}),
            stages={k: {"ms_per_step": v, "share": v / ms, "launches_per_step": stage_launches[k]} for k, v in stage_ms.items()},
            stage_roofline=roof_stages,
            mode_patterns=dict(sorted(pat.items(), key=lambda kv: -kv[1])),
            dominant_stage=dominant,
            admm_iters={"mean": float(iters.mean()), "p50": float(np.median(iters)),
                        "p99": float(np.percentile(iters, 99)), "max": int(iters.max())},
            modes={"breaking": int((modes == 0).sum()), "sticking": int((modes == 1).sum()),
                   "sliding": int((modes == 2).sum())},
            status={"not_converged": int((status & 1 != 0).sum()), "nonfinite": int((status & 2 != 0).sum()),
                    "singular": int((status & 4 != 0).sum()), "near_switch": int((status & 8 != 0).sum())},
            launches=sum(stage_launches.values()))
        del sim

    # the same step with projected Gauss-Seidel as the NCP iteration (ncp_solver = DS_PGS), FP64,
    # default schedule: same Newton polish and FP64 residual acceptance, so the comparison is at
    # equal NCP residual
    pgs = adaptive = None
    if not vjp:
        def variant(**kw):
            sim = ds.Simulator(wl, precision="fp64", **kw, **gains)
            for _ in range(max(2, args.warmup)):
                one_step(sim)
            torch.cuda.synchronize()
            pt = []
            for _ in range(max(3, min(args.steps, 10))):
                flush.fill_(1.0)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                one_step(sim)
                e1.record(stream)
                torch.cuda.synchronize()
                pt.append(e0.elapsed_time(e1))
            pit = sim.out["iters"].cpu().numpy().astype(np.int64)
            pst = sim.out["status"].cpu().numpy()
            pms = replicas.slowest_ms(float(np.mean(pt)))
            del sim
            return {"value": replicas.job_throughput(B, world, pms), "ms_per_step": pms,
                    "iters": {"mean": float(pit.mean()), "p50": float(np.median(pit)),
                              "p99": float(np.percentile(pit, 99)), "max": int(pit.max())},
                    "not_converged": int((pst & 1 != 0).sum())}
        pgs = variant(ncp_solver=ds.DS_PGS)
        adaptive = variant(admm_rho_adapt=1)

    # the mixed-robot batch as one persistent launch (schedule knob "launch"; mixed precision, the
    # form it is compiled for) against the workspace pipeline, each eager and replayed from a CUDA
    # graph; the pipeline runs the tuner's other knobs (or the default schedule without tuning)
    persist = None
    if vjp:
        sim = ds.Simulator(wl, precision="mixed", **gains)
        tuned = results["mixed"]["schedule"]
        launch_digit = ds.NUM_SCHEDULES // 4      # the launch knob: the second-highest digit
        idx = tuned["index"] if tuned else ds.schedule_index()
        pipe_idx = idx - ((idx // launch_digit) % 2) * launch_digit
        forms = {}
        try:
            for form, idx in (("persistent", ds.schedule_index(launch=1)), ("pipeline", pipe_idx)):
                sim.set_schedule(idx, "vjp")
                for _ in range(max(2, args.warmup)):
                    one_step(sim)
                torch.cuda.synchronize()
                pt, gt = [], []
                for _ in range(max(3, min(args.steps, 10))):
                    flush.fill_(1.0)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    one_step(sim)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    pt.append(e0.elapsed_time(e1))
                pst = sim.out["status"].cpu().numpy()
                replay = sim.capture("vjp", vbar)
                for _ in range(max(3, min(args.steps, 10))):
                    flush.fill_(1.0)
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    replay()
                    e1.record(stream)
                    torch.cuda.synchronize()
                    gt.append(e0.elapsed_time(e1))
                del replay
                pms, gms = replicas.slowest_ms(float(np.mean(pt))), replicas.slowest_ms(float(np.mean(gt)))
                forms[form] = {"value": replicas.job_throughput(B, world, pms), "ms_per_step": pms,
                               "cuda_graph_replay": {"value": replicas.job_throughput(B, world, gms),
                                                     "ms_per_step": gms},
                               "schedule_index": idx, "queue_timeouts": int((pst & 32 != 0).sum())}
        finally:
            sim.set_schedule(tuned["index"] if tuned else -1, "vjp")
        forms["persistent"]["launches_per_step"] = 1
        persist = forms
        del sim

    # end-to-end through the public API with host buffers (pinned), copies inside the timed region
    sim = ds.Simulator(wl, precision="fp64", **gains)
    host_in = {k: v.cpu().pin_memory() for k, v in sim.batch.items() if k != "model_slots"}
    host_out = {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True)
                for k, v in [("v_next", sim.out["v_next"]), ("q_next", sim.out["q_next"]), ("status", sim.out["status"])]}
    dkeys = ("q_bar", "v_bar", "tau_bar") if vjp else ("dv_dq", "dv_dv", "dv_dtau")
    if vjp:
        host_in["vbar"] = vbar.cpu().pin_memory()
    jac0 = one_step(sim)
    host_jac = [torch.empty(jac0[k].shape, dtype=torch.float64, pin_memory=True) for k in dkeys]
    h2d = sum(v.numel() * v.element_size() for k, v in host_in.items() if k != "model_slots")
    d2h = sum(v.numel() * v.element_size() for v in host_out.values()) + sum(v.numel() * 8 for v in host_jac)
    stream = torch.cuda.current_stream()
    e2e_ms = []
    for i in range(args.warmup + args.steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k, v in host_in.items():
            if k == "vbar":
                vbar.copy_(v, non_blocking=True)
            elif k != "model_slots":
                sim.batch[k].copy_(v, non_blocking=True)
        r = one_step(sim)
        for k, v in host_out.items():
            v.copy_(r[k], non_blocking=True)
        for hj, k in zip(host_jac, dkeys):
            hj.copy_(r[k], non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        if i >= args.warmup:
            e2e_ms.append(e0.elapsed_time(e1))
    e2e_value = replicas.job_throughput(B, world, replicas.slowest_ms(float(np.mean(e2e_ms))))

    # the FP64 oracle on the host cores: the CPU baseline, and the error of both GPU forms against it
    cpu, errors = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        recs, dt, procs = oracle_sample(wl, seconds=args.cpu_seconds)
        us1, n1 = oracle_single_thread(wl)
        cpu = {"value": len(recs) / dt, "unit": "env-steps/s", "cores": procs, "kind": "oracle",
               "cpu_model": cpu_model_name(),
               "sample": "first %d envs of the workload, step + full Jacobian (numpy oracle, spawn pool), %.1f s"
                         % (len(recs), dt),
               "single_thread_us_per_env_step": us1, "single_thread_sample": "first %d envs, one core" % n1}
        vb = vbar.cpu().numpy() if vjp else None
        alt = oracle_alternatives(wl, snaps, recs)
        errors = {prec: error_stats(wl, snaps[prec], recs, vb, alt=alt) for prec in ("fp64", "mixed")}

    collision = None
    if rank == 0:
        try:
            collision = collision_bench(262144, max(args.steps, 5), max(args.warmup, 3), flush)
        except Exception as e:      # reported in the line; the step's numbers stand
            collision = {"error": "%s: %s" % (type(e).__name__, e)}

    if rank == 0:
        r64, rmx = results["fp64"], results["mixed"]
        line = {"metric": metric, "value": r64["value"], "unit": "env-steps/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": r64["ms"], "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
                "clocks": r64["clocks"], "roofline": r64["roofline"],
                "e2e": {"value": e2e_value, "unit": "env-steps/s", "h2d_bytes_per_step": int(h2d),
                        "d2h_bytes_per_step": int(d2h)},
                "gpu_launches": args.steps * r64["launches"], "cpu_baseline": cpu,
                "stages": r64["stages"], "dominant_stage": r64["dominant_stage"], "cuda_graph_replay": r64["graph"],
                "stages_note": "kernel time per stage from a separate traced pass (CUDA events around every "
                               "library kernel, kept out of the timed loop); the finish of early-solved envs "
                               "overlaps the late ADMM rounds on a second stream, so stages can sum past the step",
                "schedule": r64["schedule"],
                "admm_iters": r64["admm_iters"], "modes": r64["modes"], "env_status": r64["status"],
                "mode_patterns": r64["mode_patterns"],
                "mode_patterns_note": "envs by the sorted modes of their active contacts (b breaking, k sticking, "
                                      "s sliding; - no contact)",
                "stage_roofline": r64["stage_roofline"],
                "error_vs_fp64_oracle": None if errors is None else errors["fp64"],
                "mixed": {"value": rmx["value"], "ms_per_step": rmx["ms"], "dtype": "f32+f64", "roofline": rmx["roofline"],
                          "cuda_graph_replay": rmx["graph"], "schedule": rmx["schedule"],
                          "stages": rmx["stages"], "dominant_stage": rmx["dominant_stage"],
                          "clocks": rmx["clocks"], "admm_iters": rmx["admm_iters"], "modes": rmx["modes"],
                          "env_status": rmx["status"], "stage_roofline": rmx["stage_roofline"],
                          "error_vs_fp64_oracle": None if errors is None else errors["mixed"]},
                "pgs_fp64": pgs,
                "adaptive_rho_fp64": adaptive,
                "adaptive_rho_note": "the FP64 step with the ADMM penalty updated between rounds by residual "
                                     "balancing (admm_rho_adapt = 1; default schedule), accepted by the same "
                                     "FP64 NCP residual test; iters = ADMM iterations",
                "persistent_launch_mixed": persist,
                "persistent_note": "mixed precision: the step + VJP as one persistent kernel (warps pull chunks "
                                   "of 32 envs of one model from an atomic queue, one env per lane) and as "
                                   "the workspace pipeline (the tuner's other knobs), eager and from a CUDA "
                                   "graph",
                "pgs_note": "the FP64 step with projected Gauss-Seidel sweeps as the NCP iteration (default "
                            "schedule), accepted by the same FP64 NCP residual test as the ADMM form; "
                            "iters = sweeps",
                "collision_detection": collision,
                "fma_peak_tflops": fma, "peaks_file": {k: peaks.get(k) for k in ("hbm_gbs", "bf16_tflops")}}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
