#!/usr/bin/env python3
"""Throughput of one batched simulation step with its full Jacobians dv+/d(q, v, tau).

Workload (default): 65536 envs of a 7-dof fixed-base arm with a 0.05 m cube at the tip, 4 corner
contacts on a plane, mu ~ U(0.2, 1.0), half the envs set up to stick and half to slide, dt = 1e-3.
One "step" = one sim_step_jac call over the whole batch (forward step, NCP solve, implicit
derivatives, all three Jacobians written).  The headline value is the plain FP64 method; the same
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

from paper_2409_07107_gb300 import scenes  # noqa: E402

WORKLOAD_B = 65536
METRIC = "env-steps/s with full dv'/d(q,v,tau) at 1 GB300"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


# ------------------------------------------------------------------------------------ flop model
def step_flops(nb, nv, depth_dofs, subtree_bodies, na, m_red, iters, polish_iters_run, jac=True):
    """Arithmetic (FMA = 2 flops) of one env-step of the kernel's algorithm, counted from its loops.

    nb, nv: bodies / dofs; depth_dofs[d]: dofs on the path root..body(d) (incl. d);
    subtree_bodies[d]: bodies in the subtree of dof d's body; na active contacts; m_red = size of
    the reduced implicit system; iters ADMM iterations; polish_iters_run Newton steps."""
    m = 3 * na
    f = 0.0
    f += nb * 340                     # placements, motion subspaces, world inertias
    f += nb * 200                     # bias RNEA
    f += sum(42 + 11 * dd for dd in depth_dofs) + 10 * nb    # composite inertia + M entries
    f += nv ** 3 / 3 + 2 * nv ** 2 + 2 * nv                    # Cholesky of M and v_f
    f += na * 27 * (sum(depth_dofs) / max(nv, 1))             # J_c rows
    f += 2 * m * nv ** 2 + m * (m + 1) * nv + 2 * m * nv      # W, G, Y, g
    if na:
        f += m ** 3 / 3 + m * m                                # factor G + rho I
        f += iters * (4 * m * m + 10 * m + 25 * na)            # ADMM iterations
        f += polish_iters_run * (2 * m ** 3 / 3 + 6 * m * m)   # Newton steps on the mode equations
        f += 3 * (4 * m * m + 60 * na)                         # residual / classification checks
    f += 2 * m * nv                                            # v+
    if not jac:
        return f
    f += nb * 120 + 2 * m * nv                                 # a* pass, contact forces, v+ velocities
    f += (2.0 / 3.0) * m_red ** 3 + 4 * m_red * m_red          # reduced system and its LU
    tq = sum(400 * s for s in subtree_bodies) + sum(11 * dd for dd in depth_dofs)
    tv = sum(200 * s for s in subtree_bodies) + sum(11 * dd for dd in depth_dofs)
    f += tq + tv                                               # tangent passes (2 nv directions)
    f += 3 * nv * (2 * nv * nv)                                # M^-1 on 3 nv columns
    f += 3 * nv * (m * 2 * nv + 2 * m_red * m_red + m * 2 * nv) + nv * na * 40   # RHS, solve, dv
    return f


def model_shape(model):
    iv = model.iv
    nd = [6 if t == scenes.FREEFLYER else 1 for t in model.jtype]
    dof_body = [i for i in range(model.nb) for _ in range(nd[i])]
    sub = []
    for i in range(model.nb):
        e = i + 1
        while e < model.nb:
            b = e
            while b > i:
                b = model.parent[b]
            if b != i:
                break
            e += 1
        sub.append(e - i)
    depth = []
    for d in range(model.nv):
        b = dof_body[d]
        n = (d - iv[b]) + 1
        b = model.parent[b]
        while b >= 0:
            n += nd[b]
            b = model.parent[b]
        depth.append(n)
    return depth, [sub[dof_body[d]] for d in range(model.nv)]


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


# ------------------------------------------------------------------------------------- CPU oracle
def _oracle_one(args):
    model, env, opt = args
    from oracle import step as S
    S.step_jac(model, env, opt)
    return 1


def cpu_oracle_rate(wl, n_envs=None, seconds=20.0, processes=None):
    """Oracle env-steps/s (step + full Jacobian) on the host cores, on a bounded sample."""
    import multiprocessing as mp
    m = wl.models[0]
    procs = processes or os.cpu_count() or 1
    if n_envs is None:
        t0 = time.perf_counter()
        _oracle_one((m, wl.batch.env(0, m), wl.options))
        per = max(time.perf_counter() - t0, 1e-3)
        n_envs = int(max(procs, min(wl.batch.B, seconds * procs / per)))
    args = [(m, wl.batch.env(e, m), wl.options) for e in range(n_envs)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        pool.map(_oracle_one, args[:procs])        # warm the workers
        t0 = time.perf_counter()
        pool.map(_oracle_one, args, chunksize=max(1, n_envs // (4 * procs)))
        dt = time.perf_counter() - t0
    return n_envs / dt, procs, n_envs, dt


# ------------------------------------------------------------------------------------------ main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--envs", type=int, default=WORKLOAD_B)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus)))
    B = args.envs
    wl_name = "arm7-cube"
    cfg = {"workload": "%s: 7-dof arm + 0.05 m cube, 4 corner contacts, %d envs per GPU, dt=1e-3" % (wl_name, B),
           "envs_per_gpu": B, "l2": "flushed between timed steps (256 MiB write)"}

    if args.impl == "reference":
        if rank != 0:
            return 0
        wl = scenes.arm_cube(B)
        rate, procs, n, dt = cpu_oracle_rate(wl, seconds=max(5.0, 12.0 * args.steps / 20.0))
        line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": "env-steps/s", "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * B / rate, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
                "cpu_baseline": {"value": rate, "unit": "env-steps/s", "cores": procs, "kind": "oracle",
                                 "sample": "first %d envs of the workload, step + full Jacobian, %.1f s" % (n, dt)},
                "e2e": {"value": rate, "unit": "env-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0

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
    wl = scenes.arm_cube(B, seed=1001 + rank * 7919)
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
    results = {}
    for prec in ("fp64", "mixed"):
        sim = ds.Simulator(wl, precision=prec)
        stream = torch.cuda.current_stream()
        for _ in range(args.warmup):
            sim.step_jac()
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        times = []
        with ClockSampler(dev) as clk:
            for _ in range(args.steps):
                flush.fill_(1.0)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                sim.step_jac()
                e1.record(stream)
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
        if world > 1:
            t = torch.tensor([sum(times)], device="cuda")
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            total_ms = t.item()
        else:
            total_ms = sum(times)
        ms = total_ms / args.steps
        out = sim.out
        iters = out["iters"].cpu().numpy()
        modes = out["modes"].cpu().numpy()
        status = out["status"].cpu().numpy()
        # algorithmic flops per launch from the per-env ADMM iteration counts and contact modes
        m = wl.models[0]
        depth, subtree = model_shape(m)
        na = (modes != 3).sum(0)
        nstk = (modes == 1).sum(0)
        nsld = (modes == 2).sum(0)
        mred = 3 * nstk + 2 * nsld
        fl = 0.0
        for k in np.unique(np.stack([na, mred, np.minimum(iters, 10 ** 6)]), axis=1).T:
            sel = (na == k[0]) & (mred == k[1]) & (iters == k[2])
            fl += sel.sum() * step_flops(m.nb, m.nv, depth, subtree, int(k[0]), int(k[1]), int(k[2]), 2)
        peak = fma["fp64"] if prec == "fp64" else fma["fp32"]
        achieved = fl / (ms * 1e-3) / 1e12
        results[prec] = dict(ms=ms, value=B * world / (total_ms / args.steps * 1e-3), clocks=clk.summary(),
                             roofline={"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                                       "frac": achieved / peak, "traffic": None,
                                       "peak_source": "measured FMA probe (%s CUDA cores) in this run" % ("FP64" if prec == "fp64" else "FP32")},
                             admm_iters={"mean": float(iters.mean()), "p50": float(np.median(iters)),
                                         "p99": float(np.percentile(iters, 99)), "max": int(iters.max())},
                             modes={"breaking": int((modes == 0).sum()), "sticking": int((modes == 1).sum()),
                                    "sliding": int((modes == 2).sum())},
                             status={"not_converged": int((status & 1 != 0).sum()), "nonfinite": int((status & 2 != 0).sum()),
                                     "singular": int((status & 4 != 0).sum()), "near_switch": int((status & 8 != 0).sum())},
                             gflop_per_step=fl / 1e9)
        del sim

    # end-to-end through the public API with host buffers (pinned), copies inside the timed region
    sim = ds.Simulator(wl, precision="fp64")
    host_in = {k: v.cpu().pin_memory() for k, v in sim.batch.items()}
    host_out = {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True)
                for k, v in [("v_next", sim.out["v_next"]), ("q_next", sim.out["q_next"]), ("status", sim.out["status"])]}
    jac0 = sim.step_jac()
    host_jac = [torch.empty(jac0[k].shape, dtype=torch.float64, pin_memory=True) for k in ("dv_dq", "dv_dv", "dv_dtau")]
    h2d = sum(v.numel() * v.element_size() for v in host_in.values())
    d2h = sum(v.numel() * v.element_size() for v in host_out.values()) + sum(v.numel() * 8 for v in host_jac)
    stream = torch.cuda.current_stream()
    e2e_ms = []
    for i in range(args.warmup + args.steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for k, v in host_in.items():
            sim.batch[k].copy_(v, non_blocking=True)
        r = sim.step_jac()
        for k, v in host_out.items():
            v.copy_(r[k], non_blocking=True)
        for hj, k in zip(host_jac, ("dv_dq", "dv_dv", "dv_dtau")):
            hj.copy_(r[k], non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        if i >= args.warmup:
            e2e_ms.append(e0.elapsed_time(e1))
    e2e_value = B * world / (np.mean(e2e_ms) * 1e-3)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, procs, n, dt = cpu_oracle_rate(wl, seconds=args.cpu_seconds)
        cpu = {"value": rate, "unit": "env-steps/s", "cores": procs, "kind": "oracle",
               "sample": "first %d envs of the workload, step + full Jacobian (numpy oracle, spawn pool), %.1f s" % (n, dt)}

    if rank == 0:
        r64, rmx = results["fp64"], results["mixed"]
        line = {"metric": METRIC, "value": r64["value"], "unit": "env-steps/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": r64["ms"], "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
                "clocks": r64["clocks"], "roofline": r64["roofline"],
                "e2e": {"value": e2e_value, "unit": "env-steps/s", "h2d_bytes_per_step": int(h2d),
                        "d2h_bytes_per_step": int(d2h)},
                "gpu_launches": args.steps * (2 + 2 * 9), "cpu_baseline": cpu,
                "admm_iters": r64["admm_iters"], "modes": r64["modes"], "env_status": r64["status"],
                "gflop_per_step": r64["gflop_per_step"],
                "mixed": {"value": rmx["value"], "ms_per_step": rmx["ms"], "dtype": "f32+f64", "roofline": rmx["roofline"],
                          "clocks": rmx["clocks"], "admm_iters": rmx["admm_iters"], "modes": rmx["modes"],
                          "env_status": rmx["status"]},
                "fma_peak_tflops": fma, "peaks_file": {k: peaks.get(k) for k in ("hbm_gbs", "bf16_tflops")}}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
