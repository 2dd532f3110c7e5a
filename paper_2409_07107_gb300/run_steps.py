"""Run a few steps of a benchmark workload and print the step time: a small driver for profilers
(ncu) and quick timings, without the benchmark's autotuning, variants and CPU baseline.

    python -m paper_2409_07107_gb300.run_steps --workload humanoid36-feet --envs 4096 \
        --precision mixed --kind jac --warmup 3 --steps 3 [--schedule INDEX]

Each step is one sim_step_jac (kind jac), sim_step_vjp with v_bar ~ N(0, 1) (kind vjp) or
sim_step (kind step) on the same seeded batch; --schedule installs a schedule index first (as
ds_set_schedule; see SCHEDULE_KNOBS)."""
import argparse

import numpy as np

from . import scenes

WORKLOADS = {"arm7-cube": lambda n: scenes.arm_cube(n, seed=1001),
             "humanoid36-feet": lambda n: scenes.humanoid_feet(n, seed=1002),
             "quadruped18-feet": lambda n: scenes.quadruped_feet(n, seed=1004),
             "uneven": lambda n: scenes.uneven(n, seed=1003)}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="arm7-cube", choices=sorted(WORKLOADS))
    ap.add_argument("--envs", type=int, default=4096)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--kind", default="jac", choices=["step", "jac", "vjp"])
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--schedule", type=int, default=None)
    args = ap.parse_args(argv)

    import torch
    from . import Simulator, build, describe_schedule
    build.build()
    sim = Simulator(WORKLOADS[args.workload](args.envs), precision=args.precision)
    vbar = torch.as_tensor(np.random.default_rng(17).normal(size=sim.workload.batch.v.shape),
                           dtype=torch.float64, device="cuda")
    if args.schedule is not None:
        sim.set_schedule(args.schedule, args.kind)
    step = {"step": lambda: sim.step(), "jac": lambda: sim.step_jac(), "vjp": lambda: sim.step_vjp(vbar)}[args.kind]
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(args.steps, 1)
    sched = describe_schedule(args.schedule) if args.schedule is not None else "default"
    print("%s %d envs %s %s: %.3f ms per step (schedule %s)" % (args.workload, args.envs, args.precision, args.kind,
                                                               ms, sched))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
