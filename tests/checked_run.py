"""Small steps of every workload through whichever build of the library DIFFSIM_LIB names (the
checked build in a child process of test_gpu_checked_build, the normal build in the test itself).

    python -m tests.checked_run OUT.npz     # runs them and saves the outputs and the check counts
"""
import sys

import numpy as np


def run_all():
    import torch
    import paper_2409_07107_gb300 as ds
    from paper_2409_07107_gb300 import scenes
    out = {}
    f64 = dict(dtype=torch.float64, device="cuda")

    def take(tag, res):
        for k, v in res.items():
            out["%s/%s" % (tag, k)] = v.detach().cpu().numpy()

    arm = scenes.arm_cube(65536)
    cases = [("arm_sphere", scenes.arm_sphere(16), "fp64", True),
             ("arm_cube_fp64", scenes.Workload(arm.name, arm.models, arm.batch.take(np.arange(300)), arm.options), "fp64", True),
             ("arm_cube_mixed", scenes.Workload(arm.name, arm.models, arm.batch.take(np.arange(300)), arm.options), "mixed", True),
             ("arm_cube_fused", scenes.Workload(arm.name, arm.models, arm.batch.take(np.arange(64)), arm.options), "fp64", False),
             ("quadruped", scenes.quadruped_feet(64), "fp64", True),
             ("humanoid", scenes.humanoid_feet(16), "mixed", True)]
    for tag, wl, prec, pipeline in cases:
        sim = ds.Simulator(wl, precision=prec, pipeline=pipeline)
        take(tag, sim.step_jac())
    wl = scenes.uneven(30)
    sim = ds.Simulator(wl, precision="fp64")
    vb = torch.as_tensor(np.random.default_rng(5).normal(size=wl.batch.v.shape), **f64)
    take("uneven_vjp", sim.step_vjp(vb))
    wl = scenes.arm_cube(48)
    sim = ds.Simulator(wl, precision="fp64", ncp_solver=ds.DS_PGS)
    take("arm_cube_pgs", sim.step_jac())
    sim = ds.Simulator(wl, precision="fp64", admm_rho_adapt=1)
    take("arm_cube_adaptive", sim.step_jac())
    # the split finish (prep + column kernels) and the persistent launch, on batch sizes of their
    # own (a schedule is kept per batch signature) and set back to the default afterwards
    for tag, wl, prec in (("quadruped_split", scenes.quadruped_feet(100), "fp64"),
                          ("humanoid_split", scenes.humanoid_feet(24), "mixed")):
        sim = ds.Simulator(wl, precision=prec)
        sim.set_schedule(ds.schedule_index(split=1))
        try:
            take(tag, sim.step_jac())
        finally:
            sim.set_schedule(-1)
    wl = scenes.uneven(33)
    sim = ds.Simulator(wl, precision="mixed")
    vb = torch.as_tensor(np.random.default_rng(6).normal(size=wl.batch.v.shape), **f64)
    sim.set_schedule(ds.schedule_index(launch=1), "vjp")
    try:
        take("uneven_persistent", sim.step_vjp(vb))
    finally:
        sim.set_schedule(-1, "vjp")
    torch.cuda.synchronize()
    return out


def main(path):
    import paper_2409_07107_gb300 as ds
    out = run_all()
    out["check/bad_indices"] = np.array(ds.check_bad_indices())
    out["check/self_test_outside"] = np.array(ds.check_self_test(7, 4))
    out["check/self_test_inside"] = np.array(ds.check_self_test(3, 4))
    np.savez(path, **out)


if __name__ == "__main__":
    main(sys.argv[1])
