"""sim_step_jac_noalloc: the allocation-free entry point for callers that cannot allocate device
memory when they step (a real-time control loop that forbids allocation after start-up, a plug-in
that does not own the process's CUDA memory).  Its result must equal sim_step_jac with a
caller-provided workspace, on two calls in a row (the fixed scratch keeps the previous call's
contents, which must not leak into the next result).  Collected last on purpose."""
import numpy as np
import pytest

from paper_2409_07107_gb300 import scenes

pytestmark = pytest.mark.gpu


def test_noalloc_matches_workspace_entry_point():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2409_07107_gb300 as ds
    from paper_2409_07107_gb300 import build
    build.build()
    wl = scenes.arm_cube(65536)
    for B, prec in ((2048, "fp64"), (1500, "mixed")):
        sub = scenes.Workload(wl.name, wl.models, wl.batch.take(np.arange(B)), wl.options)
        sim = ds.Simulator(sub, precision=prec)          # caller-owned workspace
        ref = sim.step_jac()
        torch.cuda.synchronize()
        ref = {k: v.clone() for k, v in ref.items()}
        for call in range(2):
            out = {k: torch.full_like(v, -7) for k, v in sim.out.items()}
            jac = [torch.full_like(ref[k], -7.0) for k in ("dv_dq", "dv_dv", "dv_dtau")]
            ds.sim_step_jac_noalloc(sim.models, sim.batch, sim.opt, out, *jac)
            torch.cuda.synchronize()
            got = dict(out, dv_dq=jac[0], dv_dv=jac[1], dv_dtau=jac[2])
            assert torch.equal(got["modes"], ref["modes"]), call
            assert torch.equal(got["status"], ref["status"]), call
            assert torch.equal(got["iters"], ref["iters"]), call
            for k in ("v_next", "q_next", "lambda", "dv_dq", "dv_dv", "dv_dtau"):
                err = (got[k] - ref[k]).abs().max().item() / max(ref[k].abs().max().item(), 1e-6)
                assert err <= 1e-10, (prec, call, k, err)


def test_noalloc_rejects_batches_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2409_07107_gb300 as ds
    wl = scenes.arm_cube(20000)
    sim = ds.Simulator(wl, precision="fp64", pipeline=False)
    assert ds.workspace_size(sim.models, sim.batch, sim.opt) > 16 * 1024 * 1024
    jac = [torch.zeros(7, 7, wl.batch.B, dtype=torch.float64, device="cuda") for _ in range(3)]
    with pytest.raises(ds.DiffsimError, match="too large"):
        ds.sim_step_jac_noalloc(sim.models, sim.batch, sim.opt, sim.out, *jac)
