"""The persistent launch (schedule knob "launch"): the whole step of a batch that mixes the arm +
cube, the quadruped and the humanoid as one kernel whose warps pull chunks of envs from an atomic
work queue, one env per lane.

* parity: v+ and the VJP against the oracle on sampled envs of every model, and agreement with the
  workspace pipeline (the same per-env algorithm in other kernels);
* the queue's bounded wait: with queue_poll_limit = 0 a CTA gives up at once, the envs nobody
  processed carry DS_ENV_QUEUE_TIMEOUT and NaN, the others are exact, and the next call with the
  default limit runs complete (no fault, no hang);
* CUDA-graph capture of the persistent launch replays the eager results exactly."""
import numpy as np
import pytest

from paper_2409_07107_gb300 import scenes
from tests.oracle_runner import run_oracle
from tests.test_gpu_parity import _compare, torch_cuda  # noqa: F401  (fixture)

pytestmark = pytest.mark.gpu

QUEUE_TIMEOUT = 32


def _persistent(sim, kind):
    import paper_2409_07107_gb300 as ds
    return sim.set_schedule(ds.schedule_index(launch=1), kind)


def test_persistent_uneven_vjp_parity(torch_cuda):
    """Sampled envs of each model (and the ragged tail) against the oracle's v+ and J^T v_bar at
    the mixed path's tolerances; v+, modes and the VJP against the pipeline's on the whole batch."""
    import paper_2409_07107_gb300 as ds
    torch = torch_cuda
    B = 3001
    wl = scenes.uneven(B)
    sim = ds.Simulator(wl, precision="mixed")
    wbar = np.random.default_rng(21).normal(size=wl.batch.v.shape)
    vb = torch.as_tensor(wbar, dtype=torch.float64, device="cuda")
    ref = {k: v.clone() for k, v in sim.step_vjp(vb).items()}
    _persistent(sim, "vjp")
    try:
        got = {k: v.clone() for k, v in sim.step_vjp(vb).items()}
        torch.cuda.synchronize()
    finally:
        sim.set_schedule(-1, "vjp")
    assert not (got["status"] & QUEUE_TIMEOUT).any()
    # the same per-env algorithm as the pipeline: equal up to rounding (and the rare env where Eq. 1
    # has several solutions and the two kernels stop at different iterates)
    ok = ((ref["status"] & 8) == 0) & ((got["status"] & 8) == 0)
    scale = ref["v_next"].abs().amax(0).clamp_min(1e-6)
    close = ((got["v_next"] - ref["v_next"]).abs().amax(0) / scale) <= 1e-4
    assert close[ok].float().mean().item() >= 0.99
    assert (got["modes"] == ref["modes"])[:, ok & close].float().mean().item() >= 0.995
    rng = np.random.default_rng(22)
    envs = sorted(set([0, 1, 2, B - 3, B - 2, B - 1] + [int(3 * k + r) for r in range(3)
                                                          for k in rng.choice(B // 3, 10, replace=False)]))
    g = {k: v[..., envs].cpu().numpy() for k, v in got.items()}
    sub = scenes.Workload(wl.name, wl.models, wl.batch.take(envs), wl.options)
    refs = run_oracle(sub, list(range(len(envs))))
    _compare(sub, g, refs, list(range(len(envs))), 1e-4, 1e-3, jac=False, vjp=wbar[:, envs], min_checked=24)


def test_persistent_jacobians(torch_cuda):
    """sim_step_jac under the persistent launch: v+ and the three Jacobians of sampled envs against
    the oracle."""
    import paper_2409_07107_gb300 as ds
    torch = torch_cuda
    wl = scenes.uneven(600)
    sim = ds.Simulator(wl, precision="mixed")
    sim.step_jac()
    _persistent(sim, "jac")
    try:
        out = sim.step_jac()
        torch.cuda.synchronize()
    finally:
        sim.set_schedule(-1, "jac")
    envs = list(range(0, 600, 25)) + [597, 598, 599]
    g = {k: v[..., envs].cpu().numpy() for k, v in out.items()}
    # an env of a model with nv dofs writes its Jacobians to the leading nv * nv rows of the
    # [n * n][B] arrays ((i * nv + j) * B + e): put each into the top-left block for the comparison
    n = out["dv_dq"].shape[0]
    for key in ("dv_dq", "dv_dv", "dv_dtau"):
        flat = out[key].reshape(n * n, -1)[:, envs].cpu().numpy()
        blk = np.zeros((n, n, len(envs)))
        for j, e in enumerate(envs):
            nv = wl.models[int(wl.batch.model_id[e])].nv
            blk[:nv, :nv, j] = flat[:nv * nv, j].reshape(nv, nv)
        g[key] = blk
    sub = scenes.Workload(wl.name, wl.models, wl.batch.take(envs), wl.options)
    refs = run_oracle(sub, list(range(len(envs))))
    assert not (g["status"] & QUEUE_TIMEOUT).any()
    _compare(sub, g, refs, list(range(len(envs))), 1e-4, 1e-3, min_checked=15)


def test_persistent_queue_timeout(torch_cuda):
    """queue_poll_limit = 0: the first CTA to file its share of the env lists finds the others
    still filing and gives up; every CTA then stops claiming work.  The envs left carry
    DS_ENV_QUEUE_TIMEOUT and NaN in v+, the envs processed equal the complete run's, and the
    context stays usable: the next call with the default limit completes every env."""
    import paper_2409_07107_gb300 as ds
    torch = torch_cuda
    wl = scenes.uneven(30000)
    full = ds.Simulator(wl, precision="mixed")
    _persistent(full, "step")
    try:
        full.step()
        ref = {k: v.clone() for k, v in full.out.items()}
        short = ds.Simulator(wl, precision="mixed", queue_poll_limit=0)
        short.step()
        got = {k: v.clone() for k, v in short.out.items()}
        again = ds.Simulator(wl, precision="mixed")
        again.step()
        torch.cuda.synchronize()
    finally:
        full.set_schedule(-1, "step")
    timed_out = (got["status"] & QUEUE_TIMEOUT) != 0
    assert timed_out.any()
    assert not (ref["status"] & QUEUE_TIMEOUT).any() and not (again.out["status"] & QUEUE_TIMEOUT).any()
    nv = np.array([m.nv for m in wl.models])[wl.batch.model_id]
    for e in torch.nonzero(timed_out).flatten().tolist()[:200]:
        assert torch.isnan(got["v_next"][:nv[e], e]).all()
    done = ~timed_out
    assert torch.equal(got["v_next"][:, done], ref["v_next"][:, done])
    assert torch.equal(got["status"][done], ref["status"][done])
    assert torch.equal(again.out["v_next"], ref["v_next"])


def test_persistent_cuda_graph(torch_cuda):
    """The persistent step + VJP captured in a CUDA graph (queue reset and kernel) and replayed
    gives the eager results exactly (each env is computed by one thread, whichever warp claims it)."""
    import paper_2409_07107_gb300 as ds
    torch = torch_cuda
    wl = scenes.uneven(960)
    sim = ds.Simulator(wl, precision="mixed")
    vb = torch.as_tensor(np.random.default_rng(23).normal(size=wl.batch.v.shape), dtype=torch.float64,
                         device="cuda")
    _persistent(sim, "vjp")
    try:
        eager = {k: v.clone() for k, v in sim.step_vjp(vb).items()}
        replay = sim.capture("vjp", vb)
        for t in (sim.out["v_next"], sim.out["status"], *sim.vjp_out):
            t.zero_()
        replay()
        replay()
        torch.cuda.synchronize()
    finally:
        sim.set_schedule(-1, "vjp")
    got = dict(sim.out, q_bar=sim.vjp_out[0], v_bar=sim.vjp_out[1], tau_bar=sim.vjp_out[2])
    for key in ("v_next", "q_bar", "v_bar", "tau_bar", "status", "modes"):
        assert torch.equal(got[key], eager[key]), key


def test_persistent_schedule_falls_back_to_the_pipeline(torch_cuda):
    """The persistent kernel is compiled for the mixed form of the three mixed-batch shapes; under a
    persistent schedule an FP64 batch, or a model whose fitted shape is not among them (the arm with
    4 slots), runs the workspace pipeline: the results are the default schedule's, bit for bit."""
    import paper_2409_07107_gb300 as ds
    torch = torch_cuda
    arm = scenes.arm_cube(65536)
    for wl, prec in ((scenes.uneven(90), "fp64"),
                     (scenes.Workload(arm.name, arm.models, arm.batch.take(np.arange(200)), arm.options), "mixed")):
        sim = ds.Simulator(wl, precision=prec)
        ref = {k: v.clone() for k, v in sim.step().items()}
        _persistent(sim, "step")
        try:
            got = {k: v.clone() for k, v in sim.step().items()}
            torch.cuda.synchronize()
        finally:
            sim.set_schedule(-1, "step")
        for key in ("v_next", "q_next", "lambda", "modes", "status", "iters"):
            assert torch.equal(got[key], ref[key]), (prec, key)
