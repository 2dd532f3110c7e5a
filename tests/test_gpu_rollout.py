"""Rollout pieces on the GPU against the oracle: the step's VJP with a cotangent of q+ as well (the
position-update adjoint), the raw <-> tangent cotangent maps, and reverse-mode gradients of a
multi-step rollout through torch.autograd, with and without segment recomputation."""
import numpy as np
import pytest

from oracle import rigid
from oracle import step as S
from paper_2409_07107_gb300 import scenes
from tests.oracle_runner import rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2409_07107_gb300 as ds
    from paper_2409_07107_gb300 import build
    build.build()
    ds.lib()
    return torch


def test_vjp_with_position_cotangent(torch_cuda):
    import paper_2409_07107_gb300 as ds
    torch = torch_cuda
    wl = scenes.quadruped_feet(32)
    m = wl.models[0]
    rng = np.random.default_rng(11)
    vb = rng.normal(size=wl.batch.v.shape)
    qb = rng.normal(size=wl.batch.v.shape)
    sim = ds.Simulator(wl, precision="fp64")
    t = lambda a: torch.as_tensor(a, dtype=torch.float64, device="cuda")  # noqa: E731
    out = sim.step_vjp(t(vb), q_next_bar=t(qb))
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy() for k, v in out.items()}
    checked = 0
    for e in range(12):
        env = wl.batch.env(e, m)
        st = S.step_jac(m, env, wl.options)
        if st["margin"] < 1e-3:
            continue
        ref = S.vjp(m, env, wl.options, vb[:, e], st=st, q_bar_next=qb[:, e])
        for k, key in enumerate(("q_bar", "v_bar", "tau_bar")):
            assert rel_err(g[key][:, e], ref[k]) <= 1e-9, (e, key)
        checked += 1
    assert checked >= 4


def test_cotangent_maps(torch_cuda):
    import paper_2409_07107_gb300 as ds
    torch = torch_cuda
    wl = scenes.uneven(9)
    b = wl.batch
    models = [ds.DeviceModel(mm) for mm in wl.models]
    rng = np.random.default_rng(12)
    raw, tan = rng.normal(size=b.q.shape), rng.normal(size=b.v.shape)
    t = lambda a: torch.as_tensor(a, dtype=torch.float64, device="cuda").contiguous()  # noqa: E731
    q, mid = t(b.q), torch.as_tensor(b.model_id, dtype=torch.int32, device="cuda")
    out_t = torch.zeros(b.v.shape, dtype=torch.float64, device="cuda")
    out_r = torch.zeros(b.q.shape, dtype=torch.float64, device="cuda")
    ds.cotangent_to_tangent(models, q, t(raw), out_t, mid)
    ds.cotangent_to_raw(models, q, t(tan), out_r, mid)
    torch.cuda.synchronize()
    out_t, out_r = out_t.cpu().numpy(), out_r.cpu().numpy()
    for e in range(b.B):
        mm = wl.models[int(b.model_id[e])]
        qe = b.q[:mm.nq, e]
        ref_t = rigid.tangent_to_raw_jacobian(mm, qe).T @ raw[:mm.nq, e]
        ref_r = rigid.raw_to_tangent_jacobian(mm, qe).T @ tan[:mm.nv, e]
        assert np.abs(out_t[:mm.nv, e] - ref_t).max() <= 1e-13
        assert np.abs(out_r[:mm.nq, e] - ref_r).max() <= 1e-13


@pytest.mark.parametrize("every", [0, 2])
def test_rollout_gradient(torch_cuda, every):
    """d loss / d tau_t of loss = sum_env |q_T - q_goal|^2 (raw q) over 5 steps of the quadruped,
    through SimStep + torch.autograd, against the oracle's reverse accumulation."""
    from paper_2409_07107_gb300 import rollout as R
    torch = torch_cuda
    wl = scenes.quadruped_feet(32)
    m = wl.models[0]
    T = 5
    rng = np.random.default_rng(13)
    taus = rng.normal(size=(T,) + wl.batch.v.shape) * 2.0
    taus[:, :6] = 0.0
    goal = np.stack([rigid.integrate(m, wl.batch.q[:, e], 0.01 * rng.normal(size=m.nv)) for e in range(wl.batch.B)], 1)
    sc = R.StepContext(wl, precision="fp64")
    dev = dict(dtype=torch.float64, device="cuda")
    tau_p = torch.tensor(taus, **dev, requires_grad=True)
    qT, vT = R.rollout(sc, torch.tensor(wl.batch.q, **dev), torch.tensor(wl.batch.v, **dev), list(tau_p), every)
    loss = ((qT - torch.tensor(goal, **dev)) ** 2).sum()
    loss.backward()
    g = tau_p.grad.cpu().numpy()
    qT = qT.detach().cpu().numpy()
    checked = 0
    for e in range(wl.batch.B):
        if checked >= 3:
            break
        env = wl.batch.env(e, m)
        qT_ref = S.rollout(m, env, taus[:, :, e], wl.options)[-1][0]
        ref, states, margin = S.rollout_grad(m, env, taus[:, :, e], wl.options, 2.0 * (qT_ref - goal[:, e]))
        assert rel_err(qT[:, e], states[-1][0]) <= 1e-9
        if margin < 1e-3:
            continue
        assert rel_err(g[:, :, e], ref) <= 1e-8, e
        checked += 1
    assert checked >= 2


def test_rollout_gradient_vs_gpu_central_differences(torch_cuda):
    """The rollout check on the GPU path itself: per-env directional derivatives of
    loss = |q_T - q_goal|^2 (20 steps, 8 envs, checkpoints every 5 steps) by central differences of
    GPU rollouts (h = 1e-6, FP64) against the autograd gradient.  An env whose trajectory crosses a
    mode or contact switch within h is not differentiable there, so 6 of the 8 must agree."""
    from paper_2409_07107_gb300 import rollout as R
    torch = torch_cuda
    wl = scenes.quadruped_feet(8)
    T, h = 20, 1e-6
    rng = np.random.default_rng(17)
    dev = dict(dtype=torch.float64, device="cuda")
    nv = wl.batch.v.shape[0]
    mask = torch.ones(1, nv, 1, **dev)
    mask[:, :6] = 0.0
    taus = torch.tensor(rng.normal(size=(T, nv, wl.batch.B)) * 2.0, **dev) * mask
    sc = R.StepContext(wl, precision="fp64")
    q0, v0 = torch.tensor(wl.batch.q, **dev), torch.tensor(wl.batch.v, **dev)
    with torch.no_grad():
        goal, _ = R.rollout(sc, q0, v0, list(taus + torch.tensor(rng.normal(size=taus.shape) * 0.5, **dev) * mask), 0)
    tau_p = taus.clone().requires_grad_(True)
    qT, _ = R.rollout(sc, q0, v0, list(tau_p), 5)
    ((qT - goal) ** 2).sum().backward()
    u = torch.tensor(rng.normal(size=taus.shape), **dev) * mask
    with torch.no_grad():
        lp = ((R.rollout(sc, q0, v0, list(taus + h * u), 0)[0] - goal) ** 2).sum(0)
        lm = ((R.rollout(sc, q0, v0, list(taus - h * u), 0)[0] - goal) ** 2).sum(0)
    fd = ((lp - lm) / (2 * h)).cpu().numpy()
    an = (tau_p.grad * u).sum((0, 1)).cpu().numpy()
    rel = np.abs(fd - an) / np.maximum(np.abs(an), 1e-8)
    assert (rel <= 1e-4).sum() >= 6, rel


@pytest.mark.parametrize("which,precision", [("quadruped", "fp64"), ("uneven", "mixed")])
def test_vjp_from_tape_matches_vjp(torch_cuda, which, precision):
    """sim_step_vjp_tape (finish only, impulses and modes from a preceding sim_step's outputs) gives
    the same cotangents as sim_step_vjp, which solves the NCP again."""
    import paper_2409_07107_gb300 as ds
    torch = torch_cuda
    wl = scenes.quadruped_feet(96) if which == "quadruped" else scenes.uneven(96)
    sim = ds.Simulator(wl, precision=precision)
    out = sim.step()
    tape = {"lambda": out["lambda"].clone(), "modes": out["modes"].clone(), "status": out["status"].clone()}
    rng = np.random.default_rng(19)
    t = lambda a: torch.as_tensor(a, dtype=torch.float64, device="cuda").contiguous()  # noqa: E731
    vb, qb = t(rng.normal(size=wl.batch.v.shape)), t(rng.normal(size=wl.batch.v.shape))
    ref = {k: v.clone() for k, v in sim.step_vjp(vb, q_next_bar=qb).items()}
    got = [torch.zeros_like(vb) for _ in range(3)]
    out2 = {"v_next": torch.zeros_like(vb)}
    ds.sim_step_vjp_tape(sim.models, sim.batch, sim.opt, vb, tape, out2, *got, q_next_bar=qb)
    torch.cuda.synchronize()
    # the two finish paths order their products differently (solves with M's factor in place of
    # M^-1 J_c^T when columns are split): rounding-level differences only
    tol = 1e-10 if precision == "fp64" else 1e-4
    for g, key in zip(got, ("q_bar", "v_bar", "tau_bar")):
        err = ((g - ref[key]).abs().amax(0) / ref[key].abs().amax(0).clamp_min(1e-6)).max().item()
        assert err <= tol, (key, err)
    assert ((out2["v_next"] - ref["v_next"]).abs().max() / ref["v_next"].abs().max()).item() <= tol
