"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, element by element.

Tolerances (relative, per env, ||x - x_ref||_inf / max(||x_ref||_inf, 1e-6)):
  FP64 path: v+ and the three Jacobians <= 1e-9; modes bit-exact.
  Mixed path: v+ <= 1e-4; Jacobians <= 1e-3.

Eq. 1 can have more than one solution, so the oracle solves every env by two independent routes
(ADMM and projected Gauss-Seidel, each with the Newton polish; neither shares a parameter with the
kernels).  The GPU's v+ must equal that of one of the oracle's solutions; an env where it equals
none is accepted only if the GPU impulse satisfies Eq. 1 for the oracle's G, g and mu, and such envs
must stay rare.  Modes and Jacobians are then compared with the matched oracle solution on envs
whose oracle classification margin is >= 1e-3 (away from mode switches; the decision is the
oracle's, not the kernel's), and Jacobians only where the oracle's routes agree on them (where they
do not, the derivative depends on which member of a family of solutions a solver reaches)."""
import numpy as np
import pytest

from paper_2409_07107_gb300 import scenes
from tests.oracle_runner import candidates, jac_of, rel_err, run_oracle

pytestmark = pytest.mark.gpu

DELTA = 1e-3


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


def _gpu(wl, precision, run="jac"):
    import paper_2409_07107_gb300 as ds
    sim = ds.Simulator(wl, precision=precision)
    out = sim.step_jac() if run == "jac" else sim.step()
    import torch
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _gpu_lambda(g, e, slots):
    return np.concatenate([g["lambda"][3 * k:3 * k + 3, e] for k in slots]) if len(slots) else np.zeros(0)


def _match(g, e, r, nv, tol_v):
    """The oracle solution whose v+ the GPU reached, or None after checking that the GPU impulse
    solves Eq. 1 for the oracle's problem data (another member of its solution set)."""
    from oracle.ncp import ncp_residual
    for c in candidates(r):
        if rel_err(g["v_next"][:nv, e], c["v_next"]) <= tol_v:
            return c
    lam = _gpu_lambda(g, e, r["slots"])
    scale = max(1.0, float(np.max(np.abs(r["g"])))) if len(r["g"]) else 1.0
    res = ncp_residual(r["G"], r["g"], r["mu"], lam)
    assert res <= tol_v * scale, "env %d: v+ matches no oracle solution and the impulse violates Eq. 1 (%.3e)" % (e, res)
    return None


def _jac_defined(r, c, tol=1e-8):
    """False when the oracle's routes reach the matched v+ and modes but differ in the Jacobian."""
    for o in candidates(r):
        if o is c or list(o["modes"]) != list(c["modes"]) or rel_err(o["v_next"], c["v_next"]) > 1e-9:
            continue
        if rel_err(jac_of(o), jac_of(c)) > tol:
            return False
    return True


def _compare(wl, g, refs, envs, tol_v, tol_j, jac=True, min_checked=1, vjp=None, max_other=0.05):
    """Checks every env as the module docstring states.  With ``vjp`` = v_bar [nv][B] the GPU's
    q_bar, v_bar, tau_bar are compared with J^T v_bar of the matched oracle Jacobians."""
    checked = other = 0
    for e, r in zip(envs, refs):
        mi = 0 if wl.batch.model_id is None else int(wl.batch.model_id[e])
        nv = wl.models[mi].nv
        assert g["status"][e] & 2 == 0, "env %d non-finite" % e
        c = _match(g, e, r, nv, tol_v)
        if c is None:
            other += 1
            continue
        if c["margin"] < DELTA:
            continue
        gm = [int(g["modes"][k, e]) for k in c["slots"]]
        assert gm == [int(x) for x in c["modes"]], "env %d modes %s vs %s" % (e, gm, c["modes"])
        if (jac or vjp is not None) and not _jac_defined(r, c):
            continue
        if jac:
            for key in ("dv_dq", "dv_dv", "dv_dtau"):
                ej = rel_err(g[key][:nv, :nv, e], c[key])
                assert ej <= tol_j, "env %d %s rel err %.3e" % (e, key, ej)
        if vjp is not None:
            for key, jk in (("q_bar", "dv_dq"), ("v_bar", "dv_dv"), ("tau_bar", "dv_dtau")):
                ej = rel_err(g[key][:nv, e], c[jk].T @ vjp[:nv, e])
                assert ej <= tol_j, "env %d %s rel err %.3e" % (e, key, ej)
        checked += 1
    assert checked >= min_checked, (checked, min_checked)
    assert other <= max(1, int(max_other * len(envs))), "%d envs reached no oracle solution" % other
    return checked


def test_arm_sphere_fp64(torch_cuda):
    wl = scenes.arm_sphere(16)
    g = _gpu(wl, "fp64")
    envs = list(range(16))
    refs = run_oracle(wl, envs)
    _compare(wl, g, refs, envs, 1e-9, 1e-9, min_checked=10)
    for e, r in zip(envs, refs):
        assert np.abs(g["q_next"][:, e] - r["q_next"]).max() <= 1e-12


def test_arm_cube_fp64_ragged(torch_cuda):
    """300 envs = two full 128-thread blocks and a ragged tail of 44."""
    wl = scenes.arm_cube(65536)
    idx = np.arange(300)
    sub = scenes.Workload(wl.name, wl.models, wl.batch.take(idx), wl.options)
    g = _gpu(sub, "fp64")
    envs = list(range(300))
    refs = run_oracle(sub, envs)
    _compare(sub, g, refs, envs, 1e-9, 1e-9, min_checked=200)


def test_arm_cube_mixed(torch_cuda):
    wl = scenes.arm_cube(65536)
    sub = scenes.Workload(wl.name, wl.models, wl.batch.take(np.arange(160)), wl.options)
    g = _gpu(sub, "mixed")
    envs = list(range(160))
    refs = run_oracle(sub, envs)
    _compare(sub, g, refs, envs, 1e-4, 1e-3, min_checked=100)


def test_quadruped_fp64_and_mixed(torch_cuda):
    wl = scenes.quadruped_feet(64)
    envs = list(range(24))
    refs = run_oracle(wl, envs)
    _compare(wl, _gpu(wl, "fp64"), refs, envs, 1e-9, 1e-9, min_checked=10)
    _compare(wl, _gpu(wl, "mixed"), refs, envs, 1e-4, 1e-3, min_checked=10)


def test_humanoid_fp64_and_mixed(torch_cuda):
    wl = scenes.humanoid_feet(40)
    envs = list(range(6))
    refs = run_oracle(wl, envs)
    _compare(wl, _gpu(wl, "fp64"), refs, envs, 1e-9, 1e-9, min_checked=3)
    _compare(wl, _gpu(wl, "mixed"), refs, envs, 1e-4, 1e-3, min_checked=3)


def test_point_mass_closed_form(torch_cuda):
    """Sliding point mass on a plane: v+ and dv+/dv from the closed form of App. A."""
    from tests.helpers import point_mass_model
    mass, dt, mu = 2.0, 1e-3, 0.5
    m = point_mass_model(mass)
    vlin = np.array([1.0, 0.5, -0.3])
    B = 3
    q = np.tile(np.array([0.1, -0.2, 0.3, 1.0, 0.0, 0.0, 0.0])[:, None], (1, B))
    v = np.zeros((6, B))
    v[:3] = vlin[:, None]
    batch = scenes.Batch(q, v, np.zeros((6, B)), np.zeros((1, B), np.int32), np.zeros((1, 3, B)),
                         np.zeros((1, B)), np.full((1, B), mu), np.tile(np.array([0, 0, 1.0, 0.3001])[:, None], (1, B)))
    g = _gpu(scenes.Workload("pm", [m], batch), "fp64")
    vf = vlin + dt * np.array([0, 0, -9.81])
    u = vf[:2] / np.linalg.norm(vf[:2])
    assert np.allclose(g["v_next"][:2, 0], vf[:2] + mu * vf[2] * u, atol=1e-13)
    assert abs(g["v_next"][2, 0]) < 1e-13
    J = np.zeros((3, 3))
    J[:2, :2] = np.eye(2) - mu * (-vf[2]) / np.linalg.norm(vf[:2]) * (np.eye(2) - np.outer(u, u))
    J[:2, 2] = mu * u
    assert np.allclose(g["dv_dv"][:3, :3, 0], J, atol=1e-10)
    assert int(g["modes"][0, 0]) == 2


def test_vjp_matches_jacobian_transpose(torch_cuda):
    """Dot-product identity <w, J u> = <J^T w, u> between sim_step_jac and sim_step_vjp."""
    import paper_2409_07107_gb300 as ds
    torch = torch_cuda
    for wl, prec, tol in ((scenes.arm_cube(256), "fp64", 1e-11), (scenes.quadruped_feet(128), "fp64", 1e-11),
                          (scenes.arm_cube(256), "mixed", 1e-4)):
        sim = ds.Simulator(wl, precision=prec)
        out = sim.step_jac()
        J = [out[k].clone() for k in ("dv_dq", "dv_dv", "dv_dtau")]
        rng = np.random.default_rng(0)
        w = torch.as_tensor(rng.normal(size=tuple(out["v_next"].shape)), dtype=torch.float64, device="cuda")
        vo = sim.step_vjp(w)
        torch.cuda.synchronize()
        for k, key in enumerate(("q_bar", "v_bar", "tau_bar")):
            ref = torch.einsum("ib,ijb->jb", w, J[k])
            err = (vo[key] - ref).abs().max().item() / max(ref.abs().max().item(), 1e-6)
            assert err <= tol, (prec, key, err)


def test_edge_cases(torch_cuda):
    """B = 1, an env with no active contact, a NaN input (status bit, no fault), unused slots."""
    import paper_2409_07107_gb300 as ds
    torch = torch_cuda
    wl = scenes.arm_cube(8)
    b = wl.batch.take(np.arange(3))
    b.plane[3, 1] = -10.0                     # env 1: plane far below -> no contact
    b.q[2, 2] = np.nan                        # env 2: non-finite input
    b.c_link[3, 0] = -1                       # env 0: one slot unused
    sub = scenes.Workload(wl.name, wl.models, b, wl.options)
    g = _gpu(sub, "fp64")
    assert g["status"][2] & 2
    assert (g["modes"][:, 1] == 3).all()
    assert g["modes"][3, 0] == 3
    one = scenes.Workload(wl.name, wl.models, wl.batch.take([5]), wl.options)
    g1 = _gpu(one, "fp64")
    r = run_oracle(one, [0])[0]
    _match(g1, 0, r, wl.models[0].nv, 1e-9)      # an oracle solution's v+, or a solution of Eq. 1
    empty = ds.Simulator(scenes.Workload(wl.name, wl.models, wl.batch.take([]), wl.options))
    empty.step()


def test_pipeline_matches_fused(torch_cuda):
    """The workspace pipeline (setup, compacted ADMM rounds, finish) and the fused single kernel run
    the same per-env algorithm; rounding differences between the two kernels (FMA contraction)
    can move an env across an ADMM convergence test by one iteration, so results agree to the
    parity tolerance, and iteration counts and modes almost everywhere."""
    import paper_2409_07107_gb300 as ds
    torch = torch_cuda
    wl = scenes.arm_cube(65536)
    sub = scenes.Workload(wl.name, wl.models, wl.batch.take(np.arange(2048)), wl.options)
    for prec, tol in (("fp64", 1e-10), ("mixed", 1e-5)):
        outs = []
        for pipeline in (False, True):
            sim = ds.Simulator(sub, precision=prec, pipeline=pipeline)
            o = sim.step_jac()
            torch.cuda.synchronize()
            outs.append({k: v.cpu().numpy().astype(float) for k, v in o.items()})
        f, p = outs
        assert (f["iters"] == p["iters"]).mean() >= (0.99 if prec == "fp64" else 0.9)
        assert (f["modes"] == p["modes"]).mean() >= 0.995
        for k in ("v_next", "dv_dq", "dv_dv", "dv_dtau"):
            err = np.abs(f[k] - p[k]).max(axis=tuple(range(f[k].ndim - 1))) / np.maximum(
                np.abs(f[k]).max(axis=tuple(range(f[k].ndim - 1))), 1e-6)
            assert np.quantile(err, 0.99) <= tol, (prec, k, np.quantile(err, 0.99))


def test_uneven_batch_step_and_vjp(torch_cuda):
    """A batch that mixes the arm + cube (8 slots), the quadruped (4 slots) and the humanoid (16
    slots), interleaved env by env; each model runs the kernel of its own slot count.  v+ and the
    VJP (q_bar, v_bar, tau_bar = J^T v_bar+) against the oracle's step and Jacobians."""
    import paper_2409_07107_gb300 as ds
    torch = torch_cuda
    wl = scenes.uneven(60)
    envs = list(range(18))                     # 6 envs of each model
    refs = run_oracle(wl, envs)
    rng = np.random.default_rng(7)
    wbar = rng.normal(size=wl.batch.v.shape)
    for prec, tol_v, tol_j in (("fp64", 1e-9, 1e-9), ("mixed", 1e-4, 1e-3)):
        sim = ds.Simulator(wl, precision=prec)
        out = sim.step_vjp(torch.as_tensor(wbar, dtype=torch.float64, device="cuda"))
        torch.cuda.synchronize()
        g = {k: v.cpu().numpy() for k, v in out.items()}
        assert not (g["status"] & 16).any()
        _compare(wl, g, refs, envs, tol_v, tol_j, jac=False, vjp=wbar, min_checked=12)


def test_uneven_batch_slot_dispatch(torch_cuda):
    """A used slot beyond a model's declared slot count is flagged (DS_ENV_BAD_SLOT), not read
    out of range; declared counts above ncmax or with no compiled kernel are refused."""
    import paper_2409_07107_gb300 as ds
    wl = scenes.uneven(30)
    b = wl.batch.take(np.arange(30))
    b.model_slots = np.array([4, 4, 16], np.int32)     # the arm's envs use 8 slots
    g = _gpu(scenes.Workload(wl.name, wl.models, b, wl.options), "fp64", run="step")
    arm = b.model_id == 0
    used_high = (b.c_link[4:] >= 0).any(axis=0)
    assert ((g["status"] & 16) != 0).tolist() == (arm & used_high).tolist()
    for bad in ([8, 4, 17], [8, 5, 16]):
        b.model_slots = np.array(bad, np.int32)
        with pytest.raises(ds.DiffsimError):
            _gpu(scenes.Workload(wl.name, wl.models, b, wl.options), "fp64", run="step")


def test_uneven_batch_cuda_graph(torch_cuda):
    """The mixed-robot step + VJP (three models, helper streams forked and joined with events)
    captured in a CUDA graph and replayed gives the eager call's results exactly."""
    import paper_2409_07107_gb300 as ds
    torch = torch_cuda
    wl = scenes.uneven(96)
    sim = ds.Simulator(wl, precision="mixed")
    vb = torch.as_tensor(np.random.default_rng(3).normal(size=wl.batch.v.shape), dtype=torch.float64,
                         device="cuda")
    eager = {k: v.clone() for k, v in sim.step_vjp(vb).items()}
    replay = sim.capture("vjp", vb)
    for t in (sim.out["v_next"], sim.out["status"], *sim.vjp_out):
        t.zero_()
    replay()
    torch.cuda.synchronize()
    got = dict(sim.out, q_bar=sim.vjp_out[0], v_bar=sim.vjp_out[1], tau_bar=sim.vjp_out[2])
    for key in ("v_next", "q_bar", "v_bar", "tau_bar", "status", "modes"):
        assert torch.equal(got[key], eager[key]), key


def _same_solutions(ref, got, frac=0.995):
    """Two GPU runs of one batch under different schedules: away from mode switches, v+, the modes
    and the Jacobians agree (v+ 1e-9, Jacobians 1e-8) on all but a few envs, those where Eq. 1 has
    several solutions and the runs stopped their iterations at different iterates."""
    ok = ((ref["status"] & 8) == 0) & ((got["status"] & 8) == 0)
    assert ok.float().mean().item() > 0.8
    scale = ref["v_next"].abs().amax(0).clamp_min(1e-6)
    same = ((got["v_next"] - ref["v_next"]).abs().amax(0) / scale) <= 1e-9
    assert same[ok].float().mean().item() >= frac
    both = ok & same
    for key in ("dv_dq", "dv_dv", "dv_dtau"):
        sj = ref[key].abs().amax((0, 1)).clamp_min(1e-6)
        assert ((got[key] - ref[key]).abs().amax((0, 1)) / sj)[both].max().item() <= 1e-8, key
    assert (got["modes"] == ref["modes"])[:, both].float().mean().item() >= 0.995


def test_autotune_keeps_results(torch_cuda):
    """ds_autotune picks a schedule by timing; the step's results under it agree with the
    default schedule's (schedules change how work is divided; an env's result changes by rounding,
    or, where Eq. 1 has several solutions, can be another one)."""
    import paper_2409_07107_gb300 as ds
    torch = torch_cuda
    wl = scenes.arm_cube(3000)
    sim = ds.Simulator(wl, precision="fp64")
    ref = {k: v.clone() for k, v in sim.step_jac().items()}
    desc = sim.autotune("jac")
    assert 0 <= desc["index"] < ds.NUM_SCHEDULES
    got = sim.step_jac()
    torch.cuda.synchronize()
    _same_solutions(ref, got)


@pytest.mark.parametrize("precision,tol_v,tol_j", [("fp64", 1e-9, 1e-9), ("mixed", 1e-4, 1e-3)])
def test_arm_cube_full_size_sampled(torch_cuda, precision, tol_v, tol_j):
    """The benchmark's configuration: 65536 envs in one call (one thread per env in the finish
    kernel, the implicit part applied by rows), with outputs sampled across the batch (first,
    last and 46 seeded indices) against the oracle."""
    import paper_2409_07107_gb300 as ds
    torch = torch_cuda
    wl = scenes.arm_cube(65536)
    sim = ds.Simulator(wl, precision=precision)
    out = sim.step_jac()
    torch.cuda.synchronize()
    envs = sorted(set([0, 65535] + list(np.random.default_rng(5).choice(65536, 46, replace=False))))
    g = {k: v[..., envs].cpu().numpy() for k, v in out.items()}
    sub = scenes.Workload(wl.name, wl.models, wl.batch.take(envs), wl.options)
    refs = run_oracle(sub, list(range(len(envs))))
    _compare(sub, g, refs, list(range(len(envs))), tol_v, tol_j, min_checked=30)


@pytest.mark.parametrize("pair", [0, 1])
def test_two_warp_admm_rounds(torch_cuda, pair):
    """The two-warp ADMM kernel (x-step and projection on one warp, De Saxce term and convergence
    test on the other; for the 4-slot arm the x-step summed in two halves, one lane each) runs the
    row-per-lane kernel's iteration up to the rounding of that sum: with it from round 3 (or 5)
    and halved round caps, so that many envs pass through it, v+, the iteration counts and the
    Jacobians agree with those of the row-per-lane rounds."""
    import paper_2409_07107_gb300 as ds
    torch = torch_cuda
    wl = scenes.arm_cube(3000)
    sim = ds.Simulator(wl, precision="fp64")
    sim.set_schedule(ds.schedule_index(round_caps=1, pair=2))     # row-per-lane rounds only
    ref = {k: v.clone() for k, v in sim.step_jac().items()}
    desc = sim.set_schedule(ds.schedule_index(round_caps=1, pair=pair))
    assert desc["two_warp_admm_from_round"] == (3, 5)[pair]
    try:
        got = sim.step_jac()
        torch.cuda.synchronize()
    finally:
        sim.set_schedule(-1)
    assert (got["iters"] == ref["iters"]).float().mean().item() >= 0.99
    _same_solutions(ref, got)


@pytest.mark.parametrize("overlap,reserve,B,caps", [(2, 1, 20000, 0), (3, 2, 20000, 0), (2, 1, 600, 1), (0, 1, 20000, 0)])
def test_overlapped_finish_on_reserved_sms(torch_cuda, overlap, reserve, B, caps):
    """The overlapped finish that keeps every 8th (4th) SM free claims its work items dynamically
    (the small batch: a launch of a few items per SM), also when it starts right after the setup.  Each env's finish is the same code on the
    same inputs, so every output is bitwise that of the finish on every SM (the ADMM kernels are
    the same in both)."""
    import paper_2409_07107_gb300 as ds
    torch = torch_cuda
    wl = scenes.arm_cube(B)
    sim = ds.Simulator(wl, precision="fp64")
    sim.set_schedule(ds.schedule_index(round_caps=caps, overlap=overlap, reserve=0))    # finish on every SM
    ref = {k: v.clone() for k, v in sim.step_jac().items()}
    assert (ref["iters"] > 256).sum().item() >= 1          # some envs reach the late rounds
    desc = sim.set_schedule(ds.schedule_index(round_caps=caps, overlap=overlap, reserve=reserve))
    assert desc["overlapped_finish_after_round"] == ("setup", 2, 4, 5, None)[overlap]
    assert desc["overlapped_finish_keeps_free_every_nth_sm"] == (None, 8, 4)[reserve]
    try:
        got = sim.step_jac()
        torch.cuda.synchronize()
    finally:
        sim.set_schedule(-1)
    for k in ("v_next", "q_next", "lambda", "modes", "status", "iters", "dv_dq", "dv_dv", "dv_dtau"):
        if k in ref:
            assert torch.equal(got[k], ref[k]), k


@pytest.mark.parametrize("precision,tol_v,tol_j", [("fp64", 1e-9, 1e-9), ("mixed", 1e-4, 1e-3)])
def test_baumgarte_stabilised_step(torch_cuda, precision, tol_v, tol_j):
    """Baumgarte stabilisation (App. D) with gains K_p = 0.4, K_d = 0.2: v+, modes and the three
    Jacobians against the oracle's stabilised step (its closed-form and finite-difference pins are
    in test_oracle_baumgarte.py), and the VJP against the transposed Jacobian."""
    import types
    import paper_2409_07107_gb300 as ds
    torch = torch_cuda
    wl = scenes.arm_cube(512)
    o = wl.options
    opt = types.SimpleNamespace(dt=o.dt, gravity=o.gravity, admm_max_iter=o.admm_max_iter, admm_eps=o.admm_eps,
                                polish_iters=o.polish_iters, eps_sigma=o.eps_sigma, eps_lambda=o.eps_lambda,
                                baumgarte_kp=0.4, baumgarte_kd=0.2)
    sim = ds.Simulator(wl, precision=precision)
    sim.opt.baumgarte_kp, sim.opt.baumgarte_kd = 0.4, 0.2
    out = sim.step_jac()
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy() for k, v in out.items()}
    envs = list(range(0, 512, 16))
    refs = run_oracle(wl, envs, opt=opt)
    _compare(wl, g, refs, envs, tol_v, tol_j, min_checked=8)
    if precision == "fp64":
        vbar = torch.randn(sim.nv, wl.batch.B, dtype=torch.float64, device="cuda")
        r = sim.step_vjp(vbar)
        torch.cuda.synchronize()
        qb, vb, tb = r["q_bar"], r["v_bar"], r["tau_bar"]
        ok = (out["status"] & 8) == 0
        for J, got in ((out["dv_dq"], qb), (out["dv_dv"], vb), (out["dv_dtau"], tb)):
            ref = torch.einsum("kjb,kb->jb", J, vbar)
            err = ((got - ref).abs().amax(0) / ref.abs().amax(0).clamp_min(1e-6))[ok].max().item()
            assert err <= 1e-9, err
    # unit gains: the unstabilised step, bitwise
    sim.opt.baumgarte_kp, sim.opt.baumgarte_kd = 1.0, 0.0
    a1 = {k: v.clone() for k, v in sim.step_jac().items()}
    sim2 = ds.Simulator(wl, precision=precision)
    a2 = sim2.step_jac()
    torch.cuda.synchronize()
    for k in ("v_next", "dv_dq", "dv_dv", "dv_dtau"):
        assert torch.equal(a1[k], a2[k]), k


def _sampled(B, n, seed):
    return sorted(set([0, B - 1] + [int(x) for x in np.random.default_rng(seed).choice(B, n, replace=False)]))


@pytest.mark.parametrize("precision,tol_v,tol_j", [("fp64", 1e-9, 1e-9), ("mixed", 1e-4, 1e-3)])
def test_humanoid_full_size_sampled(torch_cuda, precision, tol_v, tol_j):
    """The 36-dof humanoid at its benchmark size (16384 envs in one call: the finish kernel's launch
    shape for that size), outputs sampled across the batch against the oracle.  Envs without an
    active contact are cheap to check and are included; at least 30 envs must be fully compared."""
    import paper_2409_07107_gb300 as ds
    torch = torch_cuda
    B = 16384
    wl = scenes.humanoid_feet(B)
    sim = ds.Simulator(wl, precision=precision)
    out = sim.step_jac()
    torch.cuda.synchronize()
    envs = _sampled(B, 62, 11)
    g = {k: v[..., envs].cpu().numpy() for k, v in out.items()}
    sub = scenes.Workload(wl.name, wl.models, wl.batch.take(envs), wl.options)
    refs = run_oracle(sub, list(range(len(envs))))
    assert sum(len(r["slots"]) > 0 for r in refs) >= 20
    _compare(sub, g, refs, list(range(len(envs))), tol_v, tol_j, min_checked=30)


@pytest.mark.parametrize("precision,tol_v,tol_j", [("fp64", 1e-9, 1e-9), ("mixed", 1e-4, 1e-3)])
def test_quadruped_full_size_sampled(torch_cuda, precision, tol_v, tol_j):
    """The 18-dof quadruped at 32768 envs in one call, sampled against the oracle."""
    import paper_2409_07107_gb300 as ds
    torch = torch_cuda
    B = 32768
    wl = scenes.quadruped_feet(B)
    sim = ds.Simulator(wl, precision=precision)
    out = sim.step_jac()
    torch.cuda.synchronize()
    envs = _sampled(B, 46, 12)
    g = {k: v[..., envs].cpu().numpy() for k, v in out.items()}
    sub = scenes.Workload(wl.name, wl.models, wl.batch.take(envs), wl.options)
    refs = run_oracle(sub, list(range(len(envs))))
    _compare(sub, g, refs, list(range(len(envs))), tol_v, tol_j, min_checked=30)


@pytest.mark.parametrize("precision,tol_v,tol_j", [("fp64", 1e-9, 1e-9), ("mixed", 1e-4, 1e-3)])
def test_uneven_full_size_sampled_vjp(torch_cuda, precision, tol_v, tol_j):
    """The mixed-robot batch at 32768 envs (arm + cube, quadruped, humanoid interleaved), step and
    VJP with N(0,1) cotangents in one call, sampled (a third of the samples from each model)
    against the oracle's J^T v_bar."""
    import paper_2409_07107_gb300 as ds
    torch = torch_cuda
    B = 32768
    wl = scenes.uneven(B)
    sim = ds.Simulator(wl, precision=precision)
    wbar = np.random.default_rng(13).normal(size=wl.batch.v.shape)
    out = sim.step_vjp(torch.as_tensor(wbar, dtype=torch.float64, device="cuda"))
    torch.cuda.synchronize()
    rng = np.random.default_rng(14)
    envs = sorted(set([0, 1, 2, B - 3, B - 2, B - 1] + [int(3 * k + r) for r in range(3)
                                                          for k in rng.choice(B // 3, 16, replace=False)]))
    g = {k: v[..., envs].cpu().numpy() for k, v in out.items()}
    sub = scenes.Workload(wl.name, wl.models, wl.batch.take(envs), wl.options)
    refs = run_oracle(sub, list(range(len(envs))))
    assert not (g["status"] & 16).any()
    _compare(sub, g, refs, list(range(len(envs))), tol_v, tol_j, jac=False, vjp=wbar[:, envs], min_checked=30)


def test_speculative_newton_attempts(torch_cuda):
    """From round 3 on (the default schedule) every env still iterating gets a Newton / active-set
    attempt on its iterate, with the contact-mode enumeration as fallback: the slow envs stop far
    earlier than with attempts only where a stage's tolerance is met, and they reach the same
    solutions (up to the documented non-unique ones)."""
    import paper_2409_07107_gb300 as ds
    torch = torch_cuda
    wl = scenes.arm_cube(8000)
    sim = ds.Simulator(wl, precision="fp64")
    sim.set_schedule(ds.schedule_index(spec=2, presolve=1))     # every env through the ADMM rounds
    try:
        ref = {k: v.clone() for k, v in sim.step_jac().items()}
        sim.set_schedule(ds.schedule_index(spec=0, presolve=1))
        got = {k: v.clone() for k, v in sim.step_jac().items()}
        torch.cuda.synchronize()
    finally:
        sim.set_schedule(-1)
    _same_solutions(ref, got)
    it_ref, it_got = ref["iters"].double(), got["iters"].double()
    assert it_got.mean().item() <= it_ref.mean().item()
    assert torch.quantile(it_got, 0.999).item() < torch.quantile(it_ref, 0.999).item(), (
        torch.quantile(it_got, 0.999).item(), torch.quantile(it_ref, 0.999).item())
    assert ((got["status"] & 1) != 0).sum().item() <= ((ref["status"] & 1) != 0).sum().item()


@pytest.mark.parametrize("precision,tol_v,tol_j", [("fp64", 1e-9, 1e-9), ("mixed", 1e-4, 1e-3)])
@pytest.mark.parametrize("pipeline", [True, False])
def test_pgs_solver(torch_cuda, precision, tol_v, tol_j, pipeline):
    """The projected Gauss-Seidel form of the NCP iteration (ncp_solver = DS_PGS), with the same
    Newton polish and FP64 residual acceptance: v+, modes and the Jacobians against the oracle
    (whose second route is PGS), in the pipeline (ragged batch of 300) and in the fused kernel."""
    import paper_2409_07107_gb300 as ds
    torch = torch_cuda
    wl = scenes.arm_cube(65536)
    sub = scenes.Workload(wl.name, wl.models, wl.batch.take(np.arange(300)), wl.options)
    sim = ds.Simulator(sub, precision=precision, pipeline=pipeline, ncp_solver=ds.DS_PGS)
    sim.set_schedule(ds.schedule_index(presolve=1))      # every env with contacts through the sweeps
    try:
        out = sim.step_jac()
        torch.cuda.synchronize()
    finally:
        sim.set_schedule(-1)
    g = {k: v.cpu().numpy() for k, v in out.items()}
    assert (g["iters"] > 0).sum() > 200
    envs = list(range(0, 300, 3))
    refs = run_oracle(sub, envs)
    _compare(sub, g, refs, envs, tol_v, tol_j, min_checked=60)
    if precision == "fp64":
        assert not (g["status"] & 1).any()


@pytest.mark.parametrize("precision,tol_v,tol_j", [("fp64", 1e-9, 1e-9), ("mixed", 1e-4, 1e-3)])
@pytest.mark.parametrize("pipeline", [True, False])
def test_adaptive_rho(torch_cuda, precision, tol_v, tol_j, pipeline):
    """The adaptive-penalty ADMM (admm_rho_adapt = 1: residual balancing of rho between rounds, K
    formed again): v+, modes and the Jacobians against the oracle (whose third route is the same
    variant, with its own update points), in the pipeline (ragged batch of 300, every env through
    the ADMM rounds) and in the fused kernel; the penalty changes the iterates (iteration counts
    differ from the fixed-rho run) but not the accepted solutions."""
    import paper_2409_07107_gb300 as ds
    torch = torch_cuda
    wl = scenes.arm_cube(65536)
    sub = scenes.Workload(wl.name, wl.models, wl.batch.take(np.arange(300)), wl.options)
    outs = []
    for adapt in (0, 1):
        sim = ds.Simulator(sub, precision=precision, pipeline=pipeline, admm_rho_adapt=adapt)
        sim.set_schedule(ds.schedule_index(presolve=1))
        try:
            out = sim.step_jac()
            torch.cuda.synchronize()
        finally:
            sim.set_schedule(-1)
        outs.append({k: v.cpu().numpy() for k, v in out.items()})
    fixed, g = outs
    assert (g["iters"] != fixed["iters"]).sum() >= 20
    envs = list(range(0, 300, 3))
    refs = run_oracle(sub, envs, routes=("admm", "pgs", "admm_adaptive"))
    _compare(sub, g, refs, envs, tol_v, tol_j, min_checked=60)
    if precision == "fp64":
        assert not (g["status"] & 1).any()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_single_contact_presolve(torch_cuda, precision):
    """The setup's exact solve for single-contact solutions (default schedule) against the same
    step with every env through the ADMM rounds: most arm + cube envs are presolved (no ADMM
    iteration), and both reach the same solutions (up to the documented non-unique ones); the
    presolved envs also match the oracle."""
    import paper_2409_07107_gb300 as ds
    torch = torch_cuda
    wl = scenes.arm_cube(4000)
    sim = ds.Simulator(wl, precision=precision)
    sim.set_schedule(ds.schedule_index(presolve=1))
    try:
        ref = {k: v.clone() for k, v in sim.step_jac().items()}
        sim.set_schedule(ds.schedule_index(presolve=0))
        got = {k: v.clone() for k, v in sim.step_jac().items()}
        torch.cuda.synchronize()
    finally:
        sim.set_schedule(-1)
    if precision == "fp64":
        _same_solutions(ref, got)
    else:
        scale = ref["v_next"].abs().amax(0).clamp_min(1e-6)
        same = ((got["v_next"] - ref["v_next"]).abs().amax(0) / scale) <= 1e-4
        assert same.float().mean().item() >= 0.995
    pre = (got["iters"] == 0) & ((got["modes"] != 3).any(0))
    assert pre.float().mean().item() >= 0.6, pre.float().mean().item()
    envs = [int(e) for e in torch.nonzero(pre).flatten()[:40].cpu()]
    g = {k: v[..., envs].cpu().numpy() for k, v in got.items()}
    sub = scenes.Workload(wl.name, wl.models, wl.batch.take(envs), wl.options)
    refs = run_oracle(sub, list(range(len(envs))))
    tol_v, tol_j = (1e-9, 1e-9) if precision == "fp64" else (1e-4, 1e-3)
    _compare(sub, g, refs, list(range(len(envs))), tol_v, tol_j, min_checked=25)


def _rel_per_env(got, ref):
    axes = tuple(range(got.ndim - 1))
    return (got - ref).abs().amax(axes) / ref.abs().amax(axes).clamp_min(1e-6)


@pytest.mark.parametrize("name,B", [("arm_cube", 600), ("humanoid_feet", 300), ("quadruped_feet", 300)])
@pytest.mark.parametrize("precision,tol_v,tol_j,tol_same", [("fp64", 1e-9, 1e-9, 1e-8), ("mixed", 1e-4, 1e-3, 1e-3)])
def test_split_finish(torch_cuda, name, B, precision, tol_v, tol_j, tol_same):
    """The finish as a prep kernel and a column kernel (schedule finish = split: one warp per env,
    its state in shared memory, the columns over the lanes).  The step's outputs are the one-kernel
    finish's exactly (same solve, same F9); the Jacobians agree with it to rounding (the implicit
    part applied by rows, in FP32 in the mixed form) and with the oracle on sampled envs."""
    import paper_2409_07107_gb300 as ds
    torch = torch_cuda
    wl = getattr(scenes, name)(B)
    sim = ds.Simulator(wl, precision=precision)
    ref = {k: v.clone() for k, v in sim.step_jac().items()}
    sim.set_schedule(ds.schedule_index(split=1))
    try:
        got = {k: v.clone() for k, v in sim.step_jac().items()}
        torch.cuda.synchronize()
    finally:
        sim.set_schedule(-1)
    for key in ("v_next", "modes", "status", "iters"):
        assert torch.equal(got[key], ref[key]), key
    ok = (ref["status"] & 2) == 0
    for key in ("dv_dq", "dv_dv", "dv_dtau"):
        err = _rel_per_env(got[key], ref[key])[ok]
        assert err.max().item() <= tol_same, (key, err.max().item())
    envs = list(range(0, B, max(1, B // 40)))
    g = {k: v.cpu().numpy() for k, v in got.items()}
    refs = run_oracle(wl, envs)
    _compare(wl, g, refs, envs, tol_v, tol_j, min_checked=max(10, len(envs) // 3))


@pytest.mark.parametrize("precision,tol_same", [("fp64", 1e-8), ("mixed", 1e-3)])
def test_split_finish_vjp(torch_cuda, precision, tol_same):
    """The split finish under sim_step_vjp on the mixed-robot batch (each model's pipeline): q_bar,
    v_bar, tau_bar against the one-kernel finish's, with a cotangent of q+ as well."""
    import paper_2409_07107_gb300 as ds
    torch = torch_cuda
    wl = scenes.uneven(300)
    sim = ds.Simulator(wl, precision=precision)
    rng = np.random.default_rng(41)
    vb = torch.as_tensor(rng.normal(size=wl.batch.v.shape), dtype=torch.float64, device="cuda")
    qb = torch.as_tensor(rng.normal(size=wl.batch.v.shape), dtype=torch.float64, device="cuda")
    ref = {k: v.clone() for k, v in sim.step_vjp(vb, q_next_bar=qb).items()}
    sim.set_schedule(ds.schedule_index(split=1), "vjp")
    try:
        got = {k: v.clone() for k, v in sim.step_vjp(vb, q_next_bar=qb).items()}
        torch.cuda.synchronize()
    finally:
        sim.set_schedule(-1, "vjp")
    for key in ("v_next", "modes", "status"):
        assert torch.equal(got[key], ref[key]), key
    ok = (ref["status"] & 2) == 0
    for key in ("q_bar", "v_bar", "tau_bar"):
        err = _rel_per_env(got[key], ref[key])[ok]
        assert err.max().item() <= tol_same, (key, err.max().item())


@pytest.mark.parametrize("field,value", [("queue_poll_limit", -1), ("admm_rho_adapt", 2), ("ncp_solver", 7),
                                         ("contact_margin", -1e-3), ("baumgarte_kp", float("nan"))])
def test_option_validation(torch_cuda, field, value):
    """Out-of-range options are refused by the call (DS_EINVAL) before any kernel runs; the next call
    with valid options works."""
    import paper_2409_07107_gb300 as ds
    torch = torch_cuda
    wl = scenes.arm_sphere(16)
    bad = ds.Simulator(wl, precision="fp64", **{field: value})
    with pytest.raises(ds.DiffsimError, match="invalid"):
        bad.step()
    good = ds.Simulator(wl, precision="fp64")
    good.step()
    torch.cuda.synchronize()
    assert not (good.out["status"] & 2).any()
