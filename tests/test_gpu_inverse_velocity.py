"""Gauss-Newton estimation of an initial velocity (Sec. 4, Eq. init_id) on the GPU: cubes thrown
onto the floor in a sliding mode, their planar initial velocities (x, y, yaw rate) recovered from
the configurations their 12-step rollouts reach, against the oracle's own Gauss-Newton loop.  The
cube rests on three points of its bottom face so that the step is unique (on four corners the
normal impulse split, and with it the turning response, is statically indeterminate)."""
import multiprocessing as mp

import numpy as np
import pytest

from paper_2409_07107_gb300 import scenes
from tests.helpers import point_mass_model

pytestmark = pytest.mark.gpu

H = 0.025
T = 12
FREE = [0, 1, 5]


def _cube_workload(B, rng, mu=0.3, pen=1e-4):
    mass = 1.0
    ii = mass * (2 * H) ** 2 / 6.0
    m = point_mass_model(mass, (ii, ii, ii))
    corners = np.array([[-H, -H, -H], [H, -H, -H], [0.0, H, -H], [0.0, 0.0, 0.0]])
    nc = len(corners)                                   # the fourth slot is unused (the kernel has 4)
    q = np.tile(np.array([0.0, 0.0, H - pen, 1.0, 0.0, 0.0, 0.0])[:, None], (1, B))
    v_true = np.zeros((6, B))
    v_true[0] = rng.uniform(0.6, 1.2, B)
    v_true[1] = rng.uniform(-0.5, 0.5, B)
    v_true[5] = rng.uniform(-0.6, 0.6, B)
    c_link = np.zeros((nc, B), np.int32)
    c_link[3] = -1
    batch = scenes.Batch(q, np.zeros((6, B)), np.zeros((6, B)), c_link,
                         np.repeat(corners[:, :, None], B, axis=2), np.zeros((nc, B)), np.full((nc, B), mu),
                         np.tile(np.array([0.0, 0.0, 1.0, 0.0])[:, None], (1, B)))
    return scenes.Workload("cube3", [m], batch), v_true


def _oracle_target(args):
    from oracle import inverse as INV
    m, env, v_true, opt = args
    return INV.rollout_q(m, dict(env, v=v_true), T, opt)


def _oracle(args):
    from oracle import inverse as INV
    m, env, q_target, v_init, opt = args
    v0, hist = INV.estimate_initial_velocity(m, env, q_target, T, opt, v_init, iters=12, tol=1e-13, free=FREE)
    return v0


def test_initial_velocity_estimation_matches_oracle():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2409_07107_gb300 as ds
    from paper_2409_07107_gb300 import build, rollout as R
    from paper_2409_07107_gb300.inverse import gauss_newton_initial_velocity
    build.build()
    ds.lib()
    B = 6
    rng = np.random.default_rng(31)
    wl, v_true = _cube_workload(B, rng)
    m = wl.models[0]
    dev = dict(dtype=torch.float64, device="cuda")
    sc = R.StepContext(wl, precision="fp64")
    q0 = torch.tensor(wl.batch.q, **dev)
    taus = [torch.zeros(6, B, **dev) for _ in range(T)]
    with mp.get_context("spawn").Pool(B) as pool:
        qt = np.stack(pool.map(_oracle_target, [(m, wl.batch.env(e, m), v_true[:, e], wl.options) for e in range(B)]), 1)
    q_target = torch.tensor(qt, **dev)              # the configurations the oracle's rollouts reach
    v_init = v_true.copy()
    v_init[FREE] += rng.normal(0.0, 0.05, size=(3, B))
    v0, hist = gauss_newton_initial_velocity(sc, q0, torch.tensor(v_init, **dev), q_target, taus, FREE, iters=12,
                                             tol=1e-13)
    v0 = v0.cpu().numpy()
    assert hist[-1] <= 1e-12 and len(hist) <= 10, hist
    assert np.abs(v0 - v_true).max() <= 1e-8
    with mp.get_context("spawn").Pool(B) as pool:
        refs = pool.map(_oracle, [(m, wl.batch.env(e, m), qt[:, e], v_init[:, e], wl.options) for e in range(B)])
    for e in range(B):
        assert np.abs(v0[:, e] - refs[e]).max() <= 1e-8, e
