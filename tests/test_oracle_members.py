"""Which results of the step are unique when Eq. 1 has several solutions (oracle only, no GPU).

The GPU parity tests compare the CUDA path with the oracle's solutions; they rely on the facts
pinned here:

* on the benchmark workloads, two independent routes of the oracle (ADMM and projected
  Gauss-Seidel, each with the Newton polish) and a third with other ADMM parameters (the penalty,
  relaxation and test interval of the GPU kernels) reach the same v+, modes and Jacobians on (almost)
  every env, so these do not depend on the solver;
* on a rigid box resting on four coplanar corners (statically indeterminate), the impulses are not
  unique; v+ and the Jacobians still are while the box slides without turning or sticks, but not
  when it slides while turning (each corner's friction then points its own way, so the friction
  wrench depends on how the normal impulse is shared);
* where the free motion separates every contact, lambda = 0 solves Eq. 1, and the oracle takes it,
  although the relaxed ADMM can land on another solution there.
"""
import multiprocessing as mp
import types

import numpy as np
import pytest

from oracle import ncp
from oracle import step as S
from paper_2409_07107_gb300 import scenes
from tests.helpers import point_mass_model
from tests.oracle_runner import jac_of, rel_err

KERNEL_LIKE = (0.3, 1.6, 4)      # rho scale, relaxation, test interval of the GPU's ADMM


def _solve(model, env, opt, route, params=None):
    o = types.SimpleNamespace(**dict(vars(opt), ncp_route=route))
    old = (ncp.RHO_SCALE, ncp.RELAX, ncp.CHECK_EVERY)
    if params is not None:
        ncp.RHO_SCALE, ncp.RELAX, ncp.CHECK_EVERY = params
    try:
        return S.step_jac(model, env, o)
    finally:
        ncp.RHO_SCALE, ncp.RELAX, ncp.CHECK_EVERY = old


def _three_routes(args):
    model, env, opt = args
    outs = [_solve(model, env, opt, "admm"), _solve(model, env, opt, "pgs"),
            _solve(model, env, opt, "admm", KERNEL_LIKE)]
    ref = outs[0]
    same = all(rel_err(o["v_next"], ref["v_next"]) <= 1e-9 and list(o["modes"]) == list(ref["modes"])
               and rel_err(jac_of(o), jac_of(ref)) <= 1e-9 for o in outs[1:])
    return same, len(ref["slots"]), [int(x) for x in ref["modes"]]


@pytest.mark.slow
@pytest.mark.parametrize("name,B,n,need", [("arm7-cube", 4096, 32, 32), ("quadruped18-feet", 4096, 16, 16),
                                           ("humanoid36-feet", 16384, 8, 8)])
def test_routes_agree_on_workloads(name, B, n, need):
    wl = scenes.WORKLOADS[name](B)
    m = wl.models[0]
    envs = list(range(n))
    args = [(m, wl.batch.env(e, m), wl.options) for e in envs]
    with mp.get_context("spawn").Pool(min(8, n)) as pool:
        res = pool.map(_three_routes, args)
    agree = sum(r[0] for r in res)
    assert agree >= need, [(e, r) for e, r in zip(envs, res) if not r[0]]


def _box(vlin, w, mu=0.5):
    """A free box (2 kg) with its four bottom corners 0.1 mm into the plane."""
    m = point_mass_model(2.0, (0.02, 0.03, 0.04))
    h = 0.05
    corners = np.array([(sx * h, sy * h, -h) for sx in (1, -1) for sy in (1, -1)])
    env = dict(q=np.array([0.0, 0.0, 0.3, 1.0, 0.0, 0.0, 0.0]), v=np.concatenate([vlin, w]), tau=np.zeros(6),
               c_link=np.zeros(4, np.int32), c_point=corners, c_radius=np.zeros(4), c_mu=np.full(4, mu),
               plane=np.array([0.0, 0.0, 1.0, 0.3 - h + 1e-4]))
    return m, env


@pytest.mark.parametrize("vlin,w,unique_v", [((1.0, 0.0, -0.2), (0.0, 0.0, 0.0), True),
                                             ((0.01, 0.0, -0.2), (0.0, 0.0, 0.0), True),
                                             ((1.0, 0.3, -0.2), (0.0, 0.0, 2.0), False)])
def test_box_on_four_corners(vlin, w, unique_v):
    m, env = _box(np.array(vlin), np.array(w))
    opt = scenes.Options()
    a, b = _solve(m, env, opt, "admm"), _solve(m, env, opt, "pgs")
    scale = max(1.0, np.abs(a["g"]).max())
    for r in (a, b):
        assert r["converged"] and ncp.ncp_residual(r["G"], r["g"], r["mu"], r["lam"]) <= 1e-12 * scale
    assert np.linalg.matrix_rank(a["G"], tol=1e-9) == 6          # 12 unknowns, rank 6
    assert np.abs(a["lam"] - b["lam"]).max() > 1e-3             # the impulses differ
    assert list(a["modes"]) == list(b["modes"])
    if unique_v:
        assert rel_err(a["v_next"], b["v_next"]) <= 1e-9
        assert rel_err(jac_of(a), jac_of(b)) <= 1e-9
    else:
        assert all(int(x) == ncp.SLD for x in a["modes"])
        assert rel_err(a["v_next"], b["v_next"]) > 1e-4


def test_separating_contacts_take_zero_impulse():
    """A humanoid env whose two active foot corners both separate under the free motion: lambda = 0
    solves Eq. 1 and is returned; the relaxed ADMM reaches a different solution with a sticking
    corner and a large impulse, which satisfies Eq. 1 as well."""
    wl = scenes.humanoid_feet(64)
    m = wl.models[0]
    st = S.step(m, wl.batch.env(12, m), wl.options)
    G, g, mu = st["G"], st["g"], st["mu"]
    assert len(mu) == 2 and ncp.separating(g)
    assert np.all(st["lam"] == 0.0) and st["iters"] == 0
    old = (ncp.RHO_SCALE, ncp.RELAX, ncp.CHECK_EVERY)
    ncp.RHO_SCALE, ncp.RELAX, ncp.CHECK_EVERY = KERNEL_LIKE
    try:
        lam, it, conv, _ = ncp.admm(G, g, mu, eps=1e-13, max_iter=100000)
    finally:
        ncp.RHO_SCALE, ncp.RELAX, ncp.CHECK_EVERY = old
    scale = max(1.0, np.abs(g).max())
    assert conv and ncp.ncp_residual(G, g, mu, lam) <= 1e-10 * scale
    assert np.abs(lam).max() > 0.1
