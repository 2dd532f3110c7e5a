"""Pins of the oracle's projected Gauss-Seidel solve of Eq. 1 (the solver family the paper cites
next to ADMM), the reference for a PGS variant of the NCP stage (no GPU).

* one contact: the PGS solution is one of the solutions found by enumerating the three modes
  (ncp.brute_force_single) and satisfies Eq. 1;
* point mass on a plane (G = I/m): the closed-form impulse of each mode;
* arm + cube samples (four redundant corner contacts, lambda not unique): the NCP residual is at
  the solver tolerance and sigma = G lambda + g, which is unique, equals the staged ADMM + Newton
  solution's.
"""
import numpy as np
import pytest

from oracle import ncp, rigid
from oracle.contact import active_slots, contact_jacobian
from paper_2409_07107_gb300 import scenes


def test_single_contact_brute_force():
    rng = np.random.default_rng(12)
    for _ in range(40):
        A = rng.normal(size=(3, 3))
        G = A @ A.T + 0.1 * np.eye(3)
        g, mu = rng.normal(size=3), rng.uniform(0.2, 1.0)
        lam, sweeps, ok = ncp.pgs(G, g, np.array([mu]), eps=1e-14, max_iter=200000)
        assert ok
        assert ncp.ncp_residual(G, g, np.array([mu]), lam) < 1e-10
        sols = ncp.brute_force_single(G, g, mu, n_angles=48)
        assert any(np.allclose(lam, l, atol=1e-8 * max(1, np.abs(l).max())) for _, l in sols)


@pytest.mark.parametrize("case", ["brk", "stk", "sld"])
def test_point_mass_closed_form(case):
    mass, mu = 2.0, 0.5
    G = np.eye(3) / mass
    vf = {"brk": np.array([0.3, 0.1, 0.5]), "stk": np.array([0.05, -0.02, -0.5]),
          "sld": np.array([1.0, 0.5, -0.3])}[case]
    lam, _, ok = ncp.pgs(G, vf.copy(), np.array([mu]), eps=1e-15)
    assert ok
    if case == "brk":
        expect = np.zeros(3)
    elif case == "stk":
        expect = -mass * vf
    else:
        u = vf[:2] / np.linalg.norm(vf[:2])
        ln = -mass * vf[2]
        expect = np.array([-mu * ln * u[0], -mu * ln * u[1], ln])
    assert np.allclose(lam, expect, atol=1e-12)


def test_arm_cube_matches_staged_solve():
    wl = scenes.arm_cube(40)
    m, opt = wl.models[0], wl.options
    n = 0
    for e in range(40):
        env = wl.batch.env(e, m)
        q, v, tau = env["q"], env["v"], env["tau"]
        slots = active_slots(m, q, env)
        if not slots:
            continue
        M = rigid.crba(m, q)
        vf = v + opt.dt * rigid.aba(m, q, v, tau, np.asarray(opt.gravity, float))
        Jc = contact_jacobian(m, q, env, slots)
        mu = np.array([env["c_mu"][k] for k in slots])
        G = Jc @ rigid.chol_solve(rigid.cholesky(M), Jc.T)
        g = Jc @ vf
        lp, _, ok = ncp.pgs(G, g, mu, eps=1e-13, max_iter=50000)
        la, _, oka = ncp.solve_ncp(G, g, mu)
        if not (ok and oka):
            continue
        scale = max(1.0, np.max(np.abs(g)))
        assert ncp.ncp_residual(G, g, mu, lp) <= 1e-10 * scale
        assert np.max(np.abs((G @ lp + g) - (G @ la + g))) <= 1e-9 * scale
        n += 1
    assert n >= 20
