"""Pins of the oracle's adaptive-penalty ADMM route (residual balancing of rho, the ADMM variant
next to PGS among the solver alternatives of Sec. 2.2), the reference for the kernels' option of
the same name (no GPU).

* the balancing rule: a primal residual ten times the dual one doubles rho, the reverse halves
  it, anything in between keeps it (the rule written out on numbers);
* the fixed points do not move with rho: a solution of Eq. 1 with y = -(sigma + Gamma(sigma))
  is left unchanged by iterations at any penalty, and both residuals vanish there;
* one contact: the route's solution is one of the enumerated solutions (brute force) and
  satisfies Eq. 1; point mass: the closed-form impulse of each mode;
* arm + cube samples: the NCP residual meets the acceptance tolerance and sigma = G lambda + g
  (unique even where lambda is not) equals the plain route's; and on an ill-scaled problem (rho
  far from the Delassus scale) the penalty actually changes.
"""
import numpy as np
import pytest

from oracle import ncp, rigid
from oracle.contact import active_slots, contact_jacobian
from paper_2409_07107_gb300 import scenes


def test_balancing_rule():
    assert ncp.balance_rho(3.0, 1.0, 0.05) == 6.0
    assert ncp.balance_rho(3.0, 0.05, 1.0) == 1.5
    assert ncp.balance_rho(3.0, 1.0, 0.2) == 3.0
    assert ncp.balance_rho(3.0, 0.2, 1.0) == 3.0


def test_fixed_point_independent_of_rho():
    mass, mu = 2.0, 0.5
    G = np.eye(3) / mass
    vf = np.array([1.0, 0.5, -0.3])                      # sliding: closed form below
    u = vf[:2] / np.linalg.norm(vf[:2])
    ln = -mass * vf[2]
    lam = np.array([-mu * ln * u[0], -mu * ln * u[1], ln])
    sigma = G @ lam + vf
    st = ncp.AdmmState(3, vf)
    st.x, st.z, st.sx = lam.copy(), lam.copy(), sigma.copy()
    st.y = -(sigma + ncp.desaxce(sigma, np.array([mu])))
    assert max(ncp.admm_residuals(st.x, st.z, st.y, st.sx, np.array([mu]))) <= 1e-15
    for rho in (1e-3, 0.5, 40.0):
        st.rho = rho
        out, _, _, st = ncp.admm(G, vf, np.array([mu]), eps=0.0, max_iter=st.iters + 64, state=st, adapt=True)
        assert np.allclose(out, lam, atol=1e-13), rho


def test_single_contact_brute_force():
    rng = np.random.default_rng(31)
    for _ in range(30):
        A = rng.normal(size=(3, 3))
        G = A @ A.T + 0.1 * np.eye(3)
        g, mu = rng.normal(size=3), rng.uniform(0.2, 1.0)
        lam, _, ok = ncp.solve_ncp(G, g, np.array([mu]), route="admm_adaptive")
        assert ok
        assert ncp.ncp_residual(G, g, np.array([mu]), lam) <= 1e-12 * max(1.0, np.abs(g).max())
        sols = ncp.brute_force_single(G, g, mu, n_angles=48)
        assert any(np.allclose(lam, l, atol=1e-8 * max(1, np.abs(l).max())) for _, l in sols)


@pytest.mark.parametrize("case", ["stk", "sld"])
def test_point_mass_closed_form(case):
    mass, mu = 2.0, 0.5
    G = np.eye(3) / mass
    vf = {"stk": np.array([0.05, -0.02, -0.5]), "sld": np.array([1.0, 0.5, -0.3])}[case]
    lam, _, ok = ncp.solve_ncp(G, vf.copy(), np.array([mu]), route="admm_adaptive")
    assert ok
    if case == "stk":
        expect = -mass * vf
    else:
        u = vf[:2] / np.linalg.norm(vf[:2])
        ln = -mass * vf[2]
        expect = np.array([-mu * ln * u[0], -mu * ln * u[1], ln])
    assert np.allclose(lam, expect, atol=1e-12)


def _arm_cube_problems(n_env):
    wl = scenes.arm_cube(n_env)
    m, opt = wl.models[0], wl.options
    for e in range(n_env):
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
        yield G, Jc @ vf, mu


def test_arm_cube_matches_plain_route():
    n = 0
    for G, g, mu in _arm_cube_problems(40):
        la, _, oka = ncp.solve_ncp(G, g, mu, route="admm_adaptive")
        lp, _, okp = ncp.solve_ncp(G, g, mu)
        if not (oka and okp):
            continue
        scale = max(1.0, np.max(np.abs(g)))
        assert ncp.ncp_residual(G, g, mu, la) <= 1e-12 * scale
        assert np.max(np.abs((G @ la + g) - (G @ lp + g))) <= 1e-9 * scale
        n += 1
    assert n >= 20


def test_penalty_moves_on_an_ill_scaled_start():
    G, g, mu = next(p for p in _arm_cube_problems(40) if not ncp.separating(p[1]))
    st = ncp.AdmmState(len(g), g)
    st.rho = 1e-4 * ncp.admm_rho(G)                      # far below the Delassus scale
    lam, _, _, st = ncp.admm(G, g, mu, eps=1e-10, max_iter=4096, state=st, adapt=True)
    assert st.rho > 1e-4 * ncp.admm_rho(G)
