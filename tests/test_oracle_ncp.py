"""Pins of the oracle's NCP solve against the cone geometry, brute force and closed forms (no GPU)."""
import numpy as np
import pytest

from oracle import ncp, rigid
from oracle import step as S
from paper_2409_07107_gb300 import scenes
from tests.helpers import point_mass_model


def test_cone_projection_moreau():
    """Proj_K(x) - x is in the polar cone -K^* and orthogonal to Proj_K(x); idempotent."""
    rng = np.random.default_rng(0)
    for _ in range(200):
        x = rng.normal(size=3) * rng.uniform(0.1, 3)
        mu = rng.uniform(0.1, 1.5)
        p = ncp.proj_cone(x, mu)
        assert np.linalg.norm(p[:2]) <= mu * p[2] + 1e-12
        assert np.allclose(ncp.proj_cone(p, mu), p, atol=1e-12)
        w = p - x                                     # must lie in K^* = K_{1/mu}
        assert np.linalg.norm(w[:2]) <= w[2] / mu + 1e-12
        assert abs(p @ w) <= 1e-12 * max(1, x @ x)


def test_cone_projection_is_nearest_point():
    rng = np.random.default_rng(1)
    for _ in range(50):
        x = rng.normal(size=3)
        mu = rng.uniform(0.2, 1.0)
        p = ncp.proj_cone(x, mu)
        for _ in range(200):
            yt = rng.normal(size=2)
            y = np.array([yt[0], yt[1], np.linalg.norm(yt) / mu * rng.uniform(1, 3)]) * rng.uniform(0, 2)
            assert np.linalg.norm(x - p) <= np.linalg.norm(x - y) + 1e-12


def _random_single(rng):
    A = rng.normal(size=(3, 3))
    G = A @ A.T + 0.1 * np.eye(3)
    return G, rng.normal(size=3), rng.uniform(0.2, 1.0)


def test_single_contact_brute_force():
    """One contact: every mode is enumerated; the staged ADMM solution is one of the enumerated
    solutions and satisfies Eq. 1."""
    rng = np.random.default_rng(2)
    found = {ncp.BRK: 0, ncp.STK: 0, ncp.SLD: 0}
    for _ in range(40):
        G, g, mu = _random_single(rng)
        sols = ncp.brute_force_single(G, g, mu, n_angles=48)
        lam, _, ok = ncp.solve_ncp(G, g, np.array([mu]))
        assert ok
        assert ncp.ncp_residual(G, g, np.array([mu]), lam) < 1e-11
        assert any(np.allclose(lam, l, atol=1e-8 * max(1, np.abs(l).max())) for _, l in sols)
        for md, l in sols:
            assert ncp.ncp_residual(G, g, np.array([mu]), l) < 1e-9
        if len(sols) == 1:
            found[sols[0][0]] += 1
    assert all(v > 0 for v in found.values())


def _pm_env(vlin, mu, mass=2.0, pen=1e-4):
    m = point_mass_model(mass)
    q = np.array([0.1, -0.2, 0.3, 1.0, 0.0, 0.0, 0.0])
    env = dict(q=q, v=np.concatenate([vlin, np.zeros(3)]), tau=np.zeros(6), c_link=np.array([0]),
               c_point=np.zeros((1, 3)), c_radius=np.zeros(1), c_mu=np.array([mu]),
               plane=np.array([0.0, 0.0, 1.0, 0.3 + pen]))
    return m, env


@pytest.mark.parametrize("case", ["brk", "stk", "sld"])
def test_point_mass_closed_form(case):
    """Point mass on a plane (contact at the centre of mass, no rotation): G = I/m and Eq. 1 has
    the closed-form solution of each mode, including the sliding derivative of App. A."""
    mass, dt, mu = 2.0, 1e-3, 0.5
    vlin = {"brk": np.array([0.3, 0.1, 0.5]), "stk": np.array([0.05, -0.02, -0.5]),
            "sld": np.array([1.0, 0.5, -0.3])}[case]
    m, env = _pm_env(vlin, mu, mass)
    opt = scenes.Options()
    st = S.step_jac(m, env, opt)
    assert np.allclose(st["G"], np.eye(3) / mass, atol=1e-14)
    vf = vlin + dt * np.array([0, 0, -9.81])
    vn = st["v_next"][:3]
    J = st["dv_dv"][:3, :3]
    if case == "brk":
        assert list(st["modes"]) == [ncp.BRK]
        assert np.allclose(vn, vf, atol=1e-14)
        Jexp = np.eye(3)
    elif case == "stk":
        assert list(st["modes"]) == [ncp.STK]
        assert np.allclose(vn, 0, atol=1e-13)
        assert np.allclose(st["lam"], -mass * vf, atol=1e-12)
        Jexp = np.zeros((3, 3))
    else:
        assert list(st["modes"]) == [ncp.SLD]
        vt, vN = vf[:2], vf[2]
        u = vt / np.linalg.norm(vt)
        assert np.allclose(vn[:2], vt + mu * vN * u, atol=1e-13)
        assert abs(vn[2]) < 1e-13
        Jexp = np.zeros((3, 3))
        Jexp[:2, :2] = np.eye(2) - mu * (-vN) / np.linalg.norm(vt) * (np.eye(2) - np.outer(u, u))
        Jexp[:2, 2] = mu * u
    assert np.allclose(J, Jexp, atol=1e-10)
    assert np.allclose(st["dv_dtau"][:3, :3], Jexp * dt / mass, atol=1e-12)


def test_sliding_Q_identity():
    """Q = R^T Ktilde R = diag(0, 1) with Ktilde = [[I2, mu u], [0 0 0]] (App. A)."""
    rng = np.random.default_rng(4)
    for _ in range(100):
        mu = rng.uniform(0.1, 1.5)
        st = rng.normal(size=2)
        u = st / np.linalg.norm(st)
        lam = rng.uniform(0.1, 2) * np.array([-mu * u[0], -mu * u[1], 1.0])
        sigma = np.array([st[0], st[1], 0.0])
        R, P, Q = S.sliding_basis(lam, sigma, mu)
        Kt = np.zeros((3, 3))
        Kt[:2, :2] = np.eye(2)
        Kt[:2, 2] = mu * u
        assert np.allclose(R.T @ Kt @ R, np.diag([0.0, 1.0]), atol=1e-14)
        assert np.allclose(Q, np.diag([0.0, 1.0]))


def _sample_envs(wl, n):
    m = wl.models[0]
    return [(m, wl.batch.env(e, m)) for e in range(n)]


def test_arm_cube_ncp_solutions():
    """Arm + cube (4 redundant corners): every solution satisfies Eq. 1 to 1e-12."""
    wl = scenes.arm_cube(64)
    for m, env in _sample_envs(wl, 16):
        st = S.step(m, env, wl.options)
        assert st["converged"]
        assert st["residual"] <= 1e-12 * max(1, np.abs(st["g"]).max())


def test_all_sticking_projection():
    """All contacts sticking => v+ = v_f - Y G^+ g: the M-orthogonal projection of the free
    velocity onto ker J_c (a bilateral constraint, Sec. 3.2)."""
    wl = scenes.quadruped_feet(24)
    opt = wl.options
    n = 0
    for m, env in _sample_envs(wl, 12):
        env["v"] = np.zeros(m.nv)
        env["v"][2] = -0.3          # the base drops onto its 4 feet
        env["tau"] = np.zeros(m.nv)
        st = S.step(m, env, opt)
        if len(st["slots"]) and all(md == ncp.STK for md in st["modes"]):
            vp = st["v_f"] - st["Y"] @ np.linalg.pinv(st["G"], rcond=1e-12) @ st["g"]
            assert np.allclose(st["v_next"], vp, atol=1e-10 * max(1, np.abs(vp).max()))
            assert np.allclose(st["Jc"] @ st["v_next"], 0, atol=1e-10)
            n += 1
    assert n >= 3


def test_no_contact_derivatives():
    """No contact: dv+/dtau = dt M^-1 and dv+/dv = I - dt M^-1 db/dv (RNEA, complex step)."""
    wl = scenes.arm_sphere(16)
    m = wl.models[0]
    opt = wl.options
    G = np.array(opt.gravity)
    done = 0
    for e in range(16):
        env = wl.batch.env(e, m)
        st = S.step_jac(m, env, opt)
        if st["slots"]:
            continue
        Minv = np.linalg.inv(rigid.crba(m, env["q"]))
        assert np.allclose(st["dv_dtau"], opt.dt * Minv, atol=1e-12 * np.abs(Minv).max())
        h = 1e-30
        db = np.stack([np.imag(rigid.rnea(m, env["q"], env["v"] + 1j * h * ek, np.zeros(7), G)) / h
                       for ek in np.eye(7)], 1)
        assert np.allclose(st["dv_dv"], np.eye(7) - opt.dt * Minv @ db, atol=1e-12)
        done += 1
    assert done >= 3
