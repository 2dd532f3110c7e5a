"""Pins of the oracle's Baumgarte-stabilised step (App. D): g gains phi/dt - K_p [phi/dt]_- -
K_d (J_c v)_N on each active contact's normal row (no GPU).

* the gains K_p = 1, K_d = 0 leave g = J_c v_f exactly (the unstabilised step);
* closed form: for a point mass on a plane (contact at the centre of mass, world-aligned frame) a
  sticking or sliding contact satisfies (J_c v+)_N = K_d (J_c v)_N - (1 - K_p) phi / dt (App. D),
  so v+_z, dv+_z / dv_z = K_d and dv+_z / dq_z = -(1 - K_p) / dt are known in closed form, and the
  sliding tangent velocity follows from the impulse the normal row needs;
* the route-1 Jacobian (App. B system with the Baumgarte terms in its right-hand side) equals
  direct implicit differentiation (route 2, sigma = J_c v+ + the Baumgarte term) and central finite
  differences of the whole step.
"""
import types

import numpy as np
import pytest

from oracle import ncp
from oracle import step as S
from paper_2409_07107_gb300 import scenes
from tests.helpers import point_mass_model


def _with_gains(opt, kp, kd):
    d = {k: getattr(opt, k) for k in ("dt", "gravity", "admm_max_iter", "admm_eps", "polish_iters", "eps_sigma",
                                     "eps_lambda")}
    return types.SimpleNamespace(**d, baumgarte_kp=kp, baumgarte_kd=kd)


def test_unit_gains_leave_the_step_unchanged():
    wl = scenes.arm_cube(8)
    m = wl.models[0]
    for e in range(4):
        env = wl.batch.env(e, m)
        a = S.step(m, env, wl.options)
        b = S.step(m, env, _with_gains(wl.options, 1.0, 0.0))
        assert np.array_equal(a["g"], b["g"]) and np.array_equal(a["g"], a["Jc"] @ a["v_f"])
        assert np.array_equal(a["v_next"], b["v_next"])


def _pm_env(vlin, mu, mass, pen):
    m = point_mass_model(mass)
    q = np.array([0.1, -0.2, 0.3, 1.0, 0.0, 0.0, 0.0])
    env = dict(q=q, v=np.concatenate([vlin, np.zeros(3)]), tau=np.zeros(6), c_link=np.array([0]),
               c_point=np.zeros((1, 3)), c_radius=np.zeros(1), c_mu=np.array([mu]),
               plane=np.array([0.0, 0.0, 1.0, 0.3 + pen]))
    return m, env


@pytest.mark.parametrize("case", ["stk", "sld"])
@pytest.mark.parametrize("kp,kd", [(0.0, 0.0), (0.6, 0.3), (1.0, 0.5)])
def test_point_mass_closed_form(case, kp, kd):
    mass, mu, pen = 2.0, 0.5, 2e-4
    vlin = {"stk": np.array([0.05, -0.02, -0.5]), "sld": np.array([1.0, 0.5, -0.3])}[case]
    m, env = _pm_env(vlin, mu, mass, pen)
    opt = _with_gains(scenes.Options(), kp, kd)
    dt = opt.dt
    phi = -pen
    st = S.step_jac(m, env, opt)
    vf = vlin + dt * np.array([0.0, 0.0, -9.81])
    vn = st["v_next"][:3]
    vz = kd * vlin[2] - (1.0 - kp) * phi / dt
    assert abs(vn[2] - vz) < 1e-12
    if case == "stk":
        assert list(st["modes"]) == [ncp.STK]
        assert np.allclose(vn[:2], 0.0, atol=1e-13)
    else:
        assert list(st["modes"]) == [ncp.SLD]
        u = vf[:2] / np.linalg.norm(vf[:2])
        lam_n = mass * (vz - vf[2])                     # the normal impulse that row needs
        assert np.allclose(vn[:2], vf[:2] - mu * lam_n / mass * u, atol=1e-12)
    # dv+_z / dv_z = K_d and dv+_z / dq_z = -(1 - K_p) / dt (identity orientation: the tangent
    # perturbation of the position is the world one)
    assert abs(st["dv_dv"][2, 2] - kd) < 1e-9
    assert abs(st["dv_dq"][2, 2] - (-(1.0 - kp) / dt)) < 1e-6 * max(1.0, (1.0 - kp) / dt)


def _check(m, env, opt, tol12=1e-10, tolfd=2e-6):
    st = S.step_jac(m, env, opt)
    J1 = np.concatenate([st["dv_dq"], st["dv_dv"], st["dv_dtau"]], 1)
    J2 = S.jacobian_route2(m, env, opt, st)
    sc = max(1.0, np.abs(J1).max())
    assert np.abs(J1 - J2).max() <= tol12 * sc
    checked = False
    if st["margin"] > 1e-3:
        Jfd = S.jacobian_fd(m, env, opt)
        assert np.abs(J1 - Jfd).max() <= tolfd * sc
        checked = True
    return st, checked


def test_arm_cube_routes_and_fd():
    wl = scenes.arm_cube(64)
    m = wl.models[0]
    opt = _with_gains(wl.options, 0.4, 0.2)
    n_fd, modes = 0, set()
    for e in range(6):
        st, c = _check(m, wl.batch.env(e, m), opt)
        n_fd += c
        modes.update(int(x) for x in st["modes"])
    assert n_fd >= 2 and {1, 2} <= modes


def test_quadruped_routes_and_fd():
    wl = scenes.quadruped_feet(16)
    m = wl.models[0]
    opt = _with_gains(wl.options, 0.2, 0.5)
    n_fd = 0
    for e in range(4):
        n_fd += _check(m, wl.batch.env(e, m), opt)[1]
    assert n_fd >= 1
