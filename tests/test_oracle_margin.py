"""Pins of the oracle's contact activation margin (no GPU).

App. D's gap term phi/dt - K_p [phi/dt]_- - K_d (J_c v)_N acts on contacts that may still be
apart (phi > 0; the proportional part only acts on penetration).  With the option
contact_margin = delta a slot is active when phi <= delta, and such a contact may approach the
plane by at most phi within the step (sigma_N >= 0).  Pinned here:

* margin 0 leaves the step unchanged, and a contact above the plane outside the margin is inactive;
* closed form: a point mass at height h (0 < h <= delta) with free velocity v_f keeps v+ = v_f when
  v_f,N + h/dt - K_d v_N >= 0, and otherwise lands: v+_N = K_d v_N - h/dt, with v+_T = 0 when
  |v_f,T| <= -mu (v_f,N + h/dt - K_d v_N) and else v+_T = v_f,T + mu (v_f,N + h/dt - K_d v_N) u;
  its derivatives dv+_z/dz = -1/dt and dv+_z/dv_z = K_d follow (K_p does not enter at h > 0);
* route 1 = route 2 = central differences of the whole step on an arm with an end-effector sphere
  whose contacts lie within 2 mm of the plane, with and without Baumgarte gains.
"""
import types

import numpy as np
import pytest

from oracle import step as S
from paper_2409_07107_gb300 import scenes
from tests.helpers import point_mass_model


def _opt(margin=0.0, kp=1.0, kd=0.0, base=None):
    d = dict(vars(base or scenes.Options()))
    d.update(contact_margin=margin, baumgarte_kp=kp, baumgarte_kd=kd)
    return types.SimpleNamespace(**d)


def _pm(vlin, h, mu=0.5, mass=2.0):
    m = point_mass_model(mass)
    env = dict(q=np.array([0.1, -0.2, 0.3, 1.0, 0.0, 0.0, 0.0]), v=np.concatenate([vlin, np.zeros(3)]),
               tau=np.zeros(6), c_link=np.array([0]), c_point=np.zeros((1, 3)), c_radius=np.zeros(1),
               c_mu=np.array([mu]), plane=np.array([0.0, 0.0, 1.0, 0.3 - h]))
    return m, env


def test_margin_zero_is_the_plain_step():
    wl = scenes.arm_sphere(16)
    m = wl.models[0]
    for e in range(6):
        env = wl.batch.env(e, m)
        a, b = S.step(m, env, wl.options), S.step(m, env, _opt(0.0))
        assert a["slots"] == b["slots"]
        assert np.array_equal(a["v_next"], b["v_next"]) and np.array_equal(a["g"], b["g"])


def test_contact_outside_the_margin_is_inactive():
    m, env = _pm(np.array([0.3, 0.0, -2.0]), 1e-3)
    for margin in (0.0, 5e-4):
        st = S.step(m, env, _opt(margin))
        assert st["slots"] == []
    st = S.step(m, env, _opt(2e-3))
    assert st["slots"] == [0]


@pytest.mark.parametrize("kd", [0.0, 0.4])
@pytest.mark.parametrize("case", ["apart", "stk", "sld"])
def test_point_mass_closed_form(case, kd):
    dt, mu, h = 1e-3, 0.5, 5e-5
    vlin = {"apart": np.array([0.2, 0.1, -0.01]), "stk": np.array([0.02, -0.01, -0.3]),
            "sld": np.array([1.0, 0.5, -0.3])}[case]
    m, env = _pm(vlin, h, mu)
    opt = _opt(2e-3, kp=0.3, kd=kd)
    st = S.step_jac(m, env, opt)
    assert st["slots"] == [0]
    vf = vlin + dt * np.array([0.0, 0.0, -9.81])
    gn = vf[2] + h / dt - kd * vlin[2]          # sigma_N at lambda = 0
    vn = st["v_next"][:3]
    if case == "apart":
        assert gn > 0 and int(st["modes"][0]) == ncp_mode("brk")
        assert np.allclose(vn, vf, atol=1e-14)
        return
    assert gn < 0
    assert abs(vn[2] - (kd * vlin[2] - h / dt)) <= 1e-12
    assert abs(st["dv_dq"][2, 2] - (-1.0 / dt)) <= 1e-8
    assert abs(st["dv_dv"][2, 2] - kd) <= 1e-10
    if case == "stk":
        assert np.linalg.norm(vf[:2]) <= -mu * gn and int(st["modes"][0]) == ncp_mode("stk")
        assert np.allclose(vn[:2], 0.0, atol=1e-13)
    else:
        u = vf[:2] / np.linalg.norm(vf[:2])
        assert int(st["modes"][0]) == ncp_mode("sld")
        assert np.allclose(vn[:2], vf[:2] + mu * gn * u, atol=1e-12)
        # dv+_T/dz: the landing impulse grows by m/dt per unit height, so does the friction
        assert np.allclose(st["dv_dq"][:2, 2], mu * u / dt, atol=1e-7)


def ncp_mode(name):
    from oracle import ncp
    return {"brk": ncp.BRK, "stk": ncp.STK, "sld": ncp.SLD}[name]


@pytest.mark.slow
@pytest.mark.parametrize("kp,kd", [(1.0, 0.0), (0.4, 0.2)])
def test_routes_and_fd_with_margin(kp, kd):
    wl = scenes.arm_sphere(16)
    m = wl.models[0]
    opt = _opt(2.5e-3, kp, kd, wl.options)
    checked = 0
    for e in range(16):
        env = wl.batch.env(e, m)
        st = S.step_jac(m, env, opt)
        if not st["slots"] or st["margin"] < 1e-3:
            continue
        J1 = np.concatenate([st["dv_dq"], st["dv_dv"], st["dv_dtau"]], 1)
        J2 = S.jacobian_route2(m, env, opt, st)
        assert np.abs(J1 - J2).max() <= 1e-10 * max(1.0, np.abs(J1).max())
        Jfd = S.jacobian_fd(m, env, opt, h=1e-6)
        assert np.abs(J1 - Jfd).max() <= 2e-6 * max(1.0, np.abs(J1).max()), e
        checked += 1
        if checked >= 4:
            break
    assert checked >= 3
