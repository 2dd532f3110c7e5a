"""Pins of the oracle's implicit derivatives: the paper's reduced A/B/C system (App. B, route 1)
against direct implicit differentiation of the mode equations (route 2) and against central finite
differences of the whole step (no GPU)."""
import numpy as np
import pytest

from oracle import step as S
from paper_2409_07107_gb300 import scenes


def _check(m, env, opt, fd=True, tol12=1e-10, tolfd=2e-6):
    st = S.step_jac(m, env, opt)
    J1 = np.concatenate([st["dv_dq"], st["dv_dv"], st["dv_dtau"]], 1)
    J2 = S.jacobian_route2(m, env, opt, st)
    sc = max(1.0, np.abs(J1).max())
    assert np.abs(J1 - J2).max() <= tol12 * sc
    if fd and st["margin"] > 1e-3:
        Jfd = S.jacobian_fd(m, env, opt)
        assert np.abs(J1 - Jfd).max() <= tolfd * sc
    return st


def test_arm_sphere_all_envs():
    wl = scenes.arm_sphere(16)
    m = wl.models[0]
    modes = set()
    for e in range(16):
        st = _check(m, wl.batch.env(e, m), wl.options)
        modes.update(int(x) for x in st["modes"])
    assert len(modes) >= 2


def test_arm_cube_sample():
    wl = scenes.arm_cube(64)
    m = wl.models[0]
    modes = set()
    for e in range(8):
        st = _check(m, wl.batch.env(e, m), wl.options)
        modes.update(int(x) for x in st["modes"])
    assert {1, 2} <= modes


def test_quadruped_sample():
    wl = scenes.quadruped_feet(16)
    m = wl.models[0]
    for e in range(3):
        _check(m, wl.batch.env(e, m), wl.options)


@pytest.mark.slow
def test_humanoid_sample():
    wl = scenes.humanoid_feet(16)
    m = wl.models[0]
    e = next(e for e in range(16) if len(S.step(m, wl.batch.env(e, m), wl.options)["slots"]) >= 2)
    _check(m, wl.batch.env(e, m), wl.options)


def test_vjp_is_transpose():
    """VJP of the oracle = J^T v_bar (dot-product identity <w, J u> = <J^T w, u>)."""
    wl = scenes.arm_cube(64)
    m = wl.models[0]
    env = wl.batch.env(3, m)
    st = S.step_jac(m, env, wl.options)
    rng = np.random.default_rng(0)
    w = rng.normal(size=7)
    u = rng.normal(size=21)
    J = np.concatenate([st["dv_dq"], st["dv_dv"], st["dv_dtau"]], 1)
    qb, vb, tb = S.vjp(m, env, wl.options, w, st)
    assert np.isclose(w @ J @ u, np.concatenate([qb, vb, tb]) @ u, rtol=1e-12)
