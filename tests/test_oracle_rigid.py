"""Pins of the oracle's rigid-body recursions against identities and closed forms (no GPU)."""
import numpy as np
import pytest

from oracle import rigid
from tests.helpers import models, pendulum_model, random_state

G = np.array([0.0, 0.0, -9.81])


@pytest.mark.parametrize("mi", [0, 1, 2])
def test_rnea_inverts_aba(mi):
    """RNEA(q, v, ABA(q, v, tau)) = tau (ABA and RNEA are independent recursions)."""
    m = models()[mi]
    rng = np.random.default_rng(mi)
    for _ in range(3):
        q, v, tau = random_state(m, rng)
        a = rigid.aba(m, q, v, tau, G)
        assert np.allclose(rigid.rnea(m, q, v, a, G), tau, rtol=0, atol=1e-10 * max(1, np.abs(tau).max()))


@pytest.mark.parametrize("mi", [0, 1, 2])
def test_crba_cholesky_matches_aba(mi):
    """ABA's acceleration = M^-1 (tau - b) with M from CRBA, b = RNEA(q, v, 0); M SPD."""
    m = models()[mi]
    rng = np.random.default_rng(10 + mi)
    q, v, tau = random_state(m, rng)
    M = rigid.crba(m, q)
    assert np.allclose(M, M.T, atol=1e-14 * np.abs(M).max())
    L = rigid.cholesky(M)
    assert np.all(np.diag(L) > 0)
    assert np.allclose(L @ L.T, M, atol=1e-13 * np.abs(M).max())
    b = rigid.rnea(m, q, v, np.zeros(m.nv), G)
    a1 = rigid.chol_solve(L, tau - b)
    a2 = rigid.aba(m, q, v, tau, G)
    assert np.allclose(a1, a2, rtol=1e-10, atol=1e-10 * np.abs(a2).max())


@pytest.mark.parametrize("mi", [0, 1, 2])
def test_crba_equals_sum_of_body_jacobians(mi):
    """M = sum_i J_i^T I_i J_i with J_i from the velocity recursion alone."""
    m = models()[mi]
    q, _, _ = random_state(m, np.random.default_rng(20 + mi))
    Js = rigid.body_jacobians(m, q)
    M2 = sum(J.T @ rigid.inertia6(m, i) @ J for i, J in enumerate(Js))
    M = rigid.crba(m, q)
    assert np.allclose(M, M2, atol=1e-12 * np.abs(M).max())


@pytest.mark.parametrize("mi", [0, 1, 2])
def test_kinetic_energy_from_point_velocities(mi):
    """1/2 v^T M v = sum_i 1/2 m_i |v_com,i|^2 + 1/2 w_i^T I_i w_i, with com velocities and angular
    velocities obtained by differentiating forward kinematics along q (+) t v (complex step)."""
    m = models()[mi]
    q, v, _ = random_state(m, np.random.default_rng(30 + mi))
    h = 1e-30
    qc = rigid.integrate(m, q, 1j * h * v)
    _, w0 = rigid.fk(m, q)
    _, wc = rigid.fk(m, qc)
    T = 0.0
    for i in range(m.nb):
        R, p = w0[i]
        Rc, pc = wc[i]
        vcom = np.imag(pc + Rc @ m.com[i]) / h
        Rdot = np.imag(Rc) / h
        W = R.T @ Rdot                        # body-frame angular velocity (skew)
        w = np.array([W[2, 1], W[0, 2], W[1, 0]])
        T += 0.5 * m.mass[i] * vcom @ vcom + 0.5 * w @ rigid.inertia_matrix_com(m, i) @ w
    assert np.isclose(0.5 * v @ rigid.crba(m, q) @ v, T, rtol=1e-11)


@pytest.mark.parametrize("mi", [0, 1, 2])
def test_gravity_is_potential_gradient(mi):
    """b(q, 0) = dU/dq with U = -sum m_i g.x_com,i (complex-step gradient along the tangent)."""
    m = models()[mi]
    q, _, _ = random_state(m, np.random.default_rng(40 + mi))
    b = rigid.rnea(m, q, np.zeros(m.nv), np.zeros(m.nv), G)
    h = 1e-30
    grad = np.array([np.imag(rigid.gravity_potential(m, rigid.integrate(m, q, 1j * h * e), G)) / h
                     for e in np.eye(m.nv)])
    assert np.allclose(b, grad, atol=1e-11 * max(1, np.abs(b).max()))


@pytest.mark.parametrize("mi", [0, 1, 2])
def test_coriolis_skew_identity(mi):
    """v^T (Mdot - 2 C) v = 0 with Mdot = dM/dt along q (+) t v and C v = b(q, v) - b(q, 0)."""
    m = models()[mi]
    q, v, _ = random_state(m, np.random.default_rng(50 + mi))
    h = 1e-30
    Mdot = np.imag(rigid.crba(m, rigid.integrate(m, q, 1j * h * v))) / h
    Cv = rigid.rnea(m, q, v, np.zeros(m.nv), G) - rigid.rnea(m, q, np.zeros(m.nv), np.zeros(m.nv), G)
    assert abs(v @ Mdot @ v - 2 * v @ Cv) <= 1e-10 * max(1.0, abs(v @ Cv))


def test_pendulum_closed_form():
    """Single pendulum about x with com (0, 0, l): M = Ixx + m l^2, b(q, 0) = -m g l sin q,
    b(q, qd) - b(q, 0) = 0 (one joint: no Coriolis)."""
    mass, l, ixx = 1.5, 0.7, 0.05
    m = pendulum_model(mass, l, ixx)
    for qv in (-2.0, 0.3, 1.1):
        q = np.array([qv])
        assert np.isclose(rigid.crba(m, q)[0, 0], ixx + mass * l * l, rtol=1e-14)
        b0 = rigid.rnea(m, q, np.zeros(1), np.zeros(1), G)[0]
        assert np.isclose(b0, -mass * 9.81 * l * np.sin(qv), rtol=1e-13, atol=1e-14)
        assert np.isclose(rigid.rnea(m, q, np.array([2.0]), np.zeros(1), G)[0], b0, rtol=1e-13, atol=1e-13)


def test_integrate_free_flyer():
    """Free-flyer (+): position moves along body axes, the quaternion stays unit, (+) 0 = identity."""
    from tests.helpers import point_mass_model
    m = point_mass_model()
    rng = np.random.default_rng(3)
    q, _, _ = random_state(m, rng)
    assert np.allclose(rigid.integrate(m, q, np.zeros(6)), q, atol=1e-15)
    dv = rng.normal(size=6)
    q2 = rigid.integrate(m, q, dv)
    assert np.isclose(np.linalg.norm(q2[3:]), 1.0, atol=1e-15)
    R = rigid.quat_to_rot(q[3:])
    assert np.allclose(q2[:3], q[:3] + R @ dv[:3], atol=1e-14)
    R2 = rigid.quat_to_rot(q2[3:])
    assert np.allclose(R2, R @ rigid.rodrigues(dv[3:] / np.linalg.norm(dv[3:]), np.linalg.norm(dv[3:])), atol=1e-13)
