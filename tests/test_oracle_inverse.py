"""Pins of the oracle's Gauss-Newton inverse problems (Sec. 4: estimating an initial condition,
inverse dynamics through contacts; no GPU).

* the chain-rule Jacobian dq_T/dv_0 of a sliding cube's T-step rollout equals central finite
  differences of the rollout (tangent coordinates).  The cube rests on three points of its bottom
  face (a triangle around the centre of mass): on all four corners the split of the normal impulse
  among them is statically indeterminate,
  and so is the friction torque about the vertical (the corners slide in different directions
  once the cube turns), so the yaw response would depend on which member of the solution family
  the solver returns; three contacts make the split, and the step, unique;
* Gauss-Newton recovers the initial velocity of a cube thrown onto the floor in a sliding mode
  (its planar components: x, y and the yaw rate; the sliding premise fixes the others) from the
  configuration it reaches, the residual falling to zero;
* inverse dynamics: Gauss-Newton finds actuator torques that hold a standing quadruped at rest
  (v+ = 0), as the paper reports, in a few iterations.
"""
import numpy as np

from oracle import inverse as INV
from oracle import rigid
from paper_2409_07107_gb300 import scenes
from tests.helpers import point_mass_model

H = 0.025            # half size of the 0.05 m cube


def _cube(mu=0.3, pen=1e-4):
    mass = 1.0
    ii = mass * (2 * H) ** 2 / 6.0
    m = point_mass_model(mass, (ii, ii, ii))
    corners = np.array([[-H, -H, -H], [H, -H, -H], [0.0, H, -H]])     # a triangle under the centre
    nc = len(corners)
    env = dict(q=np.array([0.0, 0.0, H - pen, 1.0, 0.0, 0.0, 0.0]), v=np.zeros(6), tau=np.zeros(6),
               c_link=np.zeros(nc, np.int64), c_point=corners, c_radius=np.zeros(nc), c_mu=np.full(nc, mu),
               plane=np.array([0.0, 0.0, 1.0, 0.0]))
    return m, env


V_TRUE = np.array([1.0, 0.4, 0.0, 0.0, 0.0, 0.5])   # sliding in x, y with a yaw rate
T = 12


def test_rollout_jacobian_matches_finite_differences():
    m, env = _cube()
    opt = scenes.Options()
    env = dict(env, v=V_TRUE)
    qT, J = INV.rollout_q_jacobian(m, env, T, opt)
    h = 1e-6
    Jfd = np.zeros_like(J)
    for j in range(6):
        e = np.zeros(6)
        e[j] = h
        qp = INV.rollout_q(m, dict(env, v=V_TRUE + e), T, opt)
        qm = INV.rollout_q(m, dict(env, v=V_TRUE - e), T, opt)
        Jfd[:, j] = (rigid.local_difference(m, qT, qp) - rigid.local_difference(m, qT, qm)) / (2 * h)
    assert np.abs(J - Jfd).max() <= 1e-6 * max(1.0, np.abs(J).max())


def test_initial_velocity_estimation():
    m, env = _cube()
    opt = scenes.Options()
    q_target = INV.rollout_q(m, dict(env, v=V_TRUE), T, opt)
    v_init = V_TRUE + np.array([0.05, -0.03, 0.0, 0.0, 0.0, 0.1])
    v0, hist = INV.estimate_initial_velocity(m, env, q_target, T, opt, v_init, iters=12, tol=1e-13,
                                             free=[0, 1, 5])
    assert hist[-1] <= 1e-13 and len(hist) <= 8
    assert np.abs(v0 - V_TRUE).max() <= 1e-9


def test_inverse_dynamics_holds_a_quadruped_at_rest():
    wl = scenes.quadruped_feet(4)
    m = wl.models[0]
    env = wl.batch.env(0, m)
    env = dict(env, v=np.zeros(m.nv))
    Sa = np.eye(m.nv)[6:]                             # the 12 joint torques; the base is unactuated
    ta, hist = INV.inverse_dynamics(m, env, wl.options, Sa, np.zeros(m.nv), np.zeros(12), iters=20, tol=1e-10)
    assert hist[-1] <= 1e-8 * max(1.0, hist[0])
    assert len(hist) <= 15
