"""Small shared test helpers (no method arithmetic)."""
import numpy as np

from paper_2409_07107_gb300 import scenes


def point_mass_model(mass=2.0, inertia=(0.1, 0.2, 0.3)):
    """One free-flying body with its centre of mass at its origin."""
    return scenes.Model("pointmass", np.array([-1], np.int32), np.array([scenes.FREEFLYER], np.int32),
                        np.zeros((1, 3)), np.eye(3)[None], np.zeros((1, 3)), np.array([mass]),
                        np.zeros((1, 3)), np.array([[inertia[0], inertia[1], inertia[2], 0.0, 0.0, 0.0]]))


def pendulum_model(mass=1.5, length=0.7, ixx=0.05):
    """One revolute joint about x, centre of mass at (0, 0, length)."""
    return scenes.Model("pendulum", np.array([-1], np.int32), np.array([scenes.REVOLUTE], np.int32),
                        np.array([[1.0, 0.0, 0.0]]), np.eye(3)[None], np.zeros((1, 3)), np.array([mass]),
                        np.array([[0.0, 0.0, length]]), np.array([[ixx, 0.04, 0.03, 0.0, 0.0, 0.0]]))


def random_state(model, rng, qs=1.0):
    q = np.zeros(model.nq)
    iq = model.iq
    for i, jt in enumerate(model.jtype):
        if jt == scenes.REVOLUTE:
            q[iq[i]] = rng.uniform(-np.pi, np.pi) * qs
        else:
            q[iq[i]:iq[i] + 3] = rng.normal(size=3)
            qq = rng.normal(size=4)
            q[iq[i] + 3:iq[i] + 7] = qq / np.linalg.norm(qq)
    return q, rng.normal(size=model.nv), rng.normal(size=model.nv) * 3


def models():
    rng = np.random.default_rng(7)
    return [scenes.arm7(rng)[0], scenes.quadruped18(rng)[0], scenes.humanoid36(rng)[0]]
