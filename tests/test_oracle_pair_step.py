"""Pins of the oracle's step with contacts between convex shapes on the bodies (Sec. 2.1, Eq. 1-6)
and of its Jacobians with App. C's contact-placement terms, no GPU.

* The step's impulses solve Eq. 1 at the solution's own velocity: sigma = J_c v+ lies in the dual
  cone, lambda in the cone, and they are complementary (De Saxce's form), with J_c taken from the
  collision detection's contact frame.
* dv+/d(q, v, tau) by App. D's route 1 with the placement terms (dCD/dM_i by central differences of
  the collision detection) equals central differences of the whole step -- contact frame, Delassus
  matrix and NCP solve recomputed at every perturbed q -- for a capsule on an arm link against a
  fixed box and a sphere on one link against a box on another, in each mode (breaking, sticking,
  sliding), and for both pairs in contact at once.  Leaving out either placement term (the one in
  d(J_c v+)/dq or the one in d(J_c^T lambda)/dq) misses by orders of magnitude more than the
  tolerance.
* App. D's Baumgarte term and activation margin on pair contacts: the Jacobian against central
  differences, with a pair inside the margin but apart; without the term's derivative it misses.
* With no pair in contact the step is the free step v + dt ABA(q, v, tau)."""
import types

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import collision as C
from oracle import pair_step as PS
from oracle import rigid
from oracle.ncp import BRK, SLD, STK

I3 = np.eye(3)
OPT = types.SimpleNamespace(dt=0.01, gravity=(0.0, 0.0, -9.81))


def _world_case(seed, vscale, mu, pen=0.004):
    """A capsule on link 5 of a random 7-dof arm; a fixed box placed so that its top face is pen
    above the capsule's lowest point (directly below it)."""
    from paper_2409_07107_gb300 import scenes
    rng = np.random.default_rng(seed)
    model, _ = scenes.arm7(rng)
    q = rng.uniform(-np.pi, np.pi, size=7)
    env = dict(q=q, v=vscale * rng.normal(size=7), tau=rng.normal(size=7))
    E = Rotation.from_rotvec(rng.normal(size=3)).as_matrix()
    cap = C.capsule(0.05, 0.03)
    R, p = C.body_pose(model, q, 4)
    core = np.atleast_2d(C.world_core(cap, R @ E, p))
    low = core[np.argmin(core[:, 2])]
    ctr = np.array([low[0], low[1], low[2] - 0.03 + pen - 0.1])
    return model, env, [(cap, 4, (E, np.zeros(3)), C.box(0.3, 0.3, 0.1), -1, (I3, ctr), mu)]


def _self_case(seed, vscale, mu, pen=0.004):
    """A sphere at the tip of link 7 and a box on link 3 of the same arm, the box's top face (its
    own z) pen inside the sphere."""
    from paper_2409_07107_gb300 import scenes
    rng = np.random.default_rng(seed)
    model, tip = scenes.arm7(rng)
    q = rng.uniform(-np.pi, np.pi, size=7)
    env = dict(q=q, v=vscale * rng.normal(size=7), tau=rng.normal(size=7))
    R7, p7 = C.body_pose(model, q, 6)
    centre = p7 + R7 @ tip
    R3, p3 = C.body_pose(model, q, 2)
    Eb = Rotation.from_rotvec(rng.normal(size=3)).as_matrix()
    box_ctr = centre - (R3 @ Eb)[:, 2] * (0.05 - pen + 0.06)
    pair = (C.sphere(0.05), 6, (I3, np.asarray(tip, float)), C.box(0.05, 0.08, 0.06), 2,
            (Eb, R3.T @ (box_ctr - p3)), mu)
    return model, env, [pair]


CASES = [
    ("world", 2, 1.0, 0.2, SLD),
    ("world", 5, 0.01, 5.0, STK),
    ("world", 4, 2.0, 0.1, BRK),
    ("self", 7, 0.01, 5.0, STK),
    ("self", 10, 0.3, 0.2, SLD),
]


def _case(kind, seed, vscale, mu):
    return (_world_case if kind == "world" else _self_case)(seed, vscale, mu)


@pytest.mark.parametrize("kind,seed,vscale,mu,mode", CASES)
def test_pair_step_solves_eq1(kind, seed, vscale, mu, mode):
    model, env, pairs = _case(kind, seed, vscale, mu)
    st = PS.step(model, env, pairs, OPT)
    assert st["act"] == [0] and st["converged"] and int(st["modes"][0]) == mode
    lam = st["lam"]
    sigma = st["Jc"] @ st["v_next"]
    # Eq. 1 (De Saxce): lambda in K_mu, sigma + mu ||sigma_T|| e_N in K_mu*, orthogonal
    nt = np.hypot(sigma[0], sigma[1])
    s_hat = sigma + np.array([0.0, 0.0, mu * nt])
    assert np.hypot(lam[0], lam[1]) <= mu * lam[2] + 1e-10
    assert mu * np.hypot(s_hat[0], s_hat[1]) <= s_hat[2] + 1e-8
    assert abs(lam @ s_hat) <= 1e-8 * max(1.0, np.abs(lam).max())
    # and v+ is the step of Eq. 6 with the contact wrenches of lambda
    M = rigid.crba(model, env["q"])
    v_f = PS.ufd_velocity(model, env["q"], env["v"], env["tau"], OPT, None)
    assert np.allclose(M @ (st["v_next"] - v_f), st["Jc"].T @ lam, atol=1e-9)


@pytest.mark.parametrize("kind,seed,vscale,mu,mode", CASES)
def test_pair_step_jacobian_against_central_differences(kind, seed, vscale, mu, mode):
    model, env, pairs = _case(kind, seed, vscale, mu)
    st = PS.step_jac(model, env, pairs, OPT)
    assert int(st["modes"][0]) == mode
    fd = PS.jacobian_fd(model, env, pairs, OPT)
    J = np.concatenate([st["dv_dq"], st["dv_dv"], st["dv_dtau"]], axis=1)
    assert np.abs(J - fd).max() <= 1e-6 * max(1.0, np.abs(fd).max())


@pytest.mark.parametrize("dropped", ["appc_dJcv_dq", "appc_dJctlam_dq"])
def test_pair_step_jacobian_needs_both_placement_terms(monkeypatch, dropped):
    model, env, pairs = _world_case(2, 1.0, 0.2)
    fd = PS.jacobian_fd(model, env, pairs, OPT)
    full = getattr(C, dropped)
    monkeypatch.setattr(C, dropped, lambda *a: 0.0 * full(*a))
    st = PS.step_jac(model, env, pairs, OPT)
    assert np.abs(st["dv_dq"] - fd[:, :7]).max() > 1e-2


def _two_pair_case(seed, vscale, mu):
    """The capsule-against-fixed-box pair of _world_case and, on the same arm at the same q, a
    sphere at link 7's origin against a box on link 3, both active."""
    model, env, pairs = _world_case(seed, vscale, mu)
    rng = np.random.default_rng(seed + 1000)
    q = env["q"]
    _, p7 = C.body_pose(model, q, 6)
    R3, p3 = C.body_pose(model, q, 2)
    Eb = Rotation.from_rotvec(rng.normal(size=3)).as_matrix()
    box_ctr = p7 - (R3 @ Eb)[:, 2] * (0.05 - 0.004 + 0.06)
    pairs = pairs + [(C.sphere(0.05), 6, (I3, np.zeros(3)), C.box(0.05, 0.08, 0.06), 2, (Eb, R3.T @ (box_ctr - p3)), mu)]
    return model, env, pairs


@pytest.mark.parametrize("seed,vscale,mu,modes", [(21, 0.3, 0.3, (SLD, BRK)), (21, 0.02, 3.0, (STK, STK)),
                                                  (20, 0.02, 3.0, (SLD, SLD))])
def test_two_pairs_against_central_differences(seed, vscale, mu, modes):
    """Two pairs in contact at once, each with its own moving contact frame (at seed 21 the capsule's
    contact point lies on the diagonal of the box face's triangulation, the case the collision pin
    test_witness_on_a_triangulated_face_diagonal covers)."""
    model, env, pairs = _two_pair_case(seed, vscale, mu)
    st = PS.step_jac(model, env, pairs, OPT)
    assert st["act"] == [0, 1] and tuple(int(m) for m in st["modes"]) == modes
    fd = PS.jacobian_fd(model, env, pairs, OPT)
    J = np.concatenate([st["dv_dq"], st["dv_dv"], st["dv_dtau"]], axis=1)
    assert np.abs(J - fd).max() <= 1e-6 * max(1.0, np.abs(fd).max())


def test_pair_step_takes_the_smoothed_placement_derivative():
    """The step Jacobian with dCD/dM_i from App. C's smoothing estimator (the paper's route) fed
    the orthogonal samples +-sigma sqrt(6) e_j equals the one with central differences at that
    step (the estimator is then exactly those differences)."""
    model, env, pairs = _two_pair_case(21, 0.3, 0.3)
    sigma = 1e-6 / np.sqrt(6.0)
    design = np.sqrt(6.0) * sigma * np.eye(6)
    st = PS.step_jac(model, env, pairs, OPT,
                     dcd_fn=lambda m, q, pr, w: C.dcd_dbody_smoothed(m, q, pr, w, sigma, design))
    ref = PS.step_jac(model, env, pairs, OPT)
    assert np.abs(st["dv_dq"] - ref["dv_dq"]).max() <= 1e-9 * max(1.0, np.abs(ref["dv_dq"]).max())


def _opt(kp, kd, margin):
    return types.SimpleNamespace(dt=0.01, gravity=(0.0, 0.0, -9.81), baumgarte_kp=kp, baumgarte_kd=kd,
                                 contact_margin=margin)


BAUMGARTE_CASES = [
    ("world", 2, 1.0, 0.2, 0.004, (0.3, 0.2, 0.01), [SLD]),
    ("world", 34, 1.0, 0.6, -0.0005, (0.3, 0.2, 0.01), [SLD]),      # apart by 0.5 mm, inside the margin
    ("two", 21, 0.3, 0.3, None, (0.5, 0.0, 0.0), [SLD, BRK]),
    ("two", 20, 0.02, 3.0, None, (0.3, 0.2, 0.01), [STK, BRK]),
]


def _baumgarte_case(kind, seed, vscale, mu, pen):
    return _world_case(seed, vscale, mu, pen=pen) if kind == "world" else _two_pair_case(seed, vscale, mu)


@pytest.mark.parametrize("kind,seed,vscale,mu,pen,gains,modes", BAUMGARTE_CASES)
def test_pair_step_baumgarte_against_central_differences(kind, seed, vscale, mu, pen, gains, modes):
    """App. D's Baumgarte term phi/dt - K_p [phi/dt]_- - K_d (J_c v)_N on pair contacts, with the
    activation margin (a pair 0.5 mm apart is active and slides): the route-1 Jacobian, whose
    Baumgarte derivative takes d phi/dq = (J_c)_N and the placement terms for d(J_c v)_N/dq,
    equals central differences of the whole step."""
    model, env, pairs = _baumgarte_case(kind, seed, vscale, mu, pen)
    opt = _opt(*gains)
    st = PS.step_jac(model, env, pairs, opt)
    assert [int(m) for m in st["modes"]] == modes
    fd = PS.jacobian_fd(model, env, pairs, opt)
    J = np.concatenate([st["dv_dq"], st["dv_dv"], st["dv_dtau"]], axis=1)
    assert np.abs(J - fd).max() <= 1e-6 * max(1.0, np.abs(fd).max())


def test_pair_step_baumgarte_derivative_matters(monkeypatch):
    model, env, pairs = _world_case(34, 1.0, 0.6, pen=-0.0005)
    opt = _opt(0.3, 0.2, 0.01)
    fd = PS.jacobian_fd(model, env, pairs, opt)
    full = PS.partials
    monkeypatch.setattr(PS, "partials", lambda *a, **k: full(*a, **k)[:2] + (None,))
    st = PS.step_jac(model, env, pairs, opt)
    J = np.concatenate([st["dv_dq"], st["dv_dv"], st["dv_dtau"]], axis=1)
    assert np.abs(J - fd).max() > 1e-2 * np.abs(fd).max()


def test_pair_step_without_contact_is_the_free_step():
    model, env, pairs = _world_case(3, 0.5, 0.5, pen=-0.05)     # the box 5 cm below the capsule
    st = PS.step_jac(model, env, pairs, OPT)
    assert st["act"] == []
    v_f = env["v"] + OPT.dt * rigid.aba(model, env["q"], env["v"], env["tau"], np.asarray(OPT.gravity))
    assert np.allclose(st["v_next"], v_f, atol=1e-14)
    fd = PS.jacobian_fd(model, env, pairs, OPT)
    J = np.concatenate([st["dv_dq"], st["dv_dv"], st["dv_dtau"]], axis=1)
    assert np.abs(J - fd).max() <= 1e-6 * max(1.0, np.abs(fd).max())
