"""Pins of the oracle's collision detection between convex shapes (Sec. 2.1) and of its
randomized-smoothing derivative (App. C), no GPU.

* closed forms: sphere-sphere (apart and penetrating); sphere-box (the clamped centre, and the
  nearest face when the centre is inside); axis-aligned box-box (the gap, or the smallest overlap
  along an axis);
* independent references: capsule-capsule against dense sampling of the two segments; rotated
  box-box and box-capsule pairs that are apart against a QP over convex weights (scipy SLSQP);
* invariances: a rigid motion of both shapes moves c and n with it and keeps phi; swapping the
  shapes keeps phi and c and flips n;
* the smoothing estimator against the analytic derivative of phi and n for two spheres (a smooth
  pair), with a small sigma;
* App. C's contact-placement terms of d(J_c v)/dq for contacts between two bodies of an arm and
  between an arm link and a fixed box: with the bodies' velocity change they sum to central
  differences of q -> J_c(q) v, the contact frame recomputed by collision detection at every q
  (a flipped sign or swapped cross product in the terms fails it); and the second term,
  d(J_c^T lambda)/dq, by duality, against central differences of J_c(q)^T lambda with and without
  the body-to-contact transforms held.
"""
import numpy as np
import pytest
from scipy.optimize import minimize
from scipy.spatial.transform import Rotation

from oracle import collision as C

I3 = np.eye(3)


def _rot(rng):
    return Rotation.from_rotvec(rng.normal(size=3)).as_matrix()


@pytest.mark.parametrize("dist", [0.7, 0.25])
def test_sphere_sphere(dist):
    rng = np.random.default_rng(1)
    for _ in range(10):
        pa = rng.normal(size=3)
        u = rng.normal(size=3)
        u /= np.linalg.norm(u)
        pb = pa + dist * u
        res = C.collide(C.sphere(0.2), _rot(rng), pa, C.sphere(0.3), _rot(rng), pb)
        assert abs(res["phi"] - (dist - 0.5)) <= 1e-12
        assert np.allclose(res["n"], u, atol=1e-12)
        assert np.allclose(res["c"], 0.5 * ((pa + 0.2 * u) + (pb - 0.3 * u)), atol=1e-12)
        assert np.allclose(res["Rc"][:, 2], u) and np.allclose(res["Rc"].T @ res["Rc"], I3, atol=1e-12)


def test_sphere_box():
    rng = np.random.default_rng(2)
    h = np.array([0.3, 0.5, 0.4])
    for _ in range(40):
        R, p = _rot(rng), rng.normal(size=3)
        xb = rng.uniform(-1.0, 1.0, size=3) * (h + 0.3)           # centre in the box frame
        xw = p + R @ xb
        res = C.collide(C.sphere(0.1), I3, xw, C.box(*h), R, p)
        clamp = np.clip(xb, -h, h)
        if np.any(np.abs(xb) > h):
            d = np.linalg.norm(xb - clamp)
            assert abs(res["phi"] - (d - 0.1)) <= 1e-10
            assert np.allclose(res["n"], R @ (clamp - xb) / d, atol=1e-9)
        else:
            depth = np.min(h - np.abs(xb))
            assert abs(res["phi"] + depth + 0.1) <= 1e-10
            k = int(np.argmin(h - np.abs(xb)))
            assert np.allclose(res["n"], -np.sign(xb[k]) * R[:, k], atol=1e-9)


def test_axis_aligned_boxes():
    rng = np.random.default_rng(3)
    ha, hb = np.array([0.3, 0.5, 0.4]), np.array([0.2, 0.6, 0.3])
    for _ in range(40):
        delta = rng.uniform(-1.0, 1.0, size=3)
        res = C.collide(C.box(*ha), I3, np.zeros(3), C.box(*hb), I3, delta)
        overlap = ha + hb - np.abs(delta)
        if np.all(overlap > 0):
            k = int(np.argmin(overlap))
            assert abs(res["phi"] + overlap[k]) <= 1e-10
            assert np.allclose(res["n"], np.sign(delta[k]) * I3[k], atol=1e-10)
        else:
            gap = np.linalg.norm(np.maximum(-overlap, 0.0))
            assert abs(res["phi"] - gap) <= 1e-10


def test_capsule_capsule_against_sampling():
    rng = np.random.default_rng(4)
    s = np.linspace(-1.0, 1.0, 801)
    for _ in range(6):
        Ra, Rb = _rot(rng), _rot(rng)
        pa, pb = rng.normal(size=3), rng.normal(size=3)
        res = C.collide(C.capsule(0.5, 0.1), Ra, pa, C.capsule(0.4, 0.05), Rb, pb)
        A = pa + np.outer(0.5 * s, Ra[:, 2])
        B = pb + np.outer(0.4 * s, Rb[:, 2])
        d = np.sqrt(((A[:, None, :] - B[None, :, :]) ** 2).sum(-1)).min()
        assert abs(res["phi"] - (d - 0.15)) <= 2e-3


def _qp_distance(ca, cb):
    """min |sum a_i ca_i - sum b_j cb_j| over convex weights (an independent reference)."""
    na, nb = len(ca), len(cb)

    def f(w):
        return np.sum((w[:na] @ ca - w[na:] @ cb) ** 2)

    cons = [{"type": "eq", "fun": lambda w: np.sum(w[:na]) - 1.0}, {"type": "eq", "fun": lambda w: np.sum(w[na:]) - 1.0}]
    w0 = np.concatenate([np.full(na, 1.0 / na), np.full(nb, 1.0 / nb)])
    r = minimize(f, w0, bounds=[(0.0, 1.0)] * (na + nb), constraints=cons, method="SLSQP",
                 options={"ftol": 1e-16, "maxiter": 500})
    return np.sqrt(r.fun)


@pytest.mark.parametrize("pair", ["box-box", "box-capsule"])
def test_rotated_pairs_against_qp(pair):
    rng = np.random.default_rng(5)
    checked = 0
    for _ in range(30):
        Ra, Rb = _rot(rng), _rot(rng)
        pa, pb = np.zeros(3), rng.normal(size=3) * 1.5
        a = C.box(0.3, 0.2, 0.4)
        b = C.box(0.25, 0.35, 0.15) if pair == "box-box" else C.capsule(0.3, 0.0)
        res = C.collide(a, Ra, pa, b, Rb, pb)
        if res["phi"] <= 1e-3:
            continue
        ref = _qp_distance(C.world_core(a, Ra, pa), C.world_core(b, Rb, pb))
        assert abs(res["phi"] - ref) <= 1e-6
        # the witness points are on the shapes and realise the distance along n
        assert abs(np.linalg.norm(res["pb"] - res["pa"]) - res["phi"]) <= 1e-9
        assert np.allclose(res["pb"] - res["pa"], res["phi"] * res["n"], atol=1e-9)
        checked += 1
    assert checked >= 10


def test_rigid_motion_and_swap():
    rng = np.random.default_rng(6)
    shapes = [C.box(0.3, 0.2, 0.4), C.capsule(0.3, 0.1), C.sphere(0.2), C.box(0.1, 0.5, 0.2)]
    for k in range(16):
        a, b = shapes[k % 4], shapes[(k + 1) % 4]
        Ra, Rb, pa, pb = _rot(rng), _rot(rng), np.zeros(3), rng.normal(size=3) * 0.6
        res = C.collide(a, Ra, pa, b, Rb, pb)
        G, t = _rot(rng), rng.normal(size=3)
        moved = C.collide(a, G @ Ra, G @ pa + t, b, G @ Rb, G @ pb + t)
        assert abs(moved["phi"] - res["phi"]) <= 1e-9
        assert np.allclose(moved["n"], G @ res["n"], atol=1e-7)
        swapped = C.collide(b, Rb, pb, a, Ra, pa)
        assert abs(swapped["phi"] - res["phi"]) <= 1e-9
        assert np.allclose(swapped["n"], -res["n"], atol=1e-7)


def test_smoothing_jacobian_of_two_spheres():
    rng = np.random.default_rng(7)
    pa, pb = np.array([0.1, -0.2, 0.3]), np.array([0.6, 0.1, 0.1])
    ra, rb = 0.2, 0.15
    J = C.randomized_smoothing_jacobian(C.sphere(ra), I3, pa, C.sphere(rb), I3, pb, 1e-4, 6000, rng)
    dvec = pb - pa
    L = np.linalg.norm(dvec)
    n = dvec / L
    # a world twist (u, w) moves a point x by u + w x x
    dpa = np.hstack([I3, -np.array([[0, -pa[2], pa[1]], [pa[2], 0, -pa[0]], [-pa[1], pa[0], 0]])])
    dpb = np.hstack([I3, -np.array([[0, -pb[2], pb[1]], [pb[2], 0, -pb[0]], [-pb[1], pb[0], 0]])])
    dphi = np.hstack([-n @ dpa, n @ dpb])
    P = (I3 - np.outer(n, n)) / L
    dn = np.hstack([-P @ dpa, P @ dpb])
    scale = max(np.abs(dphi).max(), np.abs(dn).max())
    assert np.abs(J[0] - dphi).max() <= 0.05 * scale
    assert np.abs(J[4:7] - dn).max() <= 0.05 * scale


def _arm_pair(rng, kind):
    from paper_2409_07107_gb300 import scenes
    model, tip = scenes.arm7(rng)
    q = rng.uniform(-np.pi, np.pi, size=7)
    v = rng.normal(size=7)
    if kind == "self":
        # a sphere at the tip of link 7 and a box on link 3, both on the arm
        pair = (C.sphere(0.05), 6, (I3, np.asarray(tip, float)), C.box(0.05, 0.08, 0.06), 2, (_rot(rng), np.zeros(3)))
    else:
        # a capsule on link 5 against a fixed box in the world
        pair = (C.capsule(0.05, 0.03), 4, (_rot(rng), np.zeros(3)), C.box(0.3, 0.3, 0.1), -1, (I3, np.array([0.0, 0.0, -0.5])))
    return model, q, v, pair


@pytest.mark.parametrize("kind", ["self", "world"])
def test_appc_contact_placement_terms(kind):
    """App. C: with the contact frame moving with the collision detection, d(J_c v)/dq at fixed v is
    the bodies' velocity change seen in the contact frame plus the placement terms
    E[(cX_i V_i) x dCD/dM_i J_i - cX_i (V_i x J_i)] (signed per body); their sum equals central
    differences of q -> J_c(q) v, the contact frame recomputed at every q."""
    from oracle import rigid
    rng = np.random.default_rng(8 if kind == "self" else 9)
    model, q, v, pair = _arm_pair(rng, kind)
    h = 1e-6
    nv = 7
    fd = np.zeros((3, nv))
    vel_fd = []
    for k in range(nv):
        e = np.zeros(nv)
        e[k] = h
        qp, qm = rigid.integrate(model, q, e), rigid.integrate(model, q, -e)
        fd[:, k] = (C.pair_jcv(model, qp, v, pair) - C.pair_jcv(model, qm, v, pair)) / (2 * h)
        vp, vm = rigid.body_velocities(model, qp, v), rigid.body_velocities(model, qm, v)
        vel_fd.append([(a - b) / (2 * h) for a, b in zip(vp, vm)])
    dcd = (C.dcd_dbody(model, q, pair, 0), C.dcd_dbody(model, q, pair, 1))
    terms = C.appc_dJcv_dq(model, q, v, pair, dcd)
    Rc, c, _ = C.pair_placement(model, q, pair)
    for body, sign in ((pair[1], -1.0), (pair[4], 1.0)):
        if body < 0:
            continue
        R, p = C.body_pose(model, q, body)
        X = C.motion_transform(R.T @ Rc, R.T @ (c - p))
        for k in range(nv):
            terms[:, k] += sign * (X @ vel_fd[k][body])[:3]
    assert np.abs(terms - fd).max() <= 1e-5 * max(1.0, np.abs(fd).max())
    # and the placement terms matter: without them the sum is off
    assert np.abs(C.appc_dJcv_dq(model, q, v, pair, dcd)).max() > 1e-3


@pytest.mark.parametrize("kind", ["self", "world"])
def test_appc_transposed_terms(kind):
    """The second App. C term, d(J_c^T lambda)/dq from the contact placement, by duality with the
    first: it equals central differences of q -> J_c(q)^T lambda with the contact frame recomputed
    at every q minus those with the transforms cX_i held (only the bodies' Jacobians J_i(q)
    varying, the part App. C leaves to the other terms); J_c v agrees with J_c times v."""
    from oracle import rigid
    rng = np.random.default_rng(10 if kind == "self" else 11)
    model, q, v, pair = _arm_pair(rng, kind)
    lam = rng.normal(size=3)
    assert np.allclose(C.pair_jc(model, q, pair) @ v, C.pair_jcv(model, q, v, pair), atol=1e-12)
    transforms = C.pair_transforms(model, q, pair)
    h, nv = 1e-6, 7
    moving = np.zeros((nv, nv))
    held = np.zeros((nv, nv))
    for k in range(nv):
        e = np.zeros(nv)
        e[k] = h
        qp, qm = rigid.integrate(model, q, e), rigid.integrate(model, q, -e)
        moving[:, k] = (C.pair_jc(model, qp, pair).T @ lam - C.pair_jc(model, qm, pair).T @ lam) / (2 * h)
        held[:, k] = (C.pair_jc(model, qp, pair, transforms).T @ lam - C.pair_jc(model, qm, pair, transforms).T @ lam) / (2 * h)
    dcd = (C.dcd_dbody(model, q, pair, 0), C.dcd_dbody(model, q, pair, 1))
    terms = C.appc_dJctlam_dq(model, q, lam, pair, dcd)
    assert np.abs(terms - (moving - held)).max() <= 1e-5 * max(1.0, np.abs(moving).max())


def test_witness_on_a_triangulated_face_diagonal():
    """A sphere straight above the centre of a box face: the closest point of the Minkowski
    difference lies on the diagonal through which Qhull triangulates that face, where the two
    triangles tie in distance to rounding.  The closed form (n = -e_z from the sphere to the box,
    phi = height - r - half height, c straight below the centre) must hold to rounding, also for
    lateral offsets of 1e-12 to 1e-9 (the edge foot of the wrong triangle is off by ~1e-10)."""
    for dx in (0.0, 1e-12, -3e-11, 2e-10, 1e-9):
        for h in (0.07, 0.1, 0.2):
            r = C.collide(C.sphere(0.05), I3, np.array([dx, -dx, h]), C.box(0.3, 0.2, 0.04), I3, np.zeros(3))
            assert np.abs(r["n"] - [0.0, 0.0, -1.0]).max() <= 1e-14
            assert abs(r["phi"] - (h - 0.05 - 0.04)) <= 1e-14
            assert np.abs(r["c"][:2] - [dx, -dx]).max() <= 1e-14


@pytest.mark.parametrize("kind", ["self", "world"])
def test_smoothed_dcd_with_orthogonal_samples_is_central_differences(kind):
    """App. C's randomized-smoothing estimate of dCD/dM_i, 1/(2 S sigma^2) sum (f(+e) - f(-e)) e^T,
    fed the orthogonal design e = +-sigma sqrt(6) e_j (sum e e^T = S sigma^2 I, as for Gaussian
    samples in expectation) is exactly the central difference at step sigma sqrt(6); a wrong
    normalisation, sign or twist convention in the estimator breaks it.  With Gaussian samples it
    approaches the derivative as the samples grow (checked loosely: 20 % at 300 samples)."""
    rng = np.random.default_rng(12 if kind == "self" else 13)
    model, q, v, pair = _arm_pair(rng, kind)
    sigma = 1e-6
    design = np.sqrt(6.0) * sigma * np.eye(6)
    for which in ((0, 1) if kind == "self" else (0,)):
        est = C.dcd_dbody_smoothed(model, q, pair, which, sigma, design)
        ref = C.dcd_dbody(model, q, pair, which, h=np.sqrt(6.0) * sigma)
        assert np.abs(est - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())
    gauss = C.dcd_dbody_smoothed(model, q, pair, 0, 1e-4, rng.normal(0.0, 1e-4, size=(300, 6)))
    ref = C.dcd_dbody(model, q, pair, 0)
    assert np.abs(gauss - ref).max() <= 0.2 * np.abs(ref).max()
