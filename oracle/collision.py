"""Collision detection between convex shapes and its derivative by randomized smoothing (oracle).
Test infrastructure only; not yet wired into the step (which keeps primitive-versus-plane
contacts, contact.py).

Sec. 2.1: given two convex shapes and their poses, collision detection returns a contact point and
a contact normal, the direction separating the shapes with minimal displacement; the contact frame
has its origin at the contact point and its Z axis along the normal.  App. C writes the contact
placement as 0M_c = CD(0M_1, 0M_2) and needs dCD/dM_i, which the paper takes from a randomized
smoothing estimator (zero-order: the expectation of CD's response to random tangent perturbations
of the poses).

The plain definition is computed here, not GJK/EPA's iteration.  Every shape is a core (a point,
a segment or a convex polytope given by its vertices) swept by a radius r >= 0 (sphere = point + r,
capsule = segment + r, box = its 8 corners + 0).  The signed distance of A and B is the distance of
their cores minus rA + rB when the cores are apart, and minus (penetration depth of the cores +
rA + rB) when they overlap.  Between cores it is computed from the Minkowski difference
D = core_A - core_B:

* apart: the closest point of D to the origin, -n d with d = dist(0, D), gives the witness points
  (the same convex weights on A's and B's points) and the normal n (unit, from A towards B);
* overlapping (a polytope core on either side): the facet of conv(D) nearest the origin gives the
  depth and the normal (n is that facet's outward normal: translating A by -depth n separates the
  cores), and the projection of the origin onto that facet the witness points.

Points and segments use their closed forms; a polytope core uses the convex hull of D (scipy's
Qhull) and the exact closest point of each hull triangle to the origin.  The contact point is the
midpoint of the two witness points moved to the shapes' surfaces (pA + rA n, pB - rB n)."""
import numpy as np
from scipy.spatial import ConvexHull


class Shape:
    """A convex shape: core points in the body frame (1 = point, 2 = segment, >= 4 = polytope
    vertices) and a radius."""

    def __init__(self, core, radius=0.0):
        self.core = np.atleast_2d(np.asarray(core, dtype=float))
        self.radius = float(radius)


def sphere(r):
    return Shape([[0.0, 0.0, 0.0]], r)


def capsule(half_length, r):
    """Segment along the body z axis from -half_length to +half_length, swept by r."""
    return Shape([[0.0, 0.0, -half_length], [0.0, 0.0, half_length]], r)


def box(hx, hy, hz):
    return Shape([[sx * hx, sy * hy, sz * hz] for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)], 0.0)


def world_core(shape, R, p):
    return shape.core @ np.asarray(R, float).T + np.asarray(p, float)


def closest_on_segment(a, b, x):
    """Closest point of segment [a, b] to x and its parameter t in [0, 1]."""
    ab = b - a
    den = ab @ ab
    t = 0.0 if den == 0.0 else min(1.0, max(0.0, (x - a) @ ab / den))
    return a + t * ab, t


def closest_segments(p1, q1, p2, q2):
    """Closest points of segments [p1, q1] and [p2, q2]: the minimum of |p1 + s d1 - p2 - t d2|^2
    over [0, 1]^2 is the unconstrained minimum when it lies inside the square, else on one of the
    square's four edges, where it is a point-to-segment problem."""
    d1, d2 = q1 - p1, q2 - p2
    a, b, e = d1 @ d1, d1 @ d2, d2 @ d2
    r = p1 - p2
    den = a * e - b * b
    if den > 1e-14 * max(a * e, 1e-300):
        s = (b * (d2 @ r) - e * (d1 @ r)) / den
        t = (a * (d2 @ r) - b * (d1 @ r)) / den
        if 0.0 <= s <= 1.0 and 0.0 <= t <= 1.0:
            return p1 + s * d1, p2 + t * d2
    best = None
    for x, (ya, yb), first in ((p1, (p2, q2), True), (q1, (p2, q2), True), (p2, (p1, q1), False), (q2, (p1, q1), False)):
        y, _ = closest_on_segment(ya, yb, x)
        dist = np.sum((x - y) ** 2)
        if best is None or dist < best[0]:
            best = (dist, (x, y) if first else (y, x))
    return best[1][0].copy(), best[1][1].copy()


def closest_on_triangle(a, b, c, x=np.zeros(3)):
    """Barycentric weights (wa, wb, wc) of the closest point of triangle abc to x: the projection of
    x on the triangle's plane when it falls inside the triangle, else the nearest of the closest
    points on the three edges."""
    ab, ac = b - a, c - a
    nrm = np.cross(ab, ac)
    nn = nrm @ nrm
    if nn > 1e-300:
        # barycentric coordinates of the projection of x
        v = np.cross(x - a, ac) @ nrm / nn
        w = np.cross(ab, x - a) @ nrm / nn
        if v >= 0.0 and w >= 0.0 and v + w <= 1.0:
            return np.array([1.0 - v - w, v, w])
    best = None
    for (i, j) in ((0, 1), (1, 2), (0, 2)):
        pts = (a, b, c)
        y, t = closest_on_segment(pts[i], pts[j], x)
        dist = np.sum((x - y) ** 2)
        if best is None or dist < best[0]:
            wts = np.zeros(3)
            wts[i], wts[j] = 1.0 - t, t
            best = (dist, wts)
    return best[1]


def _hull_core_distance(ca, cb):
    """Signed distance of two cores of which one is a polytope, their witness points and the normal
    from A to B, from the convex hull of their Minkowski difference."""
    ia, ib = np.meshgrid(np.arange(len(ca)), np.arange(len(cb)), indexing="ij")
    ia, ib = ia.ravel(), ib.ravel()
    D = ca[ia] - cb[ib]
    hull = ConvexHull(D)
    off = hull.equations[:, 3]                       # n.x + off <= 0 inside, |n| = 1
    if np.all(off <= 0.0):
        # overlapping: the nearest facet plane (origin inside conv(D))
        k = int(np.argmax(off))
        m = hull.equations[k, :3]
        depth = -off[k]
        y = depth * m
        best = None
        for f, simplex in enumerate(hull.simplices):
            if not np.allclose(hull.equations[f], hull.equations[k], atol=1e-12):
                continue
            w = closest_on_triangle(*D[simplex], x=y)
            err = np.sum((w @ D[simplex] - y) ** 2)
            if best is None or err < best[0]:
                best = (err, simplex, w)
        _, simplex, w = best
        return -depth, w @ ca[ia[simplex]], w @ cb[ib[simplex]], m
    # the closest point of conv(D) to the origin is unique, but where it lies on an edge shared by
    # two hull triangles (a face of D triangulated through it) the two candidates tie in distance
    # to rounding while the edge foot of the wrong one is off by the square root of it; among
    # such ties the triangle that contains the projection (all weights > 0) gives the point
    cands = []
    for simplex in hull.simplices:
        w = closest_on_triangle(*D[simplex])
        y = w @ D[simplex]
        cands.append((y @ y, simplex, w, y))
    d2min = min(c[0] for c in cands)
    ties = [c for c in cands if c[0] <= d2min * (1.0 + 1e-12)]
    interior = [c for c in ties if np.all(c[2] > 0.0)]
    d2, simplex, w, y = min(interior or ties, key=lambda c: c[0])
    d = np.sqrt(d2)
    return d, w @ ca[ia[simplex]], w @ cb[ib[simplex]], -y / d


def core_distance(ca, cb):
    """Signed distance of cores ca, cb (world points: 1 = point, 2 = segment, more = polytope), the
    witness points on each and the unit normal from A to B.  Touching or crossing point and segment
    cores have no defined normal; the world z axis is returned for them."""
    if len(ca) <= 2 and len(cb) <= 2:
        sa = (ca[0], ca[-1])
        sb = (cb[0], cb[-1])
        pa, pb = closest_segments(sa[0], sa[1], sb[0], sb[1])
        d = np.sqrt(np.sum((pb - pa) ** 2))
        n = (pb - pa) / d if d > 1e-300 else np.array([0.0, 0.0, 1.0])
        return d, pa, pb, n
    return _hull_core_distance(ca, cb)


def tangent_basis(n):
    """Tangent axes of the contact frame for the unit normal n (the rule of contact.py: t1 =
    normalize(e_x - (n.e_x) n), e_y when |n_x| > 0.9; t2 = n x t1)."""
    e = np.array([1.0, 0.0, 0.0]) if abs(n[0]) <= 0.9 else np.array([0.0, 1.0, 0.0])
    t1 = e - (n @ e) * n
    t1 = t1 / np.sqrt(t1 @ t1)
    return t1, np.cross(n, t1)


def collide(shape_a, Ra, pa, shape_b, Rb, pb):
    """Collision detection of Sec. 2.1 for shapes A and B at world poses (R, p): returns a dict with
    the signed distance phi (< 0: penetration), the witness points on the shapes' surfaces, the
    contact point c (their midpoint), the unit normal n from A to B, and the contact frame's
    rotation Rc (columns t1, t2, n: Z along the normal)."""
    ca, cb = world_core(shape_a, Ra, pa), world_core(shape_b, Rb, pb)
    d, wa, wb, n = core_distance(ca, cb)
    phi = d - shape_a.radius - shape_b.radius
    sa, sb = wa + shape_a.radius * n, wb - shape_b.radius * n
    t1, t2 = tangent_basis(n)
    return {"phi": phi, "pa": sa, "pb": sb, "c": 0.5 * (sa + sb), "n": n,
            "Rc": np.stack([t1, t2, n], axis=1)}


def twist_pose(R, p, xi):
    """The pose (R, p) moved by the world-frame twist xi = (u, w) (linear, angular at the world
    origin): x -> exp([w]) x + V(w) u, i.e. R' = exp([w]) R, p' = exp([w]) p + V(w) u."""
    u, w = np.asarray(xi[:3], float), np.asarray(xi[3:], float)
    th = np.sqrt(w @ w)
    W = np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])
    if th < 1e-12:
        E, V = np.eye(3) + W, np.eye(3) + 0.5 * W
    else:
        E = np.eye(3) + np.sin(th) / th * W + (1 - np.cos(th)) / th ** 2 * W @ W
        V = np.eye(3) + (1 - np.cos(th)) / th ** 2 * W + (th - np.sin(th)) / th ** 3 * W @ W
    return E @ R, E @ p + V @ u


def cd_features(res):
    """The smoothed quantities: phi, the contact point and the normal (7 numbers)."""
    return np.concatenate([[res["phi"]], res["c"], res["n"]])


def randomized_smoothing_jacobian(shape_a, Ra, pa, shape_b, Rb, pb, sigma, samples, rng, eps_samples=None):
    """Zero-order randomized-smoothing estimate of the derivative of (phi, c, n) with respect to the
    world-frame twists of A's and B's poses (7 x 12; columns: A's (u, w), then B's): with eps ~
    N(0, sigma^2 I_12) the expectation of (f(eps) - f(-eps)) eps^T / (2 sigma^2), the gradient of
    the Gaussian-smoothed f (antithetic pairs; unbiased for the smoothed function).  The samples are
    drawn from rng, or taken from eps_samples (samples x 12, already scaled by sigma) when given."""
    acc = np.zeros((7, 12))
    for s in range(samples):
        eps = rng.normal(0.0, sigma, size=12) if eps_samples is None else np.asarray(eps_samples[s], float)
        fp = cd_features(collide(shape_a, *twist_pose(Ra, pa, eps[:6]), shape_b, *twist_pose(Rb, pb, eps[6:])))
        fm = cd_features(collide(shape_a, *twist_pose(Ra, pa, -eps[:6]), shape_b, *twist_pose(Rb, pb, -eps[6:])))
        acc += np.outer(fp - fm, eps)
    return acc / (2.0 * sigma ** 2 * samples)


# ------------------------------------------------------------------- contacts between two bodies
# App. C: a contact between body 1 and body 2 has J_c = E (cX_1 J_1 - cX_2 J_2) (E: the linear
# part, J_i body Jacobians in body coordinates, cX_i the motion transform from body i to the
# contact frame).  Here body A is 1's counterpart with the opposite sign: J_c v is the velocity of
# B's material point at the contact point relative to A's, in the contact frame whose Z axis is the
# normal from A to B, so sigma_N > 0 separates (the convention of the plane contacts, where A is the
# plane).  A body index of -1 is the fixed world.

def _skew(a):
    return np.array([[0.0, -a[2], a[1]], [a[2], 0.0, -a[0]], [-a[1], a[0], 0.0]])


def motion_transform(E, r):
    """6x6 transform of motion vectors (linear, angular) from a frame to the frame at (E, r) in it."""
    Et = E.T
    return np.block([[Et, -Et @ _skew(r)], [np.zeros((3, 3)), Et]])


def motion_cross(a, b):
    """Spatial motion cross product a x b, vectors (linear, angular)."""
    return np.concatenate([np.cross(a[3:], b[:3]) + np.cross(a[:3], b[3:]), np.cross(a[3:], b[3:])])


def body_pose(model, q, body):
    from .rigid import fk
    if body < 0:
        return np.eye(3), np.zeros(3)
    R, p = fk(model, q)[1][body]
    return np.asarray(R, float), np.asarray(p, float)


def pair_placement(model, q, pair, poses=None):
    """Contact placement (Rc, c) and the collision result of pair = (shape_a, body_a, (Ea, ra),
    shape_b, body_b, (Eb, rb)), each shape at placement (E, r) in its body; poses, when given,
    replaces the bodies' world poses [(Ra, pa), (Rb, pb)]."""
    sa, ba, (Ea, ra), sb, bb, (Eb, rb) = pair
    (Ra, pa), (Rb, pb) = poses if poses is not None else (body_pose(model, q, ba), body_pose(model, q, bb))
    res = collide(sa, Ra @ Ea, pa + Ra @ ra, sb, Rb @ Eb, pb + Rb @ rb)
    return res["Rc"], res["c"], res


def pair_jcv(model, q, v, pair):
    """J_c v of the pair at (q, v): the linear part of cX_b V_b - cX_a V_a (V_i = J_i v, body
    coordinates; 0 for the world)."""
    from .rigid import body_velocities
    Rc, c, _ = pair_placement(model, q, pair)
    vel = body_velocities(model, q, v)
    out = np.zeros(3)
    for body, sign in ((pair[1], -1.0), (pair[4], 1.0)):
        if body < 0:
            continue
        R, p = body_pose(model, q, body)
        X = motion_transform(R.T @ Rc, R.T @ (c - p))
        out += sign * (X @ vel[body])[:3]
    return out


def local_twist(R0, p0, R1, p1):
    """First-order local twist taking (R0, p0) to (R1, p1): (R0^T (p1 - p0), vee(R0^T R1 - I))."""
    W = R0.T @ R1 - np.eye(3)
    return np.concatenate([R0.T @ (p1 - p0), 0.5 * np.array([W[2, 1] - W[1, 2], W[0, 2] - W[2, 0], W[1, 0] - W[0, 1]])])


def dcd_dbody(model, q, pair, which, h=1e-6):
    """dCD/dM_i (6 x 6) by central differences: the local twist of the contact placement per local
    twist of body i's pose (which = 0: A, 1: B), M_i -> M_i exp(delta)."""
    poses = [body_pose(model, q, pair[1]), body_pose(model, q, pair[4])]
    Rc, c, _ = pair_placement(model, q, pair, poses)
    out = np.zeros((6, 6))
    for j in range(6):
        cols = []
        for s in (h, -h):
            R, p = poses[which]
            d = np.zeros(6)
            d[j] = s
            # local twist of the body frame: R' = R exp([w]), p' = p + R u (first order is enough
            # for central differences of a smooth map)
            R2, p2 = twist_pose(np.eye(3), np.zeros(3), d)
            moved = list(poses)
            moved[which] = (R @ R2, p + R @ p2)
            Rc2, c2, _ = pair_placement(model, q, pair, moved)
            cols.append(local_twist(Rc, c, Rc2, c2))
        out[:, j] = (cols[0] - cols[1]) / (2 * h)
    return out


def dcd_dbody_smoothed(model, q, pair, which, sigma, eps_samples):
    """dCD/dM_i (6 x 6) by App. C's zero-order randomized smoothing: with local twists eps_s of body
    i's pose (the rows of eps_samples, S x 6, drawn from N(0, sigma^2 I)), the antithetic estimate
    1 / (2 S sigma^2) sum_s (f(+eps_s) - f(-eps_s)) eps_s^T of the Gaussian-smoothed derivative of f,
    the local twist of the contact placement (as in dcd_dbody) when body i moves to M_i exp(eps)."""
    poses = [body_pose(model, q, pair[1]), body_pose(model, q, pair[4])]
    Rc, c, _ = pair_placement(model, q, pair, poses)
    eps_samples = np.asarray(eps_samples, float)
    acc = np.zeros((6, 6))
    for eps in eps_samples:
        f = []
        for s in (1.0, -1.0):
            R, p = poses[which]
            R2, p2 = twist_pose(np.eye(3), np.zeros(3), s * eps)
            moved = list(poses)
            moved[which] = (R @ R2, p + R @ p2)
            Rc2, c2, _ = pair_placement(model, q, pair, moved)
            f.append(local_twist(Rc, c, Rc2, c2))
        acc += np.outer(f[0] - f[1], eps)
    return acc / (2.0 * sigma ** 2 * len(eps_samples))


def appc_dJcv_dq(model, q, v, pair, dcd):
    """App. C's contact-placement terms of d(J_c v)/dq at fixed v and fixed body velocities V_i:
    sum over the two bodies of the sign times E [ (cX_i V_i) x dCD/dM_i J_i - cX_i (V_i x J_i) ],
    the contact frame's twist collecting both bodies' contributions (nv columns).  dcd = (dCD/dM_a,
    dCD/dM_b)."""
    from .rigid import body_jacobians, body_velocities
    Rc, c, _ = pair_placement(model, q, pair)
    Js = body_jacobians(model, q)
    vel = body_velocities(model, q, v)
    nv = Js[0].shape[1]
    dc = np.zeros((6, nv))                       # local twist of the contact frame per dof
    for which, body in ((0, pair[1]), (1, pair[4])):
        if body >= 0:
            dc += dcd[which] @ Js[body]
    out = np.zeros((3, nv))
    for which, body, sign in ((0, pair[1], -1.0), (1, pair[4], 1.0)):
        if body < 0:
            continue
        R, p = body_pose(model, q, body)
        X = motion_transform(R.T @ Rc, R.T @ (c - p))
        W = X @ vel[body]
        for k in range(nv):
            term = motion_cross(W, dc[:, k]) - X @ motion_cross(vel[body], Js[body][:, k])
            out[:, k] += sign * term[:3]
    return out


def pair_transforms(model, q, pair):
    """The motion transforms cX_a, cX_b from the bodies to the contact frame at q (None for the
    world)."""
    Rc, c, _ = pair_placement(model, q, pair)
    out = []
    for body in (pair[1], pair[4]):
        if body < 0:
            out.append(None)
            continue
        R, p = body_pose(model, q, body)
        out.append(motion_transform(R.T @ Rc, R.T @ (c - p)))
    return out


def pair_jc(model, q, pair, transforms=None):
    """J_c (3 x nv) of the pair: column k is pair_jcv at v = e_k.  With ``transforms`` (cX_a, cX_b,
    as pair_transforms returns them) held, only the bodies' Jacobians J_i(q) vary with q."""
    from .rigid import body_jacobians
    Xs = transforms if transforms is not None else pair_transforms(model, q, pair)
    Js = body_jacobians(model, q)
    out = np.zeros((3, Js[0].shape[1]), dtype=np.result_type(Js[0], 1.0))
    for X, body, sign in ((Xs[0], pair[1], -1.0), (Xs[1], pair[4], 1.0)):
        if body < 0:
            continue
        out += sign * (X @ Js[body])[:3]
    return out


def appc_dJctlam_dq(model, q, lam, pair, dcd):
    """App. C's contact-placement terms of d(J_c^T lambda)/dq (nv x nv), from the duality
    <d(J_c^T lambda) dq, v> = <lambda, d(J_c v) dq> for every v: entry (j, k) is
    lambda . (placement terms of d(J_c e_j)/dq_k)."""
    from .rigid import index_maps
    nv = index_maps(model)[3]
    out = np.zeros((nv, nv))
    for j in range(nv):
        e = np.zeros(nv)
        e[j] = 1.0
        out[j] = np.asarray(lam, float) @ appc_dJcv_dq(model, q, e, pair, dcd)
    return out
