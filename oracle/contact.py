"""Contact geometry against a plane and the contact Jacobian (oracle).  Test infrastructure only.

Collision detection (Sec. 2.1) reduced to the analytic primitive-versus-plane case: a contact slot
is a reference point x on a body (sphere centre, or a box corner with radius 0).  The signed
distance is phi = n.x - d - r and the slot is active iff phi <= 0.  The contact frame c has its
origin at the contact point x - r n and its Z axis along the plane normal (Sec. 2.1); its tangent
axes are t1 = normalize(e_x - (n.e_x) n) (or e_y when |n.e_x| > 0.9) and t2 = n x t1.  Contact
force and velocity triplets are ordered (T1, T2, N), normal last (Eq. 1, Gamma_mu = [0, 0, mu||s_T||]).

The contact Jacobian J_c = E ( cX_1 J_1 ) (App. C, Eq. contact_jaco; body 2 is the static plane so
J_2 = 0) maps joint velocities to the linear velocity, in the contact frame, of the point of body 1
that coincides with the contact point.
"""
import numpy as np

from .rigid import body_jacobians, cross, fk


def tangent_basis(n):
    n = np.asarray(n, dtype=float)
    e = np.array([1.0, 0.0, 0.0]) if abs(n[0]) <= 0.9 else np.array([0.0, 1.0, 0.0])
    t1 = e - (n @ e) * n
    t1 = t1 / np.sqrt(t1 @ t1)
    t2 = cross(n, t1)
    return t1, t2


def active_slots(model, q, env, margin=0.0):
    """Indices of the active contact slots, decided on the real part: phi <= margin (the activation
    distance; 0 unless a margin is set, see step.py)."""
    _, world = fk(model, np.real(q))
    n, d = env["plane"][:3], env["plane"][3]
    out = []
    for k, b in enumerate(env["c_link"]):
        if b < 0:
            continue
        R, p = world[b]
        x = p + R @ env["c_point"][k]
        phi = n @ x - d - env["c_radius"][k]
        if phi <= margin:
            out.append(k)
    return out


def contact_points(model, q, env, slots):
    """World contact points c_k = x_k - r_k n (x_k = body reference point) for the given slots."""
    _, world = fk(model, q)
    n = env["plane"][:3]
    pts = []
    for k in slots:
        R, p = world[env["c_link"][k]]
        pts.append(p + R @ env["c_point"][k] - env["c_radius"][k] * n)
    return pts


def signed_distances(model, q, env, slots):
    """phi_k = n . x_k - d - r_k of the given slots (= n . c_k - d with the contact point c_k)."""
    n, d = env["plane"][:3], env["plane"][3]
    return np.array([n @ c - d for c in contact_points(model, q, env, slots)])


def contact_jacobian(model, q, env, slots):
    """J_c (3 nc x nv): rows (t1, t2, n) . (velocity of body point at c_k)."""
    _, world = fk(model, q)
    Jb = body_jacobians(model, q)
    n = env["plane"][:3]
    t1, t2 = tangent_basis(n)
    Rc = np.stack([t1, t2, n])
    rows = []
    for k, c in zip(slots, contact_points(model, q, env, slots)):
        b = env["c_link"][k]
        R, p = world[b]
        lin = R @ Jb[b][:3]
        ang = R @ Jb[b][3:]
        Jp = lin + np.stack([cross(ang[:, j], c - p) for j in range(ang.shape[1])], axis=1)
        rows.append(Rc @ Jp)
    if not rows:
        return np.zeros((0, Jb[0].shape[1]), dtype=Jb[0].dtype)
    return np.concatenate(rows, axis=0)


def contact_wrenches(model, q, env, slots, lam, scale=1.0):
    """Spatial forces (body coordinates, body origin) on every body from contact impulses ``lam``
    (3 per active slot, frame coordinates) divided by ``scale`` (the time step: impulse -> force)."""
    rel, world = fk(model, q)
    nb = len(model.parent)
    n = env["plane"][:3]
    t1, t2 = tangent_basis(n)
    dt = np.result_type(q, lam, 1.0)
    f = [np.zeros(6, dtype=dt) for _ in range(nb)]
    for j, (k, c) in enumerate(zip(slots, contact_points(model, q, env, slots))):
        b = env["c_link"][k]
        R, p = world[b]
        fw = (t1 * lam[3 * j] + t2 * lam[3 * j + 1] + n * lam[3 * j + 2]) / scale
        fb = R.T @ fw
        f[b] = f[b] + np.concatenate([fb, cross(R.T @ (c - p), fb)])
    return f
