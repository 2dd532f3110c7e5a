"""Rigid multibody dynamics in body coordinates (oracle).  Test infrastructure only.

Textbook recursions (Featherstone, *Rigid Body Dynamics Algorithms*, 2008): forward kinematics,
RNEA (inverse dynamics), CRBA (joint-space inertia M), ABA (forward dynamics, the paper's UFD
with external forces, Sec. 2.3 / Eq. 3) and a plain Cholesky factorisation.  Spatial vectors are
6-vectors ordered (linear, angular); a body's spatial velocity is expressed in its own frame at its
own origin.  All functions accept real or complex arrays (complex-step differentiation).
"""
import numpy as np

REVOLUTE, FREEFLYER = 0, 1


def skew(a):
    z = 0.0 * a[0]
    return np.array([[z, -a[2], a[1]], [a[2], z, -a[0]], [-a[1], a[0], z]])


def cross(a, b):
    return np.array([a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]])


def rodrigues(axis, angle):
    """Rotation by ``angle`` about the unit vector ``axis``: I + sin K + (1 - cos) K^2."""
    K = skew(np.asarray(axis, dtype=float))
    return np.eye(3) + np.sin(angle) * K + (1.0 - np.cos(angle)) * (K @ K)


def quat_to_rot(quat):
    """Rotation matrix of the quaternion (w, x, y, z), normalised first."""
    n = np.sqrt(quat @ quat)
    w, x, y, z = quat / n
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def quat_mul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


def quat_exp(w):
    """Unit quaternion of the rotation vector ``w`` (Taylor series near 0 keeps it analytic)."""
    t2 = w @ w
    if abs(t2) < 1e-10:
        c = 1 - t2 / 8 + t2 * t2 / 384
        s = 0.5 - t2 / 48 + t2 * t2 / 3840
    else:
        t = np.sqrt(t2)
        c, s = np.cos(t / 2), np.sin(t / 2) / t
    return np.concatenate([[c], s * w])


def nq_of(jt):
    return 7 if jt == FREEFLYER else 1


def nv_of(jt):
    return 6 if jt == FREEFLYER else 1


def index_maps(model):
    iq, iv, kq, kv = [], [], 0, 0
    for jt in model.jtype:
        iq.append(kq); iv.append(kv)
        kq += nq_of(jt); kv += nv_of(jt)
    return iq, iv, kq, kv


def joint_pose(model, i, q, iq):
    """Pose (E, r) of body i in its parent's frame: rotation E (body axes in parent coordinates)
    and origin r (parent coordinates) = joint placement composed with the joint motion."""
    Rt, pt = model.jrot[i], model.jpos[i]
    k = iq[i]
    if model.jtype[i] == REVOLUTE:
        return Rt @ rodrigues(model.axis[i], q[k]), pt + 0.0 * q[k]
    pos, quat = q[k:k + 3], q[k + 3:k + 7]
    return Rt @ quat_to_rot(quat), pt + Rt @ pos


def subspace(model, i):
    """Motion subspace S_i (6 x n_i) in body coordinates."""
    if model.jtype[i] == REVOLUTE:
        return np.concatenate([np.zeros(3), model.axis[i]])[:, None]
    return np.eye(6)


def fk(model, q):
    """Parent-relative poses [(E, r)] and world poses [(R, p)] of every body."""
    iq, _, _, _ = index_maps(model)
    rel, world = [], []
    for i in range(len(model.parent)):
        E, r = joint_pose(model, i, q, iq)
        rel.append((E, r))
        par = model.parent[i]
        if par < 0:
            world.append((E, r))
        else:
            Rp, pp = world[par]
            world.append((Rp @ E, pp + Rp @ r))
    return rel, world


# spatial algebra ---------------------------------------------------------------------------

def xm(E, r, m):
    """Motion vector from parent coordinates to body coordinates."""
    v, w = m[:3], m[3:]
    return np.concatenate([E.T @ (v + cross(w, r)), E.T @ w])


def xf_to_parent(E, r, f):
    """Force from body coordinates to parent coordinates."""
    fl = E @ f[:3]
    return np.concatenate([fl, E @ f[3:] + cross(r, fl)])


def mcross(a, b):
    """Motion cross product a x b."""
    return np.concatenate([cross(a[3:], b[:3]) + cross(a[:3], b[3:]), cross(a[3:], b[3:])])


def fcross(a, f):
    """Force cross product a x* f."""
    return np.concatenate([cross(a[3:], f[:3]), cross(a[3:], f[3:]) + cross(a[:3], f[:3])])


def inertia_matrix_com(model, i):
    xx, yy, zz, xy, xz, yz = model.inertia[i]
    return np.array([[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]])


def inertia_apply(model, i, m):
    """Spatial inertia of body i (body coordinates, about its origin) times motion m."""
    mass, c = model.mass[i], model.com[i]
    lin = mass * (m[:3] + cross(m[3:], c))
    return np.concatenate([lin, cross(c, lin) + inertia_matrix_com(model, i) @ m[3:]])


def inertia6(model, i):
    mass, c = model.mass[i], np.asarray(model.com[i])
    C = skew(c)
    return np.block([[mass * np.eye(3), -mass * C], [mass * C, inertia_matrix_com(model, i) - mass * C @ C]])


def xm6(E, r):
    """6x6 motion transform, parent -> body coordinates."""
    Et = E.T
    Z = np.zeros((3, 3))
    return np.block([[Et, -Et @ skew(r)], [Z, Et]])


# algorithms ----------------------------------------------------------------------------------

def rnea(model, q, v, a, gravity, fext=None):
    """Inverse dynamics tau = M a + b(q, v) - sum_i J_i^T fext_i (RNEA).  ``fext[i]`` is a spatial
    force on body i in its own coordinates."""
    iq, iv, _, nv = index_maps(model)
    rel, _ = fk(model, q)
    nb = len(model.parent)
    dt = np.result_type(q, v, a, gravity, 1.0)
    vel, acc, frc = [None] * nb, [None] * nb, [None] * nb
    for i in range(nb):
        E, r = rel[i]
        S = subspace(model, i)
        n = S.shape[1]
        qd, qdd = v[iv[i]:iv[i] + n], a[iv[i]:iv[i] + n]
        par = model.parent[i]
        if par < 0:
            vp = np.zeros(6, dtype=dt)
            ap = np.concatenate([-np.asarray(gravity), np.zeros(3)])
        else:
            vp, ap = vel[par], acc[par]
        vj = S @ qd
        vel[i] = xm(E, r, vp) + vj
        acc[i] = xm(E, r, ap) + S @ qdd + mcross(vel[i], vj)
        frc[i] = inertia_apply(model, i, acc[i]) + fcross(vel[i], inertia_apply(model, i, vel[i]))
        if fext is not None:
            frc[i] = frc[i] - fext[i]
    tau = np.zeros(nv, dtype=np.result_type(dt, *frc))
    for i in reversed(range(nb)):
        S = subspace(model, i)
        tau[iv[i]:iv[i] + S.shape[1]] = S.T @ frc[i]
        par = model.parent[i]
        if par >= 0:
            E, r = rel[i]
            frc[par] = frc[par] + xf_to_parent(E, r, frc[i])
    return tau


def crba(model, q):
    """Joint-space inertia matrix M(q) by the composite-rigid-body algorithm."""
    iq, iv, _, nv = index_maps(model)
    rel, _ = fk(model, q)
    nb = len(model.parent)
    X = [xm6(*rel[i]) for i in range(nb)]
    IC = [inertia6(model, i) + 0.0 * X[i][0, 0] for i in range(nb)]
    M = np.zeros((nv, nv), dtype=IC[0].dtype)
    for i in reversed(range(nb)):
        par = model.parent[i]
        if par >= 0:
            IC[par] = IC[par] + X[i].T @ IC[i] @ X[i]
    for i in range(nb):
        S = subspace(model, i)
        F = IC[i] @ S
        M[iv[i]:iv[i] + S.shape[1], iv[i]:iv[i] + S.shape[1]] = S.T @ F
        j = i
        while model.parent[j] >= 0:
            F = X[j].T @ F
            j = model.parent[j]
            Sj = subspace(model, j)
            blk = F.T @ Sj
            M[iv[i]:iv[i] + S.shape[1], iv[j]:iv[j] + Sj.shape[1]] = blk
            M[iv[j]:iv[j] + Sj.shape[1], iv[i]:iv[i] + S.shape[1]] = blk.T
    return M


def aba(model, q, v, tau, gravity, fext=None):
    """Forward dynamics qdd = M^-1 (tau - b + sum J^T fext) by the articulated-body algorithm."""
    iq, iv, _, nv = index_maps(model)
    rel, _ = fk(model, q)
    nb = len(model.parent)
    dt = np.result_type(q, v, tau, 1.0)
    X = [xm6(*rel[i]) for i in range(nb)]
    vel, cc, IA, pA = [None] * nb, [None] * nb, [None] * nb, [None] * nb
    for i in range(nb):
        S = subspace(model, i)
        n = S.shape[1]
        par = model.parent[i]
        vp = np.zeros(6, dtype=dt) if par < 0 else vel[par]
        vj = S @ v[iv[i]:iv[i] + n]
        vel[i] = X[i] @ vp + vj
        cc[i] = mcross(vel[i], vj)
        IA[i] = inertia6(model, i) + 0.0 * X[i][0, 0]
        pA[i] = fcross(vel[i], inertia_apply(model, i, vel[i]))
        if fext is not None:
            pA[i] = pA[i] - fext[i]
    U, Dinv, u = [None] * nb, [None] * nb, [None] * nb
    for i in reversed(range(nb)):
        S = subspace(model, i)
        n = S.shape[1]
        U[i] = IA[i] @ S
        Dinv[i] = np.linalg.inv(S.T @ U[i])
        u[i] = tau[iv[i]:iv[i] + n] - S.T @ pA[i]
        par = model.parent[i]
        if par >= 0:
            Ia = IA[i] - U[i] @ Dinv[i] @ U[i].T
            pa = pA[i] + Ia @ cc[i] + U[i] @ (Dinv[i] @ u[i])
            IA[par] = IA[par] + X[i].T @ Ia @ X[i]
            pA[par] = pA[par] + X[i].T @ pa
    qdd = np.zeros(nv, dtype=np.result_type(dt, IA[0], pA[0], u[0]))
    acc = [None] * nb
    for i in range(nb):
        S = subspace(model, i)
        n = S.shape[1]
        par = model.parent[i]
        ap = np.concatenate([-np.asarray(gravity), np.zeros(3)]) if par < 0 else acc[par]
        a = X[i] @ ap + cc[i]
        qi = Dinv[i] @ (u[i] - U[i].T @ a)
        qdd[iv[i]:iv[i] + n] = qi
        acc[i] = a + S @ qi
    return qdd


def cholesky(M):
    """Lower-triangular L with L L^T = M (no pivoting; M symmetric positive definite)."""
    n = M.shape[0]
    L = np.zeros_like(M)
    for j in range(n):
        L[j, j] = np.sqrt(M[j, j] - L[j, :j] @ L[j, :j])
        for i in range(j + 1, n):
            L[i, j] = (M[i, j] - L[i, :j] @ L[j, :j]) / L[j, j]
    return L


def chol_solve(L, B):
    """Solve (L L^T) X = B by forward and back substitution."""
    B = np.asarray(B)
    vec = B.ndim == 1
    Y = np.array(B.reshape(B.shape[0], -1), dtype=np.result_type(L, B))
    n = L.shape[0]
    for i in range(n):
        Y[i] = (Y[i] - L[i, :i] @ Y[:i]) / L[i, i]
    for i in reversed(range(n)):
        Y[i] = (Y[i] - L[i + 1:, i] @ Y[i + 1:]) / L[i, i]
    return Y[:, 0] if vec else Y


def body_velocities(model, q, v):
    """Spatial velocity of every body (body coordinates)."""
    iq, iv, _, _ = index_maps(model)
    rel, _ = fk(model, q)
    out = []
    for i in range(len(model.parent)):
        S = subspace(model, i)
        par = model.parent[i]
        vp = np.zeros(6, dtype=np.result_type(v, 1.0)) if par < 0 else out[par]
        out.append(xm(*rel[i], vp) + S @ v[iv[i]:iv[i] + S.shape[1]])
    return out


def body_jacobians(model, q):
    """J_i (6 x nv) with body velocity v_i = J_i v (body coordinates), one unit velocity at a time."""
    _, _, _, nv = index_maps(model)
    cols = [body_velocities(model, q, np.eye(nv)[k]) for k in range(nv)]
    return [np.stack([cols[k][i] for k in range(nv)], axis=1) for i in range(len(model.parent))]


def integrate(model, q, dv):
    """q (+) dv: revolute q + dv; free-flyer position += R dv_lin (body-frame translation) and
    quaternion <- quaternion * exp(dv_ang / 2), renormalised."""
    iq, iv, _, _ = index_maps(model)
    out = np.array(q, dtype=np.result_type(q, dv, 1.0))
    for i, jt in enumerate(model.jtype):
        k, j = iq[i], iv[i]
        if jt == REVOLUTE:
            out[k] = q[k] + dv[j]
        else:
            quat = q[k + 3:k + 7]
            R = quat_to_rot(quat)
            out[k:k + 3] = q[k:k + 3] + R @ dv[j:j + 3]
            nq = quat_mul(quat, quat_exp(dv[j + 3:j + 6]))
            out[k + 3:k + 7] = nq / np.sqrt(nq @ nq)
    return out


def local_difference(model, q0, q1):
    """The tangent eta with q0 (+) eta = q1 to first order in (q1 - q0): revolute q1 - q0; free-flyer
    R0^T (p1 - p0) and 2 vec(conj(quat0) * quat1) (the first-order quaternion logarithm, quaternions
    normalised).  Exact for complex-step derivatives of maps into q, whose second-order terms do not
    reach the imaginary part."""
    iq, iv, _, _ = index_maps(model)
    out = np.zeros(sum(nv_of(jt) for jt in model.jtype), dtype=np.result_type(q0, q1, 1.0))
    for i, jt in enumerate(model.jtype):
        k, j = iq[i], iv[i]
        if jt == REVOLUTE:
            out[j] = q1[k] - q0[k]
        else:
            a, b = q0[k + 3:k + 7], q1[k + 3:k + 7]
            a = a / np.sqrt(a @ a)
            b = b / np.sqrt(b @ b)
            out[j:j + 3] = quat_to_rot(a).T @ (q1[k:k + 3] - q0[k:k + 3])
            conj = np.array([a[0], -a[1], -a[2], -a[3]])
            out[j + 3:j + 6] = 2.0 * quat_mul(conj, b)[1:]
    return out


def tangent_to_raw_jacobian(model, q):
    """d q_raw / d eta at q (nq x nv): complex step of integrate(q, eta) at eta = 0."""
    nv = sum(nv_of(jt) for jt in model.jtype)
    J = np.zeros((len(q), nv))
    for j in range(nv):
        e = np.zeros(nv, dtype=complex)
        e[j] = 1e-30j
        J[:, j] = np.imag(integrate(model, np.asarray(q, float), e)) / 1e-30
    return J


def raw_to_tangent_jacobian(model, q):
    """d eta / d q_raw at q (nv x nq): complex step of local_difference(q, q + dq_raw) at dq_raw = 0."""
    q = np.asarray(q, float)
    J = np.zeros((sum(nv_of(jt) for jt in model.jtype), len(q)))
    for j in range(len(q)):
        e = np.zeros(len(q), dtype=complex)
        e[j] = 1e-30j
        J[:, j] = np.imag(local_difference(model, q, q + e)) / 1e-30
    return J


def gravity_potential(model, q, gravity):
    """U(q) = -sum_i m_i g . x_com,i  (gravity potential energy)."""
    _, world = fk(model, q)
    U = 0.0
    for i, (R, p) in enumerate(world):
        U = U - model.mass[i] * (np.asarray(gravity) @ (p + R @ model.com[i]))
    return U
