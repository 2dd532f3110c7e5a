"""Seeded synthetic workloads: kinematic-tree models, batches of states and contact descriptors.

This module is shared by the CUDA path, the oracle tests and the benchmark, and therefore holds no
step of the simulation method (no dynamics, no contact solve, no derivative).  The robots of the
paper's timing table (Sec. 4.1, Tab. 2: UR5, Go1, Atlas, ...) are not available, so seeded stand-ins
with the same degree-of-freedom and contact counts are generated here:

* ``arm7``        7-dof fixed-base serial arm, revolute joints about random unit axes (UR5-like size);
* ``quadruped18`` free-flyer + 4 legs x 3 revolute joints, point feet (Go1-like size);
* ``humanoid36``  free-flyer + 30 revolute joints in 5 chains, box feet (Atlas-like size).

The only geometry computed here is scene set-up: where the ground plane goes and which initial
joint velocities give a wanted cube velocity.  It uses scipy's ``Rotation`` and central finite
differences of body placements; the numbers it produces are inputs, never expected outputs.

Conventions shared by every consumer of a ``Batch`` (they are data layout, not arithmetic):

* body ``i``'s frame = parent frame * joint placement (``jrot[i]``, ``jpos[i]``) * joint motion;
  revolute joint motion = rotation by ``q`` about ``axis[i]`` (a unit vector in the joint frame);
* free-flyer q = (x, y, z, qw, qx, qy, qz) (position in the parent frame, unit quaternion), its
  velocity v = (linear, angular), both expressed in the body's own frame;
* body inertias: ``mass``, centre of mass ``com`` (body frame) and rotational inertia about the
  centre of mass ``inertia`` = (xx, yy, zz, xy, xz, yz) in the body frame;
* state arrays are structure-of-arrays with the batch index last: q [nq][B], v [nv][B], ...;
* contact slot k of env e: body ``c_link[k][e]`` (-1 = unused), reference point ``c_point[k][:, e]``
  in that body's frame, sphere radius ``c_radius[k][e]`` (0 for a corner), friction ``c_mu[k][e]``;
  ground plane of env e: points x with n.x = d, ``plane[:, e] = (nx, ny, nz, d)``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
from scipy.spatial.transform import Rotation

REVOLUTE = 0
FREEFLYER = 1


@dataclass
class Model:
    name: str
    parent: np.ndarray    # int32 [nb], -1 = world, parent[i] < i
    jtype: np.ndarray     # int32 [nb]
    axis: np.ndarray      # f64 [nb, 3]
    jrot: np.ndarray      # f64 [nb, 3, 3]
    jpos: np.ndarray      # f64 [nb, 3]
    mass: np.ndarray      # f64 [nb]
    com: np.ndarray       # f64 [nb, 3]
    inertia: np.ndarray   # f64 [nb, 6]

    @property
    def nb(self) -> int:
        return int(self.parent.shape[0])

    @property
    def nq(self) -> int:
        return int(sum(7 if t == FREEFLYER else 1 for t in self.jtype))

    @property
    def nv(self) -> int:
        return int(sum(6 if t == FREEFLYER else 1 for t in self.jtype))

    @property
    def iq(self) -> np.ndarray:
        w = np.array([7 if t == FREEFLYER else 1 for t in self.jtype])
        return np.concatenate([[0], np.cumsum(w)[:-1]]).astype(np.int32)

    @property
    def iv(self) -> np.ndarray:
        w = np.array([6 if t == FREEFLYER else 1 for t in self.jtype])
        return np.concatenate([[0], np.cumsum(w)[:-1]]).astype(np.int32)


@dataclass
class Batch:
    q: np.ndarray          # [nq_max][B]
    v: np.ndarray          # [nv_max][B]
    tau: np.ndarray        # [nv_max][B]
    c_link: np.ndarray     # int32 [ncmax][B]
    c_point: np.ndarray    # [ncmax][3][B]
    c_radius: np.ndarray   # [ncmax][B]
    c_mu: np.ndarray       # [ncmax][B]
    plane: np.ndarray      # [4][B]
    model_id: np.ndarray | None = None   # int32 [B] for batches that mix models
    model_slots: np.ndarray | None = None  # int32 [nmodels]: leading slots each model's envs use

    @property
    def B(self) -> int:
        return int(self.q.shape[1])

    @property
    def ncmax(self) -> int:
        return int(self.c_link.shape[0])

    def env(self, e: int, model: Model) -> dict:
        """Plain per-env view (used by the oracle tests)."""
        return dict(q=self.q[:model.nq, e].copy(), v=self.v[:model.nv, e].copy(),
                    tau=self.tau[:model.nv, e].copy(), c_link=self.c_link[:, e].copy(),
                    c_point=self.c_point[:, :, e].copy(), c_radius=self.c_radius[:, e].copy(),
                    c_mu=self.c_mu[:, e].copy(), plane=self.plane[:, e].copy())

    def take(self, idx) -> "Batch":
        idx = np.asarray(idx, dtype=np.int64)
        return Batch(self.q[:, idx].copy(), self.v[:, idx].copy(), self.tau[:, idx].copy(),
                     self.c_link[:, idx].copy(), self.c_point[:, :, idx].copy(),
                     self.c_radius[:, idx].copy(), self.c_mu[:, idx].copy(), self.plane[:, idx].copy(),
                     None if self.model_id is None else self.model_id[idx].copy(),
                     None if self.model_slots is None else self.model_slots.copy())


@dataclass
class Options:
    dt: float = 1e-3
    gravity: tuple = (0.0, 0.0, -9.81)
    admm_max_iter: int = 2000
    admm_eps: float = 1e-12       # stopping tolerance of the NCP iteration (relative)
    polish_iters: int = 4         # Newton steps on the identified contact modes
    eps_sigma: float = 1e-8       # contact-velocity threshold of the mode test (relative)
    eps_lambda: float = 1e-8      # impulse threshold of the mode test (relative)


@dataclass
class Workload:
    name: str
    models: list
    batch: Batch
    options: Options = field(default_factory=Options)
    precision: str = "fp64"


# --------------------------------------------------------------------------- random helpers

def _rand_rot(rng, n=None):
    qq = rng.normal(size=(4,) if n is None else (n, 4))
    return Rotation.from_quat(qq).as_matrix()


def _rand_inertia(rng, mass_lo=0.5, mass_hi=3.0):
    m = rng.uniform(mass_lo, mass_hi)
    d = rng.uniform(0.01, 0.1, size=3)
    R = _rand_rot(rng)
    I = R @ np.diag(d) @ R.T
    return m, np.array([I[0, 0], I[1, 1], I[2, 2], I[0, 1], I[0, 2], I[1, 2]])


def _unit(v):
    return v / np.linalg.norm(v)


def _build(name, parent, jtype, axis, jpos, masses, coms, inertias, jrot=None):
    nb = len(parent)
    if jrot is None:
        jrot = np.tile(np.eye(3), (nb, 1, 1))
    return Model(name, np.asarray(parent, np.int32), np.asarray(jtype, np.int32),
                 np.asarray(axis, float), np.asarray(jrot, float), np.asarray(jpos, float),
                 np.asarray(masses, float), np.asarray(coms, float), np.asarray(inertias, float))


# --------------------------------------------------------------------------- models

def arm7(rng):
    """7-dof fixed-base chain: random unit axes, link lengths U(0.1,0.4), masses U(0.5,3),
    inertias diag(U(0.01,0.1)^3) under a random rotation.  Returns (model, tip) with ``tip`` the
    end point of link 7 in its own frame."""
    L = rng.uniform(0.1, 0.4, size=7)
    axis = np.array([_unit(rng.normal(size=3)) for _ in range(7)])
    jpos = np.zeros((7, 3))
    for i in range(1, 7):
        jpos[i] = (0.0, 0.0, L[i - 1])
    masses, coms, inertias = [], [], []
    for i in range(7):
        m, I = _rand_inertia(rng)
        masses.append(m)
        coms.append((0.0, 0.0, L[i] / 2))
        inertias.append(I)
    model = _build("arm7", list(range(-1, 6)), [REVOLUTE] * 7, axis, jpos, masses, coms, inertias)
    return model, np.array([0.0, 0.0, L[6]])


def _scale_mass(model, total):
    s = total / model.mass.sum()
    model.mass *= s
    model.inertia *= s


def humanoid36(rng):
    """Free-flyer base + 30 revolute joints in 5 chains (2 legs x 6, 2 arms x 7, torso/head x 4),
    total mass 70 kg.  Returns (model, feet) with ``feet`` = [(body, corners[4][3]), ...] for the
    two 0.2 x 0.1 x 0.05 m foot boxes and ``hands`` boxes of 4 corners each."""
    ex, ey, ez = np.eye(3)
    parent, jtype, axis, jpos = [-1], [FREEFLYER], [np.zeros(3)], [np.zeros(3)]
    masses, coms, inertias = [], [], []
    m, I = _rand_inertia(rng)
    masses.append(m); coms.append(np.zeros(3)); inertias.append(I)

    def chain(attach, axes, first_dir, dirs):
        idx = []
        prev = 0
        off = np.asarray(attach, float)
        for k, a in enumerate(axes):
            L = rng.uniform(0.1, 0.4)
            parent.append(prev); jtype.append(REVOLUTE); axis.append(a); jpos.append(off)
            d = first_dir if k == 0 else dirs
            m, I = _rand_inertia(rng)
            masses.append(m); coms.append(d * L / 2); inertias.append(I)
            prev = len(parent) - 1
            idx.append(prev)
            off = d * L
        return idx, off   # off = tip of the last link in its own frame

    legs, arms = [], []
    for s in (+1, -1):
        idx, tip = chain((0.0, s * 0.1, -0.1), [ez, ex, ey, ey, ey, ex], -ez, -ez)
        legs.append((idx, tip))
    for s in (+1, -1):
        idx, tip = chain((0.0, s * 0.2, 0.4), [ey, ex, ez, ey, ez, ey, ex], s * ey, -ez)
        arms.append((idx, tip))
    chain((0.0, 0.0, 0.1), [ez, ey, ex, ey], ez, ez)
    model = _build("humanoid36", parent, jtype, axis, jpos, masses, coms, inertias)
    _scale_mass(model, 70.0)
    feet = []
    for idx, tip in legs:
        body = idx[-1]
        corners = [tip + np.array([sx * 0.1, sy * 0.05, -0.05]) for sx in (1, -1) for sy in (1, -1)]
        feet.append((body, np.array(corners)))
    hands = []
    for idx, tip in arms:
        body = idx[-1]
        corners = [tip + np.array([sx * 0.04, sy * 0.04, -0.03]) for sx in (1, -1) for sy in (1, -1)]
        hands.append((body, np.array(corners)))
    return model, feet, hands


def quadruped18(rng):
    """Free-flyer base + 4 legs x (hip abduction about x, hip flexion about y, knee about y), thigh
    and shank lengths U(0.2,0.35), total mass 12 kg, point feet at the shank tips.  Returns
    (model, feet) with ``feet`` = [(body, point[3]), ...]."""
    ex, ey, ez = np.eye(3)
    parent, jtype, axis, jpos = [-1], [FREEFLYER], [np.zeros(3)], [np.zeros(3)]
    masses, coms, inertias = [], [], []
    m, I = _rand_inertia(rng)
    masses.append(m); coms.append(np.zeros(3)); inertias.append(I)
    feet = []
    for sx in (+1, -1):
        for sy in (+1, -1):
            lt, ls = rng.uniform(0.2, 0.35), rng.uniform(0.2, 0.35)
            b0 = len(parent)
            parent.append(0); jtype.append(REVOLUTE); axis.append(ex); jpos.append((sx * 0.19, sy * 0.05, 0.0))
            m, I = _rand_inertia(rng); masses.append(m); coms.append((0.0, sy * 0.04, 0.0)); inertias.append(I)
            parent.append(b0); jtype.append(REVOLUTE); axis.append(ey); jpos.append((0.0, sy * 0.08, 0.0))
            m, I = _rand_inertia(rng); masses.append(m); coms.append((0.0, 0.0, -lt / 2)); inertias.append(I)
            parent.append(b0 + 1); jtype.append(REVOLUTE); axis.append(ey); jpos.append((0.0, 0.0, -lt))
            m, I = _rand_inertia(rng); masses.append(m); coms.append((0.0, 0.0, -ls / 2)); inertias.append(I)
            feet.append((b0 + 2, np.array([0.0, 0.0, -ls])))
    model = _build("quadruped18", parent, jtype, axis, jpos, masses, coms, inertias)
    _scale_mass(model, 12.0)
    return model, feet


# --------------------------------------------------------------------------- scene placement
# Body placements for set-up only (plane height, initial velocities).  Uses scipy's Rotation.

def _placements(model: Model, q: np.ndarray):
    """q: [nq][B] -> list of (R [B,3,3], p [B,3]) per body."""
    B = q.shape[1]
    iq = model.iq
    out = []
    for i in range(model.nb):
        if model.parent[i] < 0:
            Rp, pp = np.tile(np.eye(3), (B, 1, 1)), np.zeros((B, 3))
        else:
            Rp, pp = out[model.parent[i]]
        R0 = Rp @ model.jrot[i]
        p0 = pp + np.einsum("bij,j->bi", Rp, model.jpos[i])
        if model.jtype[i] == REVOLUTE:
            Rj = Rotation.from_rotvec(model.axis[i][None, :] * q[iq[i]][:, None]).as_matrix()
            out.append((R0 @ Rj, p0))
        else:
            pos = q[iq[i]:iq[i] + 3].T
            quat = q[iq[i] + 3:iq[i] + 7].T                       # (w, x, y, z)
            Rj = Rotation.from_quat(quat[:, [1, 2, 3, 0]]).as_matrix()
            out.append((R0 @ Rj, p0 + np.einsum("bij,bj->bi", R0, pos)))
    return out


def _point_world(model, q, body, point_local):
    R, p = _placements(model, q)[body]
    return p + np.einsum("bij,bj->bi", R, np.broadcast_to(point_local, p.shape))


def _twist_fd(model, q, body, point_world, h=1e-6):
    """Central-difference [6 x nv] map from joint velocities to (velocity of the body point
    currently at ``point_world``, angular velocity), both in world axes.  Revolute-only models."""
    B = q.shape[1]
    J = np.zeros((B, 6, model.nv))
    for j in range(model.nv):
        qp, qm = q.copy(), q.copy()
        qp[j] += h
        qm[j] -= h
        Rp_, pp_ = _placements(model, qp)[body]
        Rm_, pm_ = _placements(model, qm)[body]
        R, p = _placements(model, q)[body]
        w = Rotation.from_matrix(Rp_ @ np.transpose(Rm_, (0, 2, 1))).as_rotvec() / (2 * h)
        vo = (pp_ - pm_) / (2 * h)
        J[:, :3, j] = vo + np.cross(w, point_world - p)
        J[:, 3:, j] = w
    return J


# --------------------------------------------------------------------------- workloads

def _empty_contacts(ncmax, B):
    return (np.full((ncmax, B), -1, np.int32), np.zeros((ncmax, 3, B)), np.zeros((ncmax, B)),
            np.zeros((ncmax, B)), np.zeros((4, B)))


def arm_sphere(B=16, seed=1000):
    """7-dof arm, end-effector sphere r=0.05 over a horizontal plane (0-1 contacts), mu=0.5.
    q ~ U(-pi,pi), v ~ N(0,1), tau ~ N(0,5); the plane sits at the sphere's lowest point
    + U(-2e-3, 2e-3), so about half of the envs touch."""
    rng = np.random.default_rng(seed)
    model, tip = arm7(rng)
    q = rng.uniform(-np.pi, np.pi, size=(7, B))
    v = rng.normal(0.0, 1.0, size=(7, B))
    tau = rng.normal(0.0, 5.0, size=(7, B))
    r = 0.05
    centre = _point_world(model, q, 6, tip)
    delta = rng.uniform(-2e-3, 2e-3, size=B)
    c_link, c_point, c_radius, c_mu, plane = _empty_contacts(1, B)
    c_link[0] = 6
    c_point[0] = tip[:, None]
    c_radius[0] = r
    c_mu[0] = 0.5
    plane[2] = 1.0
    plane[3] = centre[:, 2] - r + delta
    return Workload("arm7-sphere", [model], Batch(q, v, tau, c_link, c_point, c_radius, c_mu, plane))


def arm_cube(B=65536, seed=1001, slots=4):
    """7-dof arm with a 0.05 m cube rigidly mounted at the tip, bottom face parallel to a horizontal
    plane, 4 bottom corners penetrating by U(0,1e-3) (``slots=8`` also lists the 4 top corners,
    which stay clear of the plane).  mu ~ U(0.2,1.0).  The initial joint velocity gives the
    cube's bottom centre a normal approach speed U(0.1,0.5) m/s and a tangential speed of
    U(0, 0.2 mu v_N) for even envs (meant to stick) and U(0.5,2) m/s for odd envs (meant to slide)."""
    rng = np.random.default_rng(seed)
    model, tip = arm7(rng)
    q = rng.uniform(-np.pi, np.pi, size=(7, B))
    tau = rng.normal(0.0, 5.0, size=(7, B))
    mu = rng.uniform(0.2, 1.0, size=B)
    h = 0.025
    R7, p7 = _placements(model, q)[6]
    tipw = p7 + np.einsum("bij,j->bi", R7, tip)
    yaw = rng.uniform(0, 2 * np.pi, size=B)
    Rz = Rotation.from_rotvec(np.outer(yaw, [0, 0, 1.0])).as_matrix()
    loc = [(sx * h, sy * h, -2 * h) for sx in (1, -1) for sy in (1, -1)]
    if slots == 8:
        loc += [(sx * h, sy * h, 0.0) for sx in (1, -1) for sy in (1, -1)]
    c_link, c_point, c_radius, c_mu, plane = _empty_contacts(slots, B)
    for k, lk in enumerate(loc):
        cw = tipw + np.einsum("bij,j->bi", Rz, np.array(lk))
        c_link[k] = 6
        c_point[k] = np.einsum("bji,bj->bi", R7, cw - p7).T
        c_mu[k] = mu
    pen = rng.uniform(0.0, 1e-3, size=B)
    plane[2] = 1.0
    plane[3] = tipw[:, 2] - 2 * h + pen
    # initial velocity: damped least squares on a finite-difference twist map of link 7
    bottom = tipw + np.array([0.0, 0.0, -2 * h])
    J = _twist_fd(model, q, 6, bottom)
    vN = rng.uniform(0.1, 0.5, size=B)
    stick = (np.arange(B) % 2) == 0
    speed = np.where(stick, rng.uniform(0.0, 1.0, size=B) * 0.2 * mu * vN, rng.uniform(0.5, 2.0, size=B))
    ang = rng.uniform(0, 2 * np.pi, size=B)
    want = np.zeros((B, 6))
    want[:, 0] = speed * np.cos(ang)
    want[:, 1] = speed * np.sin(ang)
    want[:, 2] = -vN
    want[:, 5] = rng.normal(0.0, 0.3, size=B)
    JJt = J @ np.transpose(J, (0, 2, 1)) + 1e-4 * np.eye(6)
    v = np.einsum("bji,bj->bi", J, np.linalg.solve(JJt, want[:, :, None])[:, :, 0]).T
    return Workload("arm7-cube", [model], Batch(q, v, tau, c_link, c_point, c_radius, c_mu, plane))


def _quat_small(rng, B, s):
    rv = rng.normal(0.0, s, size=(B, 3))
    xyzw = Rotation.from_rotvec(rv).as_quat()
    return xyzw[:, [3, 0, 1, 2]].T


def humanoid_feet(B=16384, seed=1002, model_seed=None, hands=False):
    """36-dof humanoid near standing: base orientation identity + N(0,0.05) rotation vector, legs
    and torso N(0,0.05), arms N(0,0.3), v ~ N(0,0.1), joint torques N(0,5) (base 0).  Plane at the
    lowest foot corner + U(-2e-3, 5e-3): 0-8 active corner contacts, mu=0.8.  ``hands`` adds two
    hand boxes (8 more slots, normally clear of the plane)."""
    rng = np.random.default_rng(seed if model_seed is None else model_seed)
    model, feet, hand_boxes = humanoid36(rng)
    if model_seed is not None:
        rng = np.random.default_rng(seed)
    q = np.zeros((model.nq, B))
    q[0:2] = rng.normal(0.0, 0.05, size=(2, B))
    q[2] = 1.0
    q[3:7] = _quat_small(rng, B, 0.05)
    iq = model.iq
    for i in range(1, model.nb):
        # legs are bodies 1..12, arms 13..26, torso 27..30
        s = 0.3 if 13 <= i <= 26 else 0.05
        q[iq[i]] = rng.normal(0.0, s, size=B)
    v = rng.normal(0.0, 0.1, size=(model.nv, B))
    tau = rng.normal(0.0, 5.0, size=(model.nv, B))
    tau[:6] = 0.0
    boxes = feet + (hand_boxes if hands else [])
    ncmax = 4 * len(boxes)
    c_link, c_point, c_radius, c_mu, plane = _empty_contacts(ncmax, B)
    zs = []
    k = 0
    for body, corners in boxes:
        for c in corners:
            c_link[k] = body
            c_point[k] = c[:, None]
            c_mu[k] = 0.8
            if k < 8:
                zs.append(_point_world(model, q, body, c)[:, 2])
            k += 1
    plane[2] = 1.0
    plane[3] = np.min(np.array(zs), axis=0) + rng.uniform(-2e-3, 5e-3, size=B)
    return Workload("humanoid36-feet", [model], Batch(q, v, tau, c_link, c_point, c_radius, c_mu, plane),
                    precision="mixed")


def quadruped_feet(B=4096, seed=1004, model_seed=None):
    """18-dof quadruped standing on its 4 point feet (bent knees), base orientation identity +
    N(0,0.05), joints N(0,0.05) around the stance, v ~ N(0,0.1), joint torques N(0,2), plane at the
    highest foot + U(0, 2e-3) so that all 4 feet touch, mu=0.8."""
    rng = np.random.default_rng(seed if model_seed is None else model_seed)
    model, feet = quadruped18(rng)
    if model_seed is not None:
        rng = np.random.default_rng(seed)
    q = np.zeros((model.nq, B))
    q[0:2] = rng.normal(0.0, 0.05, size=(2, B))
    q[2] = 0.5
    q[3:7] = _quat_small(rng, B, 0.05)
    iq = model.iq
    stance = [0.0, 0.7, -1.4]
    for leg in range(4):
        for k in range(3):
            q[iq[1 + 3 * leg + k]] = stance[k] + rng.normal(0.0, 0.05, size=B)
    v = rng.normal(0.0, 0.1, size=(model.nv, B))
    tau = rng.normal(0.0, 2.0, size=(model.nv, B))
    tau[:6] = 0.0
    c_link, c_point, c_radius, c_mu, plane = _empty_contacts(4, B)
    zs = []
    for k, (body, p) in enumerate(feet):
        c_link[k] = body
        c_point[k] = p[:, None]
        c_mu[k] = 0.8
        zs.append(_point_world(model, q, body, p)[:, 2])
    plane[2] = 1.0
    plane[3] = np.max(np.array(zs), axis=0) + rng.uniform(0.0, 2e-3, size=B)
    return Workload("quadruped18-feet", [model], Batch(q, v, tau, c_link, c_point, c_radius, c_mu, plane),
                    precision="mixed")


def uneven(B=32768, seed=1003):
    """Mixed batch: envs e = 0,1,2 (mod 3) hold a 7-dof arm with a cube (8 corner slots), an
    18-dof quadruped (4 feet) and a 36-dof humanoid (8 foot + 8 hand corners); 16 slots per env."""
    n = [(B - r + 2) // 3 for r in range(3)]
    parts = [arm_cube(n[0], seed, slots=8), quadruped_feet(n[1], seed + 10, model_seed=1004),
             humanoid_feet(n[2], seed + 20, model_seed=1002, hands=True)]
    models = [p.models[0] for p in parts]
    nqm = max(m.nq for m in models)
    nvm = max(m.nv for m in models)
    ncmax = 16
    q = np.zeros((nqm, B)); v = np.zeros((nvm, B)); tau = np.zeros((nvm, B))
    c_link, c_point, c_radius, c_mu, plane = _empty_contacts(ncmax, B)
    mid = (np.arange(B) % 3).astype(np.int32)
    for k, p in enumerate(parts):
        sel = np.nonzero(mid == k)[0]
        b = p.batch
        q[:b.q.shape[0], sel] = b.q
        v[:b.v.shape[0], sel] = b.v
        tau[:b.tau.shape[0], sel] = b.tau
        nc = b.ncmax
        c_link[:nc, sel] = b.c_link
        c_point[:nc, :, sel] = b.c_point
        c_radius[:nc, sel] = b.c_radius
        c_mu[:nc, sel] = b.c_mu
        plane[:, sel] = b.plane
    return Workload("uneven-arm-quadruped-humanoid", models,
                    Batch(q, v, tau, c_link, c_point, c_radius, c_mu, plane, mid,
                          np.array([p.batch.ncmax for p in parts], np.int32)), precision="mixed")


WORKLOADS = {
    "arm7-sphere": arm_sphere,
    "arm7-cube": arm_cube,
    "humanoid36-feet": humanoid_feet,
    "uneven": uneven,
    "quadruped18-feet": quadruped_feet,
}
