"""Pins of the oracle's position-update adjoint (q+ = q (+) dt v+, the configuration half of the
symplectic-Euler step of Sec. 2.3), used to chain steps in a rollout (no GPU).

* closed forms: a revolute joint's update is q + dq (Jacobians = I); the free-flyer's is the
  R^3 x SO(3) update p+ = p + R dq_lin, R+ = R Exp(dq_ang), whose tangent Jacobians are the textbook
  Lie-group ones: d eta_lin = E^T (eps_lin - [dq_lin]x eps_ang + d_lin), d eta_ang = E^T eps_ang +
  Jr(dq_ang) d_ang with E = Exp(dq_ang) and Jr the right Jacobian of SO(3);
* central finite differences with the exact (arc-cosine) rotation logarithm of scipy;
* the one-step adjoint with both cotangents against central differences of the whole step."""
import numpy as np
from scipy.spatial.transform import Rotation

from oracle import rigid
from oracle import step as S
from paper_2409_07107_gb300 import scenes
from tests.helpers import point_mass_model, random_state


def _skew(a):
    return np.array([[0.0, -a[2], a[1]], [a[2], 0.0, -a[0]], [-a[1], a[0], 0.0]])


def _exp_so3(phi):
    return Rotation.from_rotvec(phi).as_matrix()


def _jr(phi):
    t = np.linalg.norm(phi)
    K = _skew(phi)
    return np.eye(3) - (1 - np.cos(t)) / t ** 2 * K + (t - np.sin(t)) / t ** 3 * (K @ K)


def _log_diff(model, q0, q1):
    """Exact tangent difference (scipy's rotation-vector logarithm), for finite differences."""
    out = np.zeros(model.nv)
    for i, jt in enumerate(model.jtype):
        k, j = model.iq[i], model.iv[i]
        if jt == scenes.REVOLUTE:
            out[j] = q1[k] - q0[k]
        else:
            R0 = Rotation.from_quat(np.r_[q0[k + 4:k + 7], q0[k + 3]]).as_matrix()
            R1 = Rotation.from_quat(np.r_[q1[k + 4:k + 7], q1[k + 3]]).as_matrix()
            out[j:j + 3] = R0.T @ (q1[k:k + 3] - q0[k:k + 3])
            out[j + 3:j + 6] = Rotation.from_matrix(R0.T @ R1).as_rotvec()
    return out


def test_revolute_identity():
    rng = np.random.default_rng(3)
    m = scenes.arm7(rng)[0]
    q, v, _ = random_state(m, rng)
    Jq, Jd = S.integrate_jacobians(m, q, 1e-3 * v)
    assert np.abs(Jq - np.eye(m.nv)).max() == 0.0
    assert np.abs(Jd - np.eye(m.nv)).max() == 0.0


def test_free_flyer_closed_form():
    rng = np.random.default_rng(4)
    m = point_mass_model()
    for scale in (1e-3, 0.3, 1.7):
        q, v, _ = random_state(m, rng)
        dq = scale * v
        Jq, Jd = S.integrate_jacobians(m, q, dq)
        E = _exp_so3(dq[3:])
        Jq_ref = np.zeros((6, 6))
        Jq_ref[:3, :3] = E.T
        Jq_ref[:3, 3:] = -E.T @ _skew(dq[:3])
        Jq_ref[3:, 3:] = E.T
        Jd_ref = np.zeros((6, 6))
        Jd_ref[:3, :3] = E.T
        Jd_ref[3:, 3:] = _jr(dq[3:])
        assert np.abs(Jq - Jq_ref).max() <= 1e-13
        assert np.abs(Jd - Jd_ref).max() <= 1e-13


def test_quadruped_central_differences():
    rng = np.random.default_rng(5)
    m = scenes.quadruped18(rng)[0]
    q, v, _ = random_state(m, rng)
    dq = 0.05 * v
    Jq, Jd = S.integrate_jacobians(m, q, dq)
    qp = rigid.integrate(m, q, dq)
    h = 1e-6
    for j in range(m.nv):
        e = np.zeros(m.nv)
        e[j] = h
        cq = (_log_diff(m, qp, rigid.integrate(m, rigid.integrate(m, q, e), dq))
              - _log_diff(m, qp, rigid.integrate(m, rigid.integrate(m, q, -e), dq))) / (2 * h)
        cd = (_log_diff(m, qp, rigid.integrate(m, q, dq + e)) - _log_diff(m, qp, rigid.integrate(m, q, dq - e))) / (2 * h)
        assert np.abs(cq - Jq[:, j]).max() <= 1e-8
        assert np.abs(cd - Jd[:, j]).max() <= 1e-8


def test_step_adjoint_with_position_cotangent():
    """<q_bar, u_q> + <v_bar, u_v> + <tau_bar, u_tau> equals the directional derivative of
    <q_bar+, eta(q+)> + <v_bar+, v+> along u, by central differences of the whole step."""
    wl = scenes.quadruped_feet(8)
    m = wl.models[0]
    rng = np.random.default_rng(6)
    done = 0
    for e in range(8):
        env = wl.batch.env(e, m)
        st = S.step_jac(m, env, wl.options)
        if st["margin"] < 1e-3:
            continue
        vb, qb = rng.normal(size=m.nv), rng.normal(size=m.nv)
        gq, gv, gt = S.vjp(m, env, wl.options, vb, st=st, q_bar_next=qb)
        u = rng.normal(size=(3, m.nv))
        h = 1e-6
        f = []
        for s in (1, -1):
            en = dict(env)
            en["q"] = rigid.integrate(m, env["q"], s * h * u[0])
            en["v"] = env["v"] + s * h * u[1]
            en["tau"] = env["tau"] + s * h * u[2]
            r = S.step(m, en, wl.options)
            f.append(qb @ _log_diff(m, st["q_next"], r["q_next"]) + vb @ r["v_next"])
        fd = (f[0] - f[1]) / (2 * h)
        an = gq @ u[0] + gv @ u[1] + gt @ u[2]
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))
        done += 1
    assert done >= 3


def test_raw_tangent_maps():
    """d eta / d q_raw and d q_raw / d eta: closed form [R, 0; 0, Q(quat)[:, 1:] / 2] for the
    free-flyer, left-inverse of each other, no response to the quaternion's own direction."""
    rng = np.random.default_rng(8)
    m = scenes.quadruped18(rng)[0]
    q, _, _ = random_state(m, rng)
    Jt = rigid.tangent_to_raw_jacobian(m, q)
    Jr = rigid.raw_to_tangent_jacobian(m, q)
    assert np.abs(Jr @ Jt - np.eye(m.nv)).max() <= 1e-14
    w, x, y, z = q[3:7]
    R = Rotation.from_quat([x, y, z, w]).as_matrix()
    Qc = np.array([[-x, -y, -z], [w, -z, y], [z, w, -x], [-y, x, w]])
    assert np.abs(Jt[:3, :3] - R).max() <= 1e-14
    assert np.abs(Jt[3:7, 3:6] - 0.5 * Qc).max() <= 1e-14
    assert np.abs(Jr[3:6, 3:7] @ q[3:7]).max() <= 1e-14
    assert np.abs(Jt[7:, 6:] - np.eye(m.nv - 6)).max() == 0.0


def test_rollout_gradient_central_differences():
    """The reverse-mode rollout gradient against central differences of the loss through the
    oracle's own rollout, along random torque directions (3 steps, quadruped on the ground)."""
    wl = scenes.quadruped_feet(16)
    m = wl.models[0]
    rng = np.random.default_rng(9)
    T = 3
    checked = 0
    for e in range(16):
        if checked >= 3:
            break
        env = wl.batch.env(e, m)
        taus = rng.normal(size=(T, m.nv)) * 2.0
        taus[:, :6] = 0.0
        goal = rigid.integrate(m, env["q"], 0.01 * rng.normal(size=m.nv))

        def loss(ts):
            qT = S.rollout(m, env, ts, wl.options)[-1][0]
            return float(np.sum((qT - goal) ** 2))

        qT = S.rollout(m, env, taus, wl.options)[-1][0]
        g, _, margin = S.rollout_grad(m, env, taus, wl.options, 2.0 * (qT - goal))
        if margin < 1e-3:
            continue
        for _ in range(3):
            u = rng.normal(size=taus.shape)
            u[:, :6] = 0.0
            h = 1e-5
            fd = (loss(taus + h * u) - loss(taus - h * u)) / (2 * h)
            an = float(np.sum(g * u))
            assert abs(fd - an) <= 1e-6 * max(abs(an), 1e-8) + 1e-12, (e, fd, an)
        checked += 1
    assert checked >= 2
