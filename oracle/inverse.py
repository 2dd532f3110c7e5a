"""Gauss-Newton inverse problems through the differentiable step (oracle).  Test infrastructure only.

Sec. 4 uses the step's forward-mode Jacobians in a Gauss-Newton loop on two problems:

* estimating an initial condition (Eq. init_id): the initial velocity v_0 of a cube thrown onto
  the floor in a sliding mode, from the configuration q_T* it reaches after T steps,
  min 1/2 ||q_T(v_0) - q_T*||^2, read with the difference taken in the tangent space of q_T
  (q_T* (-) q_T, the local difference of the free-flyer; the raw quaternion is not a vector);
  dq_T/dv_0 follows by the chain rule through the steps: with the step Jacobians dv+/dq, dv+/dv
  (route 1 of step.py) and the position-update Jacobians q+ = q (+) dt v+ (integrate_jacobians),
  dv_{t+1} = dv+/dq dq_t + dv+/dv dv_t and dq_{t+1} = Jq dq_t + dt Jd dv_{t+1};
* inverse dynamics through contacts (Eq. exp_id): the actuator torques tau_act with
  v+(q, v, S^T tau_act) = v*, Jacobian dv+/dtau S^T.

Each Gauss-Newton step is the minimum-norm least-squares step of the linearised residual (the
Jacobians are rank deficient where contacts pin directions of motion).
"""
import numpy as np

from . import rigid
from . import step as S


def rollout_q_jacobian(model, env0, T, opt):
    """q_T after T steps from env0 (fixed tau) and dq_T / dv_0 in tangent coordinates (nv x nv)."""
    env = dict(env0)
    nv = len(env["v"])
    dq = np.zeros((nv, nv))
    dv = np.eye(nv)
    for _ in range(T):
        st = S.step_jac(model, env, opt)
        dvn = st["dv_dq"] @ dq + st["dv_dv"] @ dv
        Jq, Jd = S.integrate_jacobians(model, env["q"], opt.dt * st["v_next"])
        dq = Jq @ dq + opt.dt * (Jd @ dvn)
        dv = dvn
        env = dict(env, q=st["q_next"], v=st["v_next"])
    return env["q"], dq


def rollout_q(model, env0, T, opt):
    env = dict(env0)
    for _ in range(T):
        st = S.step(model, env, opt)
        env = dict(env, q=st["q_next"], v=st["v_next"])
    return env["q"]


def estimate_initial_velocity(model, env0, q_target, T, opt, v_init, iters=20, tol=1e-12, free=None):
    """Gauss-Newton on 1/2 ||q_target (-) q_T(v_0)||^2 from v_init, over the components `free` of
    v_0 (all by default; for a body sliding on the floor the planar ones, the others being pinned
    by the contacts).  Returns (v_0, residual norms)."""
    v0 = np.array(v_init, dtype=float)
    free = np.arange(len(v0)) if free is None else np.asarray(free)
    hist = []
    for _ in range(iters):
        qT, J = rollout_q_jacobian(model, dict(env0, v=v0), T, opt)
        r = rigid.local_difference(model, q_target, qT)
        hist.append(float(np.linalg.norm(r)))
        if hist[-1] <= tol:
            break
        v0[free] = v0[free] - np.linalg.lstsq(J[:, free], r, rcond=1e-12)[0]
    return v0, hist


def inverse_dynamics(model, env, opt, Sa, v_target, tau_act0, iters=20, tol=1e-12):
    """Gauss-Newton on 1/2 ||v+(q, v, S^T tau_act) - v_target||^2 from tau_act0 (Sa: actuation
    matrix, n_act x nv).  Returns (tau_act, residual norms)."""
    ta = np.array(tau_act0, dtype=float)
    hist = []
    for _ in range(iters):
        st = S.step_jac(model, dict(env, tau=Sa.T @ ta), opt)
        r = st["v_next"] - v_target
        hist.append(float(np.linalg.norm(r)))
        if hist[-1] <= tol:
            break
        ta = ta - np.linalg.lstsq(st["dv_dtau"] @ Sa.T, r, rcond=1e-12)[0]
    return ta, hist
