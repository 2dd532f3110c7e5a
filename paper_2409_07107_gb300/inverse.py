"""Gauss-Newton inverse problems through the differentiable step (Sec. 4) over a batch of envs:
inverse dynamics through contacts (Eq. exp_id) and the estimation of an initial velocity from the
configuration a rollout reaches (Eq. init_id, `gauss_newton_initial_velocity`).

Inverse dynamics: min over tau_act of 1/2 ||v+(q, v, S^T tau_act) - v*||^2 for every env at once.  Each iteration
evaluates the step and dv+/dtau (sim_step_jac through `simulator_step_jac`), then takes the
Gauss-Newton step: the minimum-norm least-squares solution of J d = r with J = dv+/dtau S^T per
env.  J is rank deficient whenever contacts stick (four sticking feet of an 18-dof quadruped
leave rank 6 of 12), so the step is taken with a pseudo-inverse (SVD), not a full-rank solver.
Its cut-off follows the accuracy of the Jacobian: singular values below rtol x the largest are
treated as zero, with rtol = 1e-10 for the FP64 step and 1e-5 for the mixed-precision step (its
Jacobian entries carry FP32 rounding, about 1e-6 relative, which in the null directions of J would
otherwise be inverted into huge steps; the true small singular values of these problems are about
1e-2 of the largest).  This module only marshals tensors; the step and its derivatives are the
library's kernels.
"""
import torch


RTOL = {"fp64": 1e-10, "mixed": 1e-5}


def simulator_step_jac(sim):
    """A step function for gauss_newton_inverse_dynamics: tau [nv][B] -> (v+ [nv][B], dv+/dtau
    [nv][nv][B]) through sim_step_jac on the Simulator's batch (its tau is overwritten).  Its
    ``rtol`` attribute is the pseudo-inverse cut-off for the Simulator's precision."""
    def fn(tau):
        sim.batch["tau"].copy_(tau)
        out = sim.step_jac()
        return out["v_next"], out["dv_dtau"]
    fn.rtol = RTOL["fp64" if int(sim.opt.precision) == 0 else "mixed"]
    return fn


def gauss_newton_inverse_dynamics(step_jac, Sa, v_target, tau_act0, iters=20, tol=1e-12, rtol=None):
    """step_jac: tau [nv][B] -> (v+ [nv][B], dv+/dtau [nv][nv][B], element [k][d][e] = dv_k/dtau_d);
    Sa: actuation matrix [n_act][nv]; v_target [nv][B]; tau_act0 [n_act][B]; rtol: the
    pseudo-inverse cut-off (default: step_jac.rtol if it has one, else 1e-10).  Returns (tau_act,
    the largest per-env residual norm before each step)."""
    if rtol is None:
        rtol = getattr(step_jac, "rtol", 1e-10)
    ta = tau_act0.clone()
    hist = []
    for _ in range(iters):
        v_next, dv_dtau = step_jac(Sa.t() @ ta)
        r = v_next - v_target                                       # [nv][B]
        hist.append(float(torch.linalg.vector_norm(r, dim=0).max()))
        if hist[-1] <= tol:
            break
        J = torch.einsum("kdb,ad->bka", dv_dtau, Sa)                # [B][nv][n_act]
        step = torch.linalg.pinv(J, rtol=rtol) @ r.t().unsqueeze(-1)  # [B][n_act][1]
        ta = ta - step.squeeze(-1).t()
    return ta, hist


def gauss_newton_initial_velocity(sc, q0, v_init, q_target, taus, free, iters=20, tol=1e-12, rtol=None):
    """Gauss-Newton estimate of the initial velocity (Sec. 4, Eq. init_id): the v_0 whose rollout of
    len(taus) steps from (q0, v_0) ends at the configuration q_target, for every env of the batch
    at once.  sc is a rollout.StepContext; q0, q_target [nq][B]; v_init [nv][B]; free: the indices
    of the components of v_0 that are estimated (a body sliding on the floor: x, y and the yaw
    rate; the contacts pin the others).  The residual is the raw configuration difference
    q_T - q_target (zero exactly where the tangent difference is); its Jacobian with respect to
    v_0[free] is assembled row by row from reverse-mode passes through the rollout (sim_step
    forward, the tape's VJP backward), and the step is its minimum-norm least-squares solution
    (pseudo-inverse, cut-off rtol: by default the step context's precision, as for
    gauss_newton_inverse_dynamics).  Returns (v_0, the largest per-env residual norm before each
    step)."""
    from . import rollout as R
    if rtol is None:
        rtol = RTOL["fp64" if int(sc.opt.precision) == 0 else "mixed"]
    free = torch.as_tensor(free, dtype=torch.long, device=v_init.device)
    v = v_init.clone()
    hist = []
    for _ in range(iters):
        v0 = v.clone().requires_grad_(True)
        qT, _ = R.rollout(sc, q0, v0, taus, 0)
        r = (qT - q_target).detach()                                 # [nq][B]
        hist.append(float(torch.linalg.vector_norm(r, dim=0).max()))
        if hist[-1] <= tol:
            break
        rows = [torch.autograd.grad(qT[k].sum(), v0, retain_graph=k + 1 < qT.shape[0])[0][free]
                for k in range(qT.shape[0])]                          # d q_T[k] / d v_0[free], [nf][B]
        J = torch.stack(rows, 0).permute(2, 0, 1)                     # [B][nq][nf]
        step = torch.linalg.pinv(J, rtol=rtol) @ r.t().unsqueeze(-1)  # [B][nf][1]
        v[free] = v[free] - step.squeeze(-1).t()
    return v, hist
