"""Gauss-Newton inverse dynamics through contacts (Sec. 4, Eq. exp_id) over a batch of envs.

min over tau_act of 1/2 ||v+(q, v, S^T tau_act) - v*||^2 for every env at once.  Each iteration
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
