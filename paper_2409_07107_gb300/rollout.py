"""Differentiable rollouts: the C-ABI step as a torch.autograd.Function, chained over time.

Every step runs in the library (sim_step forward; sim_step_vjp backward, which chains the adjoint of
the position update q+ = q (+) dt v+ when given a cotangent of q+; the cotangent maps between raw q
and its tangent coordinates are library kernels too).  This module only marshals tensors:

* ``StepContext`` holds what does not change along a rollout: device models, contact descriptors,
  options and the pipeline workspace;
* ``SimStep.apply(q, v, tau, ctx)`` -> (q+, v+), differentiable w.r.t. q (raw coordinates, the
  free-flyer quaternion included), v and tau; its forward keeps the step's tape (impulses, modes,
  status) and its backward differentiates that solution (sim_step_vjp_tape: no second NCP solve);
* ``rollout(ctx, q0, v0, taus, checkpoint_every)`` runs len(taus) steps; with checkpoint_every = k
  the reverse pass recomputes each k-step segment from its first state instead of keeping every
  step's inputs (torch.utils.checkpoint), trading one extra forward step per step for memory.
"""
import torch
import torch.utils.checkpoint

from . import (DeviceModel, autotune, batch_to_device, cotangent_to_raw, cotangent_to_tangent, describe_schedule,
               make_options, sim_step, sim_step_vjp, sim_step_vjp_tape, workspace_size)


class StepContext:
    """The fixed part of a rollout's batch (models, contacts, options, workspace)."""

    def __init__(self, workload, precision=None, device="cuda", **opt):
        self.models = [DeviceModel(m) for m in workload.models]
        self.base = batch_to_device(workload.batch, device)
        self.opt = make_options(precision or workload.precision, dt=workload.options.dt,
                                gravity=workload.options.gravity, **opt)
        b = workload.batch
        self.B, self.nq, self.nv, self.nc = b.B, b.q.shape[0], b.v.shape[0], b.ncmax
        self.device = device
        self.model_id = self.base.get("model_id")
        self.workspace = torch.empty(max(workspace_size(self.models, self.base, self.opt), 1), dtype=torch.uint8,
                                     device=device)
        f64 = dict(dtype=torch.float64, device=device)
        # per-call scratch outputs that nothing keeps (impulses, modes, status, iteration counts)
        self.scratch = {"lambda": torch.zeros(3 * self.nc, self.B, **f64),
                        "modes": torch.zeros(self.nc, self.B, dtype=torch.uint8, device=device),
                        "status": torch.zeros(self.B, dtype=torch.int32, device=device),
                        "iters": torch.zeros(self.B, dtype=torch.int32, device=device)}

    def _batch(self, q, v, tau):
        d = dict(self.base)
        d.update(q=q, v=v, tau=tau)
        return d

    def step(self, q, v, tau):
        """(q+, v+) as new tensors, and the step's tape (impulses, modes, status) for its VJP."""
        tape = {"lambda": torch.empty(3 * self.nc, self.B, dtype=torch.float64, device=self.device),
                "modes": torch.empty(self.nc, self.B, dtype=torch.uint8, device=self.device),
                "status": torch.empty(self.B, dtype=torch.int32, device=self.device)}
        out = dict(self.scratch, **tape, v_next=torch.empty(self.nv, self.B, dtype=torch.float64, device=self.device),
                   q_next=torch.empty(self.nq, self.B, dtype=torch.float64, device=self.device))
        sim_step(self.models, self._batch(q, v, tau), self.opt, out, self.workspace)
        return out["q_next"], out["v_next"], tape

    def autotune(self, q, v, tau):
        """Pick the pipeline schedule of this batch's forward step by timing (ds_autotune on
        sim_step at the state (q, v, tau)); returns the chosen schedule's description."""
        out = dict(self.scratch, v_next=torch.empty(self.nv, self.B, dtype=torch.float64, device=self.device),
                   q_next=torch.empty(self.nq, self.B, dtype=torch.float64, device=self.device))
        idx = autotune(self.models, self._batch(q, v, tau), self.opt, 0, out, workspace=self.workspace)
        return dict(describe_schedule(idx), index=idx)

    def vjp(self, q, v, tau, q_next, q_next_bar_raw, v_next_bar, tape=None):
        """Cotangents of (q raw, v, tau) from those of (q+ raw, v+); with the forward step's tape,
        the VJP of that very solution (only the finish kernel runs)."""
        e = lambda rows: torch.empty(rows, self.B, dtype=torch.float64, device=self.device)  # noqa: E731
        qn_t = e(self.nv)
        cotangent_to_tangent(self.models, q_next, q_next_bar_raw, qn_t, self.model_id)
        out = dict(self.scratch, v_next=e(self.nv), q_next=None)
        q_bar_t, v_bar, tau_bar = e(self.nv), e(self.nv), e(self.nv)
        if tape is not None:
            sim_step_vjp_tape(self.models, self._batch(q, v, tau), self.opt, v_next_bar, tape, out, q_bar_t, v_bar,
                              tau_bar, q_next_bar=qn_t)
        else:
            sim_step_vjp(self.models, self._batch(q, v, tau), self.opt, v_next_bar, out, q_bar_t, v_bar, tau_bar,
                         workspace=self.workspace, q_next_bar=qn_t)
        q_bar = torch.zeros(self.nq, self.B, dtype=torch.float64, device=self.device)
        cotangent_to_raw(self.models, q, q_bar_t, q_bar, self.model_id)
        return q_bar, v_bar, tau_bar


class SimStep(torch.autograd.Function):
    """(q, v, tau) -> (q+, v+) through sim_step; backward through sim_step_vjp."""

    @staticmethod
    def forward(ctx, q, v, tau, sc):
        q, v, tau = q.detach().contiguous(), v.detach().contiguous(), tau.detach().contiguous()
        qn, vn, tape = sc.step(q, v, tau)
        ctx.sc = sc
        ctx.save_for_backward(q, v, tau, qn, tape["lambda"], tape["modes"], tape["status"])
        return qn, vn

    @staticmethod
    def backward(ctx, gq, gv):
        q, v, tau, qn, lam, modes, status = ctx.saved_tensors
        gq = torch.zeros_like(qn) if gq is None else gq.contiguous()
        gv = torch.zeros_like(v) if gv is None else gv.contiguous()
        tape = {"lambda": lam, "modes": modes, "status": status}
        qb, vb, tb = ctx.sc.vjp(q, v, tau, qn, gq, gv, tape)
        return qb, vb, tb, None


def _segment(sc, q, v, *taus):
    for tau in taus:
        q, v = SimStep.apply(q, v, tau, sc)
    return q, v


def rollout(sc, q0, v0, taus, checkpoint_every=20):
    """(q_T, v_T) after len(taus) steps from (q0, v0); taus is a sequence of [nv][B] tensors."""
    q, v = q0, v0
    T = len(taus)
    if not checkpoint_every:
        return _segment(sc, q, v, *taus)
    for t0 in range(0, T, checkpoint_every):
        seg = list(taus[t0:t0 + checkpoint_every])
        q, v = torch.utils.checkpoint.checkpoint(_segment, sc, q, v, *seg, use_reentrant=False)
    return q, v
