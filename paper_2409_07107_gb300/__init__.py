"""GB300-native batched differentiable contact-simulation step (Python binding of libdiffsim.so).

The library computes, for B independent environments at once, one time step of frictional-contact
multibody simulation and its implicit derivatives (arXiv 2409.07107, Sec. 2-3, App. A-D).  This
module only marshals arguments: every step of the computation runs in the CUDA kernels behind the
C ABI declared in include/diffsim.h.  There is no CPU fallback: if the library is missing the calls
raise.

    from paper_2409_07107_gb300 import scenes, Simulator
    sim = Simulator(scenes.arm_cube(4096), precision="fp64")
    out = sim.step_jac()          # v_next, q_next, lambda, modes, status, dv_dq, dv_dv, dv_dtau
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# DIFFSIM_LIB selects another build of the library (the checked build, libdiffsim_check.so)
LIB_PATH = os.environ.get("DIFFSIM_LIB") or os.path.join(HERE, "libdiffsim.so")

DS_OK, DS_EINVAL, DS_ECUDA, DS_ENOMEM, DS_EUNSUPPORTED, DS_ETOOLARGE = 0, -1, -2, -3, -4, -5
DS_FP64, DS_MIXED = 0, 1
DS_ADMM, DS_PGS = 0, 1
MODE_BREAKING, MODE_STICKING, MODE_SLIDING, MODE_INACTIVE = 0, 1, 2, 3
ENV_NOT_CONVERGED, ENV_NONFINITE, ENV_SINGULAR, ENV_NEAR_SWITCH, ENV_BAD_SLOT, ENV_QUEUE_TIMEOUT = 1, 2, 4, 8, 16, 32

EXPORTS = ("ds_model_create", "ds_model_destroy", "ds_model_dims", "ds_options_default",
           "ds_status_string", "sim_step", "sim_step_jac", "sim_step_vjp", "ds_fma_peak", "ds_workspace_size",
           "sim_step_jac_noalloc", "ds_profile", "ds_profile_read", "ds_cotangent_to_tangent",
           "ds_cotangent_to_raw", "ds_autotune", "sim_step_vjp_tape", "ds_set_schedule", "ds_check_bad_indices",
           "ds_check_self_test", "ds_collide", "ds_collide_smoothed")


class ds_model_desc(ctypes.Structure):
    _fields_ = [("nbodies", ctypes.c_int32), ("parent", ctypes.c_void_p), ("joint_type", ctypes.c_void_p),
                ("axis", ctypes.c_void_p), ("joint_rot", ctypes.c_void_p), ("joint_pos", ctypes.c_void_p),
                ("mass", ctypes.c_void_p), ("com", ctypes.c_void_p), ("inertia", ctypes.c_void_p)]


class ds_batch(ctypes.Structure):
    _fields_ = [("B", ctypes.c_int32), ("ncmax", ctypes.c_int32), ("model_id", ctypes.c_void_p),
                ("q", ctypes.c_void_p), ("v", ctypes.c_void_p), ("tau", ctypes.c_void_p),
                ("c_link", ctypes.c_void_p), ("c_point", ctypes.c_void_p), ("c_radius", ctypes.c_void_p),
                ("c_mu", ctypes.c_void_p), ("plane", ctypes.c_void_p), ("model_slots", ctypes.c_void_p)]


class ds_options(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_double), ("gravity", ctypes.c_double * 3), ("admm_max_iter", ctypes.c_int32),
                ("admm_eps", ctypes.c_double), ("polish_iters", ctypes.c_int32), ("ncp_tol", ctypes.c_double),
                ("eps_sigma", ctypes.c_double), ("eps_lambda", ctypes.c_double),
                ("margin_delta", ctypes.c_double), ("precision", ctypes.c_int32),
                ("baumgarte_kp", ctypes.c_double), ("baumgarte_kd", ctypes.c_double),
                ("contact_margin", ctypes.c_double), ("ncp_solver", ctypes.c_int32),
                ("queue_poll_limit", ctypes.c_int32), ("admm_rho_adapt", ctypes.c_int32)]


class ds_step_out(ctypes.Structure):
    _fields_ = [("v_next", ctypes.c_void_p), ("q_next", ctypes.c_void_p), ("lambda_", ctypes.c_void_p),
                ("modes", ctypes.c_void_p), ("env_status", ctypes.c_void_p), ("iters", ctypes.c_void_p)]


_lib = None


def lib():
    """Load libdiffsim.so (built in-tree by build.py).  Raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libdiffsim.so is not built (run paper_2409_07107_gb300.build.build()); "
                               "there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32 = ctypes.c_void_p, ctypes.c_int32
        L.ds_model_create.argtypes = [ctypes.POINTER(ds_model_desc), ctypes.POINTER(vp)]
        L.ds_model_destroy.argtypes = [vp]
        L.ds_model_dims.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)]
        L.ds_options_default.argtypes = [ctypes.POINTER(ds_options)]
        L.ds_options_default.restype = None
        L.ds_status_string.argtypes = [ctypes.c_int]
        L.ds_status_string.restype = ctypes.c_char_p
        common = [vp, i32, ctypes.POINTER(ds_batch), ctypes.POINTER(ds_options)]
        sz = ctypes.c_size_t
        L.sim_step.argtypes = common + [ctypes.POINTER(ds_step_out), vp, sz, vp]
        L.sim_step_jac.argtypes = common + [ctypes.POINTER(ds_step_out), vp, vp, vp, vp, sz, vp]
        L.sim_step_vjp.argtypes = common + [vp, vp, ctypes.POINTER(ds_step_out), vp, vp, vp, vp, sz, vp]
        L.ds_workspace_size.argtypes = common + [ctypes.POINTER(sz)]
        L.sim_step_jac_noalloc.argtypes = common + [ctypes.POINTER(ds_step_out), vp, vp, vp, vp]
        L.ds_profile.argtypes = [i32]
        L.ds_profile_read.argtypes = [vp, vp]
        L.ds_fma_peak.argtypes = [vp, i32, i32, i32, vp]
        L.ds_collide.argtypes = [i32, vp, vp, vp, vp, vp, vp, vp, i32, vp, vp]
        L.ds_collide_smoothed.argtypes = [i32, vp, vp, vp, vp, vp, vp, vp, i32, i32, vp, ctypes.c_double, vp, vp]
        for f in ("ds_cotangent_to_tangent", "ds_cotangent_to_raw"):
            getattr(L, f).argtypes = [vp, i32, i32, vp, vp, vp, vp, vp]
        L.ds_autotune.argtypes = common + [i32, vp, ctypes.POINTER(ds_step_out), vp, vp, vp, vp, sz, vp, vp]
        L.sim_step_vjp_tape.argtypes = common + [vp, vp, ctypes.POINTER(ds_step_out), ctypes.POINTER(ds_step_out),
                                                 vp, vp, vp, vp]
        L.ds_set_schedule.argtypes = common + [i32, i32]
        L.ds_check_bad_indices.argtypes = [ctypes.POINTER(ctypes.c_uint64)]
        L.ds_check_self_test.argtypes = [i32, i32, ctypes.POINTER(ctypes.c_uint64)]
        for f in ("ds_model_create", "ds_model_destroy", "ds_model_dims", "sim_step", "sim_step_jac", "sim_step_vjp",
                  "ds_fma_peak", "ds_workspace_size", "sim_step_jac_noalloc", "ds_profile", "ds_profile_read",
                  "ds_cotangent_to_tangent", "ds_cotangent_to_raw", "ds_autotune", "sim_step_vjp_tape",
                  "ds_set_schedule", "ds_check_bad_indices", "ds_check_self_test"):
            getattr(L, f).restype = ctypes.c_int
        _lib = L
    return _lib


class DiffsimError(RuntimeError):
    pass


def _check(status):
    if status != DS_OK:
        raise DiffsimError("diffsim: %s (%d)" % (lib().ds_status_string(status).decode(), status))


def _ptr(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


class DeviceModel:
    """A model copied to the current CUDA device (ds_model_create)."""

    def __init__(self, model):
        self._keep = [np.ascontiguousarray(model.parent, np.int32), np.ascontiguousarray(model.jtype, np.int32),
                      np.ascontiguousarray(model.axis, np.float64), np.ascontiguousarray(model.jrot, np.float64),
                      np.ascontiguousarray(model.jpos, np.float64), np.ascontiguousarray(model.mass, np.float64),
                      np.ascontiguousarray(model.com, np.float64), np.ascontiguousarray(model.inertia, np.float64)]
        k = self._keep
        d = ds_model_desc(model.nb, *[a.ctypes.data for a in k])
        h = ctypes.c_void_p()
        _check(lib().ds_model_create(ctypes.byref(d), ctypes.byref(h)))
        self.handle = h
        self.nb, self.nq, self.nv = model.nb, model.nq, model.nv

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.ds_model_destroy(self.handle)
            self.handle = None


def make_options(precision="fp64", **kw):
    o = ds_options()
    lib().ds_options_default(ctypes.byref(o))
    o.precision = DS_MIXED if precision in ("mixed", DS_MIXED) else DS_FP64
    for k, v in kw.items():
        if k == "gravity":
            o.gravity[:] = list(v)
        else:
            setattr(o, k, v)
    return o


def _models_array(models):
    arr = (ctypes.c_void_p * len(models))(*[m.handle.value for m in models])
    return arr


def _batch_struct(t):
    return ds_batch(t["q"].shape[1], t["c_link"].shape[0], _ptr(t.get("model_id")), _ptr(t["q"]), _ptr(t["v"]),
                    _ptr(t["tau"]), _ptr(t["c_link"]), _ptr(t["c_point"]), _ptr(t["c_radius"]), _ptr(t["c_mu"]),
                    _ptr(t["plane"]), _host_ptr(t.get("model_slots")))


def _host_ptr(a):
    """Address of a host int32 numpy array (kept alive by the caller's dict), or NULL."""
    return ctypes.c_void_p(0 if a is None else a.ctypes.data)


def _out_struct(o):
    return ds_step_out(_ptr(o["v_next"]), _ptr(o.get("q_next")), _ptr(o.get("lambda")), _ptr(o.get("modes")),
                       _ptr(o.get("status")), _ptr(o.get("iters")))


def _stream(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ws(workspace):
    if workspace is None:
        return ctypes.c_void_p(0), 0
    return ctypes.c_void_p(workspace.data_ptr()), workspace.numel() * workspace.element_size()


def workspace_size(models, batch, opt):
    b = _batch_struct(batch)
    n = ctypes.c_size_t()
    _check(lib().ds_workspace_size(_models_array(models), len(models), ctypes.byref(b), ctypes.byref(opt),
                                   ctypes.byref(n)))
    return n.value


def sim_step(models, batch, opt, out, workspace=None, stream=None):
    """C-ABI sim_step on device tensors (dicts of torch tensors, see Simulator)."""
    b, o = _batch_struct(batch), _out_struct(out)
    _check(lib().sim_step(_models_array(models), len(models), ctypes.byref(b), ctypes.byref(opt),
                          ctypes.byref(o), *_ws(workspace), _stream(stream)))


def sim_step_jac(models, batch, opt, out, dv_dq, dv_dv, dv_dtau, workspace=None, stream=None):
    b, o = _batch_struct(batch), _out_struct(out)
    _check(lib().sim_step_jac(_models_array(models), len(models), ctypes.byref(b), ctypes.byref(opt),
                              ctypes.byref(o), _ptr(dv_dq), _ptr(dv_dv), _ptr(dv_dtau), *_ws(workspace),
                              _stream(stream)))


def sim_step_jac_noalloc(models, batch, opt, out, dv_dq, dv_dv, dv_dtau, stream=None):
    """C-ABI sim_step_jac_noalloc: sim_step_jac with the library's fixed scratch, no allocation."""
    b, o = _batch_struct(batch), _out_struct(out)
    _check(lib().sim_step_jac_noalloc(_models_array(models), len(models), ctypes.byref(b), ctypes.byref(opt),
                                      ctypes.byref(o), _ptr(dv_dq), _ptr(dv_dv), _ptr(dv_dtau), _stream(stream)))


def sim_step_vjp(models, batch, opt, v_next_bar, out, q_bar, v_bar, tau_bar, workspace=None, stream=None,
                 q_next_bar=None):
    b, o = _batch_struct(batch), _out_struct(out)
    _check(lib().sim_step_vjp(_models_array(models), len(models), ctypes.byref(b), ctypes.byref(opt),
                              _ptr(v_next_bar), _ptr(q_next_bar), ctypes.byref(o), _ptr(q_bar), _ptr(v_bar),
                              _ptr(tau_bar), *_ws(workspace), _stream(stream)))


def cotangent_to_tangent(models, q, q_bar_raw, q_bar_tangent, model_id=None, stream=None):
    """C-ABI ds_cotangent_to_tangent: (dq_raw/deta)^T q_bar_raw at q, all [rows][B] device tensors."""
    _check(lib().ds_cotangent_to_tangent(_models_array(models), len(models), q.shape[1], _ptr(model_id), _ptr(q),
                                         _ptr(q_bar_raw), _ptr(q_bar_tangent), _stream(stream)))


def cotangent_to_raw(models, q, q_bar_tangent, q_bar_raw, model_id=None, stream=None):
    """C-ABI ds_cotangent_to_raw: (deta/dq_raw)^T q_bar_tangent at q, all [rows][B] device tensors."""
    _check(lib().ds_cotangent_to_raw(_models_array(models), len(models), q.shape[1], _ptr(model_id), _ptr(q),
                                     _ptr(q_bar_tangent), _ptr(q_bar_raw), _stream(stream)))


# Schedule knobs and their options, as the library encodes them: the schedule index is the
# mixed-radix number of the option positions, the first knob the lowest digit.
SCHEDULE_KNOBS = (
    ("round_caps", ("default", "halved", "doubled")),
    ("row_per_lane_admm_from_round", (3, 5, None)),
    ("finish_ctas_per_sm", (0, 4, 8)),
    ("newton", ("cooperative", "one thread per env")),
    ("overlapped_finish_after_round", ("setup", 2, 4, 5, None)),
    ("two_warp_admm_from_round", (3, 5, None)),
    ("overlapped_finish_keeps_free_every_nth_sm", (None, 8, 4)),
    ("speculative_newton_from_round", (3, 5, None)),
    ("single_contact_presolve", (True, False)),
    ("launch", ("pipeline", "persistent")),
    ("finish", ("one kernel", "split")),
)
NUM_SCHEDULES = 58320


def describe_schedule(index):
    """The schedule with this index (as ds_autotune returns it), knob by knob."""
    i, d = int(index), {}
    for name, opts in SCHEDULE_KNOBS:
        d[name] = opts[i % len(opts)]
        i //= len(opts)
    return d


def schedule_index(round_caps=0, wide=1, finish=1, newton=0, overlap=3, pair=1, reserve=1, spec=2, presolve=0,
                   launch=0, split=0):
    """Schedule index from option positions (each the position in its SCHEDULE_KNOBS tuple); the
    defaults give the library's default schedule."""
    idx, mul = 0, 1
    for pos, (_, opts) in zip((round_caps, wide, finish, newton, overlap, pair, reserve, spec, presolve, launch, split),
                              SCHEDULE_KNOBS):
        assert 0 <= pos < len(opts)
        idx += pos * mul
        mul *= len(opts)
    return idx


def autotune(models, batch, opt, mode, out, o0=None, o1=None, o2=None, v_next_bar=None, workspace=None,
             stream=None):
    """C-ABI ds_autotune; returns the chosen schedule index."""
    b, o = _batch_struct(batch), _out_struct(out)
    chosen = ctypes.c_int32(-1)
    _check(lib().ds_autotune(_models_array(models), len(models), ctypes.byref(b), ctypes.byref(opt), int(mode),
                             _ptr(v_next_bar), ctypes.byref(o), _ptr(o0), _ptr(o1), _ptr(o2), *_ws(workspace),
                             _stream(stream), ctypes.byref(chosen)))
    return chosen.value


def set_schedule(models, batch, opt, mode, index):
    """C-ABI ds_set_schedule: later calls of `mode` on batches of this signature use schedule
    `index` (as returned by autotune); -1 restores the default."""
    b = _batch_struct(batch)
    _check(lib().ds_set_schedule(_models_array(models), len(models), ctypes.byref(b), ctypes.byref(opt), int(mode),
                                 int(index)))


def sim_step_vjp_tape(models, batch, opt, v_next_bar, tape, out, q_bar, v_bar, tau_bar, q_next_bar=None, stream=None):
    """C-ABI sim_step_vjp_tape: the VJP of the solution recorded in `tape` (a dict with "lambda",
    "modes", "status" from a preceding step on the same inputs); only the finish kernel runs."""
    b, o, t = _batch_struct(batch), _out_struct(out), _out_struct(dict(tape, v_next=None))
    _check(lib().sim_step_vjp_tape(_models_array(models), len(models), ctypes.byref(b), ctypes.byref(opt),
                                   _ptr(v_next_bar), _ptr(q_next_bar), ctypes.byref(t), ctypes.byref(o), _ptr(q_bar),
                                   _ptr(v_bar), _ptr(tau_bar), _stream(stream)))


def fma_peak(out, blocks, iters, fp64, stream=None):
    """Launch the FMA-throughput probe (2 * 8 * iters * blocks * 256 flops)."""
    _check(lib().ds_fma_peak(_ptr(out), blocks, iters, 1 if fp64 else 0, _stream(stream)))


CONVEX_SPHERE, CONVEX_CAPSULE, CONVEX_BOX, CONVEX_HULL = 0, 1, 2, 3
CONVEX_HULL_MAX = 32
COLLIDE_OUT = 19


def _hull_pool(hull_vertices):
    return (ctypes.c_void_p(0), 0) if hull_vertices is None else (_ptr(hull_vertices), hull_vertices.shape[0])


def _check_pairs(type_a, size_a, pose_a, type_b, size_b, pose_b, hull_vertices, extra=()):
    """The kernels read n pairs from each buffer: reject a dtype, shape, device or layout that would
    make them read past it."""
    import torch
    n = type_a.shape[0] if type_a.dim() == 1 else -1
    want = [(type_a, torch.int32, (n,)), (type_b, torch.int32, (n,)), (size_a, torch.float64, (n, 3)),
            (size_b, torch.float64, (n, 3)), (pose_a, torch.float64, (n, 12)), (pose_b, torch.float64, (n, 12))]
    if hull_vertices is not None:
        want.append((hull_vertices, torch.float64, (hull_vertices.shape[0], 3)))
    want += list(extra)
    for t, dtype, shape in want:
        if t.dtype != dtype or tuple(t.shape) != tuple(shape) or not t.is_contiguous() or t.device != type_a.device \
                or (t.numel() and not t.is_cuda):
            raise ValueError("diffsim: expected a contiguous CUDA %s tensor of shape %s, got %s %s on %s"
                             % (dtype, tuple(shape), t.dtype, tuple(t.shape), t.device))
    return n


def collide(type_a, size_a, pose_a, type_b, size_b, pose_b, hull_vertices=None, out=None, stream=None):
    """Collision detection between convex shapes (ds_collide), one pair per row: type (int32, n),
    size (FP64, n x 3; a hull's is (first vertex, count, radius)), pose (FP64, n x 12: R row-major,
    then p), hull_vertices (FP64, V x 3, body frames), all CUDA tensors.  Returns out (FP64,
    n x 19): phi, c, n, t1, t2, the witness points on A's and B's surfaces."""
    import torch
    n = _check_pairs(type_a, size_a, pose_a, type_b, size_b, pose_b, hull_vertices)
    if out is None:
        out = torch.empty((n, COLLIDE_OUT), dtype=torch.float64, device=type_a.device)
    _check_pairs(type_a, size_a, pose_a, type_b, size_b, pose_b, None, [(out, torch.float64, (n, COLLIDE_OUT))])
    hv, nhv = _hull_pool(hull_vertices)
    _check(lib().ds_collide(n, _ptr(type_a), _ptr(size_a), _ptr(pose_a), _ptr(type_b), _ptr(size_b),
                            _ptr(pose_b), hv, nhv, _ptr(out), _stream(stream)))
    return out


def collide_smoothed(type_a, size_a, pose_a, type_b, size_b, pose_b, eps, sigma, hull_vertices=None, out=None,
                     stream=None):
    """Randomized-smoothing derivative of the collision detection (ds_collide_smoothed): eps (FP64,
    S x 12 CUDA tensor, samples of N(0, sigma^2 I)); returns (n x 7 x 12) d(phi, c, n)/d(twists of
    A and B)."""
    import torch
    n = _check_pairs(type_a, size_a, pose_a, type_b, size_b, pose_b, hull_vertices,
                     [(eps, torch.float64, (eps.shape[0], 12))])
    if out is None:
        out = torch.empty((n, 7, 12), dtype=torch.float64, device=type_a.device)
    _check_pairs(type_a, size_a, pose_a, type_b, size_b, pose_b, None, [(out, torch.float64, (n, 7, 12))])
    hv, nhv = _hull_pool(hull_vertices)
    _check(lib().ds_collide_smoothed(n, _ptr(type_a), _ptr(size_a), _ptr(pose_a), _ptr(type_b), _ptr(size_b),
                                     _ptr(pose_b), hv, nhv, eps.shape[0], _ptr(eps), float(sigma), _ptr(out),
                                     _stream(stream)))
    return out


STAGES = ("setup", "admm", "newton", "finish", "fused")


def profile(enable):
    """Turn stage tracing (CUDA events around every library kernel) on or off."""
    _check(lib().ds_profile(1 if enable else 0))


def profile_read():
    """{stage: (milliseconds, launches)} since the last read; waits for the recorded events."""
    ms = (ctypes.c_double * 5)()
    n = (ctypes.c_int32 * 5)()
    _check(lib().ds_profile_read(ctypes.cast(ms, ctypes.c_void_p), ctypes.cast(n, ctypes.c_void_p)))
    return {k: (ms[i], n[i]) for i, k in enumerate(STAGES)}


def check_bad_indices():
    """Checked build: indices found out of range by the kernels since the last call (cleared).
    Raises DiffsimError (unsupported) with the normal build."""
    n = ctypes.c_uint64()
    _check(lib().ds_check_bad_indices(ctypes.byref(n)))
    return n.value


def check_self_test(index, n):
    """Checked build: the count one check of `index` against [0, n) gives (1 outside, 0 inside)."""
    c = ctypes.c_uint64()
    _check(lib().ds_check_self_test(int(index), int(n), ctypes.byref(c)))
    return c.value


def batch_to_device(batch, device="cuda"):
    import torch
    f64 = dict(dtype=torch.float64, device=device)
    i32 = dict(dtype=torch.int32, device=device)
    t = dict(q=torch.as_tensor(batch.q, **f64).contiguous(), v=torch.as_tensor(batch.v, **f64).contiguous(),
             tau=torch.as_tensor(batch.tau, **f64).contiguous(), c_link=torch.as_tensor(batch.c_link, **i32).contiguous(),
             c_point=torch.as_tensor(batch.c_point, **f64).contiguous(),
             c_radius=torch.as_tensor(batch.c_radius, **f64).contiguous(),
             c_mu=torch.as_tensor(batch.c_mu, **f64).contiguous(), plane=torch.as_tensor(batch.plane, **f64).contiguous())
    if batch.model_id is not None:
        t["model_id"] = torch.as_tensor(batch.model_id, **i32).contiguous()
    if batch.model_slots is not None:
        t["model_slots"] = np.ascontiguousarray(batch.model_slots, dtype=np.int32)   # host array
    return t


class Simulator:
    """Device-resident batch + outputs for one workload; thin wrapper over the three C-ABI calls.
    Keyword options are ds_options fields (e.g. admm_max_iter, baumgarte_kp, baumgarte_kd); the
    rest keep ds_options_default's values, dt and gravity come from the workload."""

    def __init__(self, workload, precision=None, device="cuda", pipeline=True, **opt):
        import torch
        self.workload = workload
        self.models = [DeviceModel(m) for m in workload.models]
        self.batch = batch_to_device(workload.batch, device)
        prec = precision or workload.precision
        self.opt = make_options(prec, dt=workload.options.dt, gravity=workload.options.gravity, **opt)
        B = workload.batch.B
        nq = workload.batch.q.shape[0]
        nv = workload.batch.v.shape[0]
        nc = workload.batch.ncmax
        f64 = dict(dtype=torch.float64, device=device)
        self.nv = nv
        self.out = dict(v_next=torch.zeros(nv, B, **f64), q_next=torch.zeros(nq, B, **f64),
                        **{"lambda": torch.zeros(3 * nc, B, **f64)},
                        modes=torch.zeros(nc, B, dtype=torch.uint8, device=device),
                        status=torch.zeros(B, dtype=torch.int32, device=device),
                        iters=torch.zeros(B, dtype=torch.int32, device=device))
        self.jac = None
        self.vjp_out = None
        self.workspace = None
        if pipeline and B > 0:
            nbytes = workspace_size(self.models, self.batch, self.opt)
            self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=device)

    def step(self, stream=None):
        sim_step(self.models, self.batch, self.opt, self.out, self.workspace, stream)
        return self.out

    def step_jac(self, stream=None):
        import torch
        B = self.workload.batch.B
        if self.jac is None:
            n = self.nv
            self.jac = [torch.zeros(n, n, B, dtype=torch.float64, device=self.out["v_next"].device) for _ in range(3)]
        sim_step_jac(self.models, self.batch, self.opt, self.out, *self.jac, workspace=self.workspace, stream=stream)
        return dict(self.out, dv_dq=self.jac[0], dv_dv=self.jac[1], dv_dtau=self.jac[2])

    def autotune(self, kind="jac", v_next_bar=None):
        """Pick this batch's pipeline schedule by timing the candidates (ds_autotune); returns the
        chosen schedule's description.  Later calls on batches of the same signature use it."""
        import torch
        mode = {"step": 0, "jac": 1, "vjp": 2}[kind]
        B = self.workload.batch.B
        dev = self.out["v_next"].device
        if kind == "jac":
            if self.jac is None:
                n = self.nv
                self.jac = [torch.zeros(n, n, B, dtype=torch.float64, device=dev) for _ in range(3)]
            o = self.jac
        elif kind == "vjp":
            if self.vjp_out is None:
                self.vjp_out = [torch.zeros_like(self.out["v_next"]) for _ in range(3)]
            o = self.vjp_out
        else:
            o = [None, None, None]
        idx = autotune(self.models, self.batch, self.opt, mode, self.out, *o, v_next_bar=v_next_bar,
                       workspace=self.workspace)
        return dict(describe_schedule(idx), index=idx)

    def set_schedule(self, index, kind="jac"):
        """Use schedule `index` for this batch's `kind` calls (-1: the default); returns its description."""
        set_schedule(self.models, self.batch, self.opt, {"step": 0, "jac": 1, "vjp": 2}[kind], index)
        return None if index < 0 else dict(describe_schedule(index), index=index)

    def capture(self, kind="jac", v_next_bar=None, q_next_bar=None):
        """Capture one step (kind "step", "jac" or "vjp", on this Simulator's buffers) in a CUDA
        graph and return a function that replays it on the current stream.  Inputs are read from
        self.batch (and the given cotangent tensors) at replay time, outputs land in the same
        tensors as the eager calls.  Run one eager call first: the library's first call on a device
        creates its helper streams, which must not happen during capture."""
        import torch
        fn = {"step": lambda: self.step(), "jac": lambda: self.step_jac(),
              "vjp": lambda: self.step_vjp(v_next_bar, q_next_bar=q_next_bar)}[kind]
        fn()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fn()
        return g.replay

    def step_vjp(self, v_next_bar, stream=None, q_next_bar=None):
        import torch
        if self.vjp_out is None:
            self.vjp_out = [torch.zeros_like(self.out["v_next"]) for _ in range(3)]
        sim_step_vjp(self.models, self.batch, self.opt, v_next_bar.contiguous(), self.out, *self.vjp_out,
                     workspace=self.workspace, stream=stream,
                     q_next_bar=None if q_next_bar is None else q_next_bar.contiguous())
        return dict(self.out, q_bar=self.vjp_out[0], v_bar=self.vjp_out[1], tau_bar=self.vjp_out[2])
