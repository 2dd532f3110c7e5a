"""The C-ABI library loads, exports every symbol include/diffsim.h declares, and rejects bad
arguments before touching a GPU (no compute call here)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2409_07107_gb300 as ds

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "diffsim.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = "\n".join(l for l in src.splitlines() if not l.lstrip().startswith("#"))
    return sorted(set(re.findall(r"\b(\w+)\s*\([^;{]*\)\s*;", src)) - {"if", "while", "sizeof"})


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(ds.LIB_PATH):
        from paper_2409_07107_gb300 import build
        build.build()
    return ds.lib()


def test_exports_every_declared_symbol(L):
    names = _declared()
    assert set(ds.EXPORTS) <= set(names)
    for n in names:
        assert hasattr(L, n), n


def test_status_strings_and_defaults(L):
    assert L.ds_status_string(0) == b"ok"
    assert b"invalid" in L.ds_status_string(-1)
    o = ds.make_options()
    assert o.dt == 1e-3 and o.precision == ds.DS_FP64 and o.admm_max_iter > 0
    # the last fields of ds_options sit where the binding expects them (the C default fills them)
    assert o.margin_delta == 1e-3 and o.baumgarte_kp == 1.0 and o.baumgarte_kd == 0.0
    raw = ds.ds_options()
    raw.contact_margin = 7.0
    raw.queue_poll_limit = 7
    raw.admm_rho_adapt = 7                   # the C default must overwrite the binding's last field
    L.ds_options_default(ctypes.byref(raw))
    assert raw.contact_margin == 0.0 and raw.queue_poll_limit == 1 << 22 and raw.admm_rho_adapt == 0


def _desc(nb=2, parent=(-1, 0), jtype=(0, 0), axis=None):
    arrs = [np.array(parent, np.int32), np.array(jtype, np.int32),
            np.array(axis if axis is not None else [[1.0, 0, 0]] * nb), np.tile(np.eye(3), (nb, 1, 1)),
            np.zeros((nb, 3)), np.ones(nb), np.zeros((nb, 3)), np.tile([0.1, 0.1, 0.1, 0, 0, 0], (nb, 1))]
    arrs = [np.ascontiguousarray(a) for a in arrs]
    return arrs, ds.ds_model_desc(nb, *[a.ctypes.data for a in arrs])


@pytest.mark.parametrize("kw", [dict(parent=(0, -1)), dict(jtype=(0, 1)), dict(axis=[[2.0, 0, 0], [1.0, 0, 0]]),
                                dict(jtype=(5, 0))])
def test_model_create_rejects_bad_descriptions(L, kw):
    keep, d = _desc(**kw)
    h = ctypes.c_void_p()
    assert L.ds_model_create(ctypes.byref(d), ctypes.byref(h)) == ds.DS_EINVAL
    assert L.ds_model_create(None, ctypes.byref(h)) == ds.DS_EINVAL


def test_model_create_rejects_non_preorder(L):
    # body 3 is a child of body 1 but comes after body 2 (a child of 0): subtree of 1 not contiguous
    keep, d = _desc(nb=4, parent=(-1, 0, 0, 1), jtype=(0, 0, 0, 0))
    h = ctypes.c_void_p()
    assert L.ds_model_create(ctypes.byref(d), ctypes.byref(h)) == ds.DS_EINVAL


def test_step_rejects_bad_arguments(L):
    o = ds.make_options()
    b = ds.ds_batch(4, 1, None, None, None, None, None, None, None, None, None)
    out = ds.ds_step_out(None, None, None, None, None, None)
    models = (ctypes.c_void_p * 1)(None)
    assert L.sim_step(models, 1, ctypes.byref(b), ctypes.byref(o), ctypes.byref(out), None, 0, None) == ds.DS_EINVAL
    assert L.sim_step(None, 1, ctypes.byref(b), ctypes.byref(o), ctypes.byref(out), None, 0, None) == ds.DS_EINVAL
    n = ctypes.c_size_t()
    # the workspace holds each model's forward state, so sizing it needs the models
    assert L.ds_workspace_size(models, 1, ctypes.byref(b), ctypes.byref(o), ctypes.byref(n)) == ds.DS_EINVAL
    b.B = -1
    assert L.sim_step_jac(models, 1, ctypes.byref(b), ctypes.byref(o), ctypes.byref(out), None, None, None,
                          None, 0, None) == ds.DS_EINVAL
    assert L.ds_workspace_size(models, 1, ctypes.byref(b), ctypes.byref(o), ctypes.byref(n)) == ds.DS_EINVAL
    b.ncmax = 99
    assert L.sim_step_vjp(models, 1, ctypes.byref(b), ctypes.byref(o), None, None, ctypes.byref(out), None, None,
                          None, None, 0, None) == ds.DS_EINVAL


def test_collide_rejects_bad_arguments(L):
    buf = ctypes.c_void_p(1)
    assert L.ds_collide(-1, buf, buf, buf, buf, buf, buf, None, 0, buf, None) == ds.DS_EINVAL
    assert L.ds_collide(4, None, buf, buf, buf, buf, buf, None, 0, buf, None) == ds.DS_EINVAL
    assert L.ds_collide(4, buf, buf, buf, buf, buf, buf, None, 0, None, None) == ds.DS_EINVAL
    assert L.ds_collide(4, buf, buf, buf, buf, buf, buf, buf, -1, buf, None) == ds.DS_EINVAL
    assert L.ds_collide(0, None, None, None, None, None, None, None, 0, None, None) == ds.DS_OK


def test_collide_smoothed_rejects_bad_arguments(L):
    buf = ctypes.c_void_p(1)
    args = [buf] * 6 + [None, 0]
    assert L.ds_collide_smoothed(-1, *args, 4, buf, 1e-3, buf, None) == ds.DS_EINVAL
    assert L.ds_collide_smoothed(4, *args, 0, buf, 1e-3, buf, None) == ds.DS_EINVAL
    assert L.ds_collide_smoothed(4, *args, 4, buf, 0.0, buf, None) == ds.DS_EINVAL
    assert L.ds_collide_smoothed(4, *args, 4, buf, float("nan"), buf, None) == ds.DS_EINVAL
    assert L.ds_collide_smoothed(4, *args, 4, None, 1e-3, buf, None) == ds.DS_EINVAL
    assert L.ds_collide_smoothed(4, *([buf] * 6), buf, -2, 4, buf, 1e-3, buf, None) == ds.DS_EINVAL
    assert L.ds_collide_smoothed(0, *([None] * 6), None, 0, 0, None, 0.0, None, None) == ds.DS_OK


def test_collide_binding_rejects_bad_tensors():
    """The binding checks dtype, shape and layout before any launch (a float32 size or a short pose
    buffer would be read past its end); checked on CPU tensors, which it also rejects."""
    torch = pytest.importorskip("torch")
    n = 4
    t = torch.zeros(n, dtype=torch.int32)
    z = torch.zeros((n, 3), dtype=torch.float64)
    p = torch.zeros((n, 12), dtype=torch.float64)
    with pytest.raises(ValueError):
        ds.collide(t, z.float(), p, t, z, p)
    with pytest.raises(ValueError):
        ds.collide(t, z, p[:, :9].contiguous(), t, z, p)
    with pytest.raises(ValueError):
        ds.collide(t.long(), z, p, t, z, p)
    with pytest.raises(ValueError):
        ds.collide(t, z, p, t, z, p)                     # CPU tensors
    with pytest.raises(ValueError):
        ds.collide_smoothed(t, z, p, t, z, p, torch.zeros((2, 6), dtype=torch.float64), 1e-3)
