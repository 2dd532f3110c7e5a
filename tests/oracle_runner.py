"""Runs the oracle over many envs in a spawn-started process pool (safe next to a CUDA context)."""
import multiprocessing as mp
import os

import numpy as np


def _one(args):
    model, env, opt, jac = args
    from oracle import step as S
    st = S.step_jac(model, env, opt) if jac else S.step(model, env, opt)
    keep = ("v_next", "q_next", "lam", "modes", "margin", "slots", "residual", "converged", "dv_dq", "dv_dv", "dv_dtau")
    return {k: st[k] for k in keep if k in st}


def run_oracle(workload, envs, jac=True, opt=None, processes=None):
    """Oracle results for the given env indices of a workload (list of dicts)."""
    b = workload.batch
    opt = opt or workload.options
    args = []
    for e in envs:
        mi = 0 if b.model_id is None else int(b.model_id[e])
        m = workload.models[mi]
        args.append((m, b.env(e, m), opt, jac))
    n = processes or min(len(args), max(1, (os.cpu_count() or 2)))
    if n <= 1 or len(args) <= 2:
        return [_one(a) for a in args]
    ctx = mp.get_context("spawn")
    with ctx.Pool(n) as pool:
        return pool.map(_one, args, chunksize=max(1, len(args) // (4 * n)))


def rel_err(x, ref, floor=1e-6):
    x, ref = np.asarray(x, float), np.asarray(ref, float)
    return float(np.max(np.abs(x - ref)) / max(np.max(np.abs(ref)) if ref.size else 0.0, floor)) if ref.size else 0.0
