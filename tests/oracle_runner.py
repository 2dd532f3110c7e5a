"""Runs the oracle over many envs in a spawn-started process pool (safe next to a CUDA context).

Eq. 1 can have more than one solution (redundant contacts, and the non-monotone De Saxce form of
Coulomb friction), so each env can be solved by two independent routes of the oracle: the ADMM
iteration and projected Gauss-Seidel sweeps, each followed by the Newton polish on the identified
modes.  The first route's results are the env's record; the second route's are in its "alt" list.
"""
import multiprocessing as mp
import os
import types

import numpy as np

KEEP = ("v_next", "q_next", "lam", "modes", "margin", "slots", "residual", "converged", "dv_dq", "dv_dv",
        "dv_dtau", "G", "g", "mu", "iters")


def _with_route(opt, route):
    d = dict(vars(opt))
    d["ncp_route"] = route
    return types.SimpleNamespace(**d)


def _one(args):
    model, env, opt, jac, routes = args
    from oracle import step as S
    recs = []
    for route in routes:
        o = _with_route(opt, route)
        st = S.step_jac(model, env, o) if jac else S.step(model, env, o)
        rec = {k: st[k] for k in KEEP if k in st}
        rec["route"] = route
        recs.append(rec)
    out = recs[0]
    out["alt"] = recs[1:]
    return out


def run_oracle(workload, envs, jac=True, opt=None, processes=None, routes=("admm", "pgs")):
    """Oracle results for the given env indices of a workload (list of dicts, one per env; the
    results of the second and later routes are under "alt")."""
    b = workload.batch
    opt = opt or workload.options
    args = []
    for e in envs:
        mi = 0 if b.model_id is None else int(b.model_id[e])
        m = workload.models[mi]
        args.append((m, b.env(e, m), opt, jac, tuple(routes)))
    n = processes or min(len(args), max(1, (os.cpu_count() or 2)))
    if n <= 1 or len(args) <= 2:
        return [_one(a) for a in args]
    ctx = mp.get_context("spawn")
    with ctx.Pool(n) as pool:
        return pool.map(_one, args, chunksize=max(1, len(args) // (4 * n)))


def rel_err(x, ref, floor=1e-6):
    x, ref = np.asarray(x, float), np.asarray(ref, float)
    return float(np.max(np.abs(x - ref)) / max(np.max(np.abs(ref)) if ref.size else 0.0, floor)) if ref.size else 0.0


def jac_of(r):
    return np.concatenate([r["dv_dq"], r["dv_dv"], r["dv_dtau"]], axis=1)


def candidates(r):
    """The env's oracle solutions: the first route's and those of the other routes."""
    return [r] + list(r.get("alt", []))


def member_invariant(r, tol=1e-9):
    """True when every route of the oracle gives the same v+, modes and Jacobians for this env (the
    derivative does not depend on which solution of Eq. 1 a solver reaches)."""
    c = candidates(r)
    for o in c[1:]:
        if rel_err(o["v_next"], c[0]["v_next"]) > tol or list(o["modes"]) != list(c[0]["modes"]):
            return False
        if "dv_dq" in o and rel_err(jac_of(o), jac_of(c[0])) > tol:
            return False
    return True
