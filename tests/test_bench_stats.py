"""The benchmark's error statistics against the oracle (no GPU): an env whose v+ is off and whose
impulse does not solve Eq. 1 is an error; one whose impulse solves Eq. 1 for the oracle's problem
data (another solution, as the parity tests accept) is counted apart and left out of the maxima."""
import numpy as np

import bench
from oracle import step as S
from paper_2409_07107_gb300 import scenes


def _snapshot(wl, envs):
    m = wl.models[0]
    recs, lams = [], []
    for e in envs:
        env = wl.batch.env(e, m)
        st = S.step_jac(m, env, wl.options)
        recs.append({k: st[k] for k in ("v_next", "modes", "margin", "slots", "dv_dq", "dv_dv", "dv_dtau",
                                         "G", "g", "mu")})
        lams.append(st["lam"])
    n, nc = len(envs), wl.batch.ncmax
    snap = {"v_next": np.stack([r["v_next"] for r in recs], 1), "modes": np.full((nc, n), 3, np.uint8),
            "lambda": np.zeros((3 * nc, n)), "_form": "fp64"}
    for k in ("dv_dq", "dv_dv", "dv_dtau"):
        snap[k] = np.stack([r[k] for r in recs], 2)
    for j, r in enumerate(recs):
        for i, s in enumerate(r["slots"]):
            snap["modes"][s, j] = r["modes"][i]
            snap["lambda"][3 * s:3 * s + 3, j] = lams[j][3 * i:3 * i + 3]
    return recs, snap


def test_error_and_other_solution_counts():
    wl = scenes.arm_cube(64)
    envs = [e for e in range(64) if S.step(wl.models[0], wl.batch.env(e, wl.models[0]), wl.options)["slots"]][:6]
    sub = scenes.Workload(wl.name, wl.models, wl.batch.take(envs), wl.options)
    recs, snap = _snapshot(sub, range(len(envs)))
    exact = bench.error_stats(sub, snap, recs)
    assert exact["v_next"]["max"] <= 1e-15 and exact["v_next_off_by_1e6"] == 0
    assert exact["other_solution_of_eq1"]["envs"] == 0
    # env 0: v+ moved, impulse still a solution of Eq. 1 -> counted apart, not an error
    snap["v_next"][0, 0] += 0.5
    # env 1: v+ moved and the impulse zeroed (not a solution while contacts push) -> an error
    snap["v_next"][0, 1] += 0.5
    snap["lambda"][:, 1] = 0.0
    st = bench.error_stats(sub, snap, recs)
    assert st["other_solution_of_eq1"]["envs"] == 1
    assert st["other_solution_of_eq1"]["v_next_max_diff"] > 1e-3
    assert st["v_next_off_by_1e6"] == 1
    assert st["v_next"]["envs"] == len(envs) - 1 and st["v_next"]["max"] > 1e-3
