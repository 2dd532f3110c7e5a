"""GPU parity of the batched collision detection (ds_collide, one pair per thread) against the
oracle's collision detection by its definition (oracle/collision.py).

* 2048 random sphere, capsule and box pairs (about half overlapping), every one compared with the
  oracle: phi within 1e-12, the contact point, normal, tangent axes and witness points within
  1e-10 (the host build of the same code agrees with the oracle to 4e-13);
* 262144 pairs (the size of a batch of 16384 humanoids with 16 candidate pairs each) with a
  ragged tail: 512 sampled pairs against the oracle, and every pair checked for what holds at any
  size: n unit, (t1, t2, n) orthonormal and right-handed, sb - sa = phi n;
* an unknown shape type gives NaN for that pair only, and an empty batch launches nothing;
* the randomized-smoothing derivative (ds_collide_smoothed) against the oracle's estimator fed the
  same samples."""
import numpy as np
import pytest

import paper_2409_07107_gb300 as ds
from tests.convex_pairs import pairs
from tests.test_collision_host import compare, oracle_collide

pytestmark = pytest.mark.gpu


def _device(P):
    import torch
    return {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in P.items()}


def _run(P):
    import torch
    D = _device(P)
    hv = D["hull_vertices"] if P["hull_vertices"].size else None
    out = ds.collide(D["type_a"], D["size_a"], D["pose_a"], D["type_b"], D["size_b"], D["pose_b"], hull_vertices=hv)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_collide_against_oracle():
    P = pairs(2048, seed=2024)
    got = _run(P)
    n_over, n_apart = compare(P, got)
    assert n_over >= 200 and n_apart >= 200


def test_collide_large_batch_sampled_and_properties():
    n = 262144 + 37
    P = pairs(n, seed=77)
    got = _run(P)
    assert np.isfinite(got).all()
    phi, nrm, t1, t2, sa, sb = got[:, 0], got[:, 4:7], got[:, 7:10], got[:, 10:13], got[:, 13:16], got[:, 16:19]
    assert np.abs(np.einsum("ij,ij->i", nrm, nrm) - 1.0).max() <= 1e-12
    assert np.abs(np.einsum("ij,ij->i", t1, nrm)).max() <= 1e-12
    assert np.abs(np.einsum("ij,ij->i", t1, t1) - 1.0).max() <= 1e-12
    assert np.abs(t2 - np.cross(nrm, t1)).max() <= 1e-12
    assert np.abs(sb - sa - phi[:, None] * nrm).max() <= 1e-12
    rng = np.random.default_rng(3)
    idx = np.concatenate([rng.choice(n, size=500, replace=False), np.arange(n - 12, n)])
    sub = {k: (v if k == "hull_vertices" else v[idx]) for k, v in P.items()}
    compare(sub, got[idx])


def test_collide_unknown_type_and_empty_batch():
    import torch
    P = pairs(300, seed=9)
    P["type_a"][17] = 5
    got = _run(P)
    assert np.isnan(got[17]).all()
    ok = np.ones(len(got), bool)
    ok[17] = False
    assert np.isfinite(got[ok]).all()
    ref = oracle_collide(P, 16)
    assert abs(got[16, 0] - ref["phi"]) <= 1e-12
    e = torch.empty(0, dtype=torch.int32, device="cuda")
    f = torch.empty((0, 3), dtype=torch.float64, device="cuda")
    g = torch.empty((0, 12), dtype=torch.float64, device="cuda")
    out = ds.collide(e, f, g, e, f, g)
    assert out.shape == (0, ds.COLLIDE_OUT)


def test_collide_smoothed_against_oracle():
    """App. C's randomized-smoothing derivative (ds_collide_smoothed) against the oracle's estimator
    fed the same samples: 4096 pairs, 8 samples, every 64th pair compared (relative 1e-8)."""
    import torch
    from oracle import collision as C
    from tests.convex_pairs import oracle_shape
    P = pairs(4096, seed=31)
    D = _device(P)
    sigma, S = 2e-3, 8
    eps = np.random.default_rng(6).normal(0.0, sigma, size=(S, 12))
    J = ds.collide_smoothed(D["type_a"], D["size_a"], D["pose_a"], D["type_b"], D["size_b"], D["pose_b"],
                            torch.from_numpy(eps).cuda(), sigma)
    torch.cuda.synchronize()
    J = J.cpu().numpy()
    assert np.isfinite(J).all()
    for k in range(0, 4096, 64):
        pa, pb = P["pose_a"][k], P["pose_b"][k]
        ref = C.randomized_smoothing_jacobian(oracle_shape(P["type_a"][k], P["size_a"][k]), pa[:9].reshape(3, 3), pa[9:],
                                              oracle_shape(P["type_b"][k], P["size_b"][k]), pb[:9].reshape(3, 3), pb[9:],
                                              sigma, S, None, eps_samples=eps)
        assert np.abs(J[k] - ref).max() <= 1e-8 * max(1.0, np.abs(ref).max()), k
