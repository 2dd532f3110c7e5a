"""GPU parity of the batched collision detection for convex hulls (ds_collide with a hull vertex
pool) against the oracle's collision detection by its definition (the hull of the whole Minkowski
difference): hulls of 8 to 20 vertices against hulls, boxes, spheres and capsules, GJK when apart
and the expanding polytope when the cores overlap, every pair compared.  Collected after the step
suites on purpose (the newest device path; its host build is checked in test_collision_host.py)."""
import numpy as np
import pytest

from tests.convex_pairs import BOX, CAPSULE, HULL, SPHERE, pairs
from tests.test_collision_host import compare
from tests.test_gpu_collision import _run

pytestmark = pytest.mark.gpu


def test_collide_hulls_against_oracle():
    """Convex hulls (8 to 20 vertices from a shared pool) against hulls, boxes, spheres and
    capsules: GJK when apart, the expanding polytope when the cores overlap; 1536 pairs, every one
    compared with the oracle."""
    P = pairs(1536, seed=4242, types=[(HULL, HULL), (HULL, BOX), (SPHERE, HULL), (HULL, CAPSULE)])
    got = _run(P)
    assert np.isfinite(got).all()
    n_over, n_apart = compare(P, got)
    assert n_over >= 150 and n_apart >= 150
