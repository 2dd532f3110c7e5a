"""Seeded random pairs of convex shapes for the collision-detection tests (inputs only: no
collision arithmetic here).  Types 0 sphere (r), 1 capsule (half length, r), 2 box (half extents),
3 hull (first vertex, count, r: 8 to 20 random points on an ellipsoid with semi-axes in
[0.03, 0.1], kept in a shared pool, swept by r in [0, 0.02]); poses are uniformly random rotations
(normalised Gaussian quaternions) and positions in a cube of side 2 * spread, so that about half of
the pairs overlap for the default sizes.  Hulls appear only where ``types`` asks for them."""
import numpy as np

SPHERE, CAPSULE, BOX, HULL = 0, 1, 2, 3


def random_rotation(rng):
    w, x, y, z = rng.normal(size=4) / 1.0
    s = np.sqrt(w * w + x * x + y * y + z * z)
    w, x, y, z = w / s, x / s, y / s, z / s
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def random_size(rng, t, pool=None):
    if t == HULL:
        count = int(rng.integers(8, 21))
        axes = rng.uniform(0.03, 0.1, size=3)
        x = rng.normal(size=(count, 3))
        x = x / np.linalg.norm(x, axis=1, keepdims=True) * axes
        first = len(pool)
        pool.extend(x)
        return np.array([float(first), float(count), rng.uniform(0.0, 0.02)])
    if t == SPHERE:
        return np.array([rng.uniform(0.03, 0.1), 0.0, 0.0])
    if t == CAPSULE:
        return np.array([rng.uniform(0.03, 0.12), rng.uniform(0.02, 0.06), 0.0])
    return rng.uniform(0.03, 0.12, size=3)


def pairs(n, seed, spread=0.12, types=None):
    """n pairs: arrays type_a (n,), size_a (n, 3), pose_a (n, 12) and the same for B, and the hull
    vertex pool hull_vertices (V, 3)."""
    rng = np.random.default_rng(seed)
    out = {k: [] for k in ("type_a", "size_a", "pose_a", "type_b", "size_b", "pose_b")}
    pool = []
    for i in range(n):
        ta, tb = types[i % len(types)] if types is not None else (int(rng.integers(3)), int(rng.integers(3)))
        for side, t in (("a", ta), ("b", tb)):
            R = random_rotation(rng)
            p = rng.uniform(-spread, spread, size=3)
            out["type_" + side].append(t)
            out["size_" + side].append(random_size(rng, t, pool))
            out["pose_" + side].append(np.concatenate([R.ravel(), p]))
    res = {k: np.asarray(v, dtype=np.int32 if k.startswith("type") else np.float64) for k, v in out.items()}
    res["hull_vertices"] = np.asarray(pool, dtype=np.float64).reshape(-1, 3)
    return res


def oracle_shape(t, size, pool=None):
    """The oracle's shape for (type, size); a hull's vertices come from the pool."""
    from oracle import collision as C
    if t == HULL:
        first, count = int(size[0]), int(size[1])
        return C.Shape(pool[first:first + count], size[2])
    if t == SPHERE:
        return C.sphere(size[0])
    if t == CAPSULE:
        return C.capsule(size[0], size[1])
    return C.box(*size[:3])
