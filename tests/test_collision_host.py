"""The device collision detection (ds_collision.cuh: GJK for separated cores, the nearest facet of
the Minkowski difference for overlapping ones), compiled for the host with nvcc and run on the
CPU, against the oracle's collision detection by its definition (oracle/collision.py), no GPU.

Random sphere, capsule and box pairs (sizes of centimetres to decimetres), about half of them
overlapping: phi agrees within 1e-12 and the contact point, the normal, the tangent axes and the
witness points within 1e-10 (observed: 1e-16 for phi, 4e-13 for the normal).  The oracle takes
the convex hull of the whole Minkowski difference (Qhull) and the device GJK or the separating
axes, so a mistake in either one's region tests, support features or axis set shows up here.
Random poses put no two faces or edges exactly parallel, where the witness points would not be
unique.  Each check runs on a plain host build and on one with fused multiply-adds contracted (as
on the device), whose rounding differs in the near-degenerate decisions."""
import os
import platform
import shutil
import subprocess

import numpy as np
import pytest

from oracle import collision as C
from paper_2409_07107_gb300 import build

from tests.convex_pairs import BOX, CAPSULE, HULL, SPHERE, oracle_shape, pairs

PROG = r'''
#include "ds_collision.cuh"
#include <cstdio>
#include <vector>
int main() {
  int ta, tb, nhv;
  double sa[3], sb[3], pa[12], pb[12], out[DS_COLLIDE_OUT];
  if (std::scanf("%d", &nhv) != 1) return 1;
  std::vector<double> hv(3 * nhv + 3);
  for (int i = 0; i < 3 * nhv; ++i) std::scanf("%lf", &hv[i]);
  while (std::scanf("%d", &ta) == 1) {
    for (double& x : sa) std::scanf("%lf", &x);
    for (double& x : pa) std::scanf("%lf", &x);
    std::scanf("%d", &tb);
    for (double& x : sb) std::scanf("%lf", &x);
    for (double& x : pb) std::scanf("%lf", &x);
    ds::cd::collide(ta, sa, pa, tb, sb, pb, hv.data(), nhv, out);
    if (nhv == 0) {
      // the form without hulls (what the device runs for a batch without a hull pool) must give
      // the same numbers, bit for bit
      double o2[DS_COLLIDE_OUT];
      ds::cd::collide<false>(ta, sa, pa, tb, sb, pb, nullptr, 0, o2);
      for (int k = 0; k < DS_COLLIDE_OUT; ++k)
        if (!(o2[k] == out[k]) && !(o2[k] != o2[k] && out[k] != out[k])) return 3;
    }
    for (int k = 0; k < DS_COLLIDE_OUT; ++k) std::printf("%.17g ", out[k]);
    std::printf("\n");
  }
  return 0;
}
'''


def _host_build(tmp_path_factory, contracted):
    nvcc = build._nvcc()
    if not ((os.path.isabs(nvcc) and os.path.exists(nvcc)) or shutil.which(nvcc)):
        pytest.skip("nvcc not found")
    d = tmp_path_factory.mktemp("cd")
    src, exe = d / "cd.cu", d / "cd"
    src.write_text(PROG)
    flags = []
    if contracted:
        # fused multiply-adds wherever the compiler can form them, as the device code has: the
        # rounding differs from the plain build's, which moves near-degenerate decisions
        flags = ["-Xcompiler", "-ffp-contract=fast"] + (["-Xcompiler", "-mfma"] if platform.machine() == "x86_64" else [])
    r = subprocess.run([nvcc, "-std=c++17", "-O2", *flags, "-I" + build.INCLUDE, "-I" + build.CSRC, str(src), "-o", str(exe)],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]

    def run(P):
        hv = P.get("hull_vertices", np.zeros((0, 3)))
        lines = ["%d %s" % (len(hv), " ".join("%.17g" % x for x in np.ravel(hv)))]
        for k in range(len(P["type_a"])):
            fa = " ".join("%.17g" % x for x in np.concatenate([P["size_a"][k], P["pose_a"][k]]))
            fb = " ".join("%.17g" % x for x in np.concatenate([P["size_b"][k], P["pose_b"][k]]))
            lines.append("%d %s %d %s" % (P["type_a"][k], fa, P["type_b"][k], fb))
        out = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True, text=True, timeout=300)
        assert out.returncode == 0
        return np.array([[float(x) for x in ln.split()] for ln in out.stdout.splitlines() if ln.strip()])
    return run


@pytest.fixture(scope="module", params=["plain", "contracted"])
def host_collide(request, tmp_path_factory):
    return _host_build(tmp_path_factory, request.param == "contracted")


def oracle_collide(P, k):
    pool = P.get("hull_vertices")
    sa = oracle_shape(P["type_a"][k], P["size_a"][k], pool)
    sb = oracle_shape(P["type_b"][k], P["size_b"][k], pool)
    pa, pb = P["pose_a"][k], P["pose_b"][k]
    return C.collide(sa, pa[:9].reshape(3, 3), pa[9:], sb, pb[:9].reshape(3, 3), pb[9:])


def compare(P, got, tol=1e-12, tol_x=1e-10):
    """Per pair: phi, c, n, t1, t2, sa, sb against the oracle; returns (#overlapping, #apart)."""
    n_over = 0
    for k in range(len(P["type_a"])):
        ref = oracle_collide(P, k)
        g = got[k]
        assert abs(g[0] - ref["phi"]) <= tol, (k, g[0], ref["phi"])
        assert np.abs(g[4:7] - ref["n"]).max() <= tol_x, (k, g[4:7], ref["n"])
        Rc = ref["Rc"]
        assert np.abs(g[7:10] - Rc[:, 0]).max() <= tol_x and np.abs(g[10:13] - Rc[:, 1]).max() <= tol_x, k
        assert np.abs(g[1:4] - ref["c"]).max() <= tol_x, (k, g[1:4], ref["c"])
        assert np.abs(g[13:16] - ref["pa"]).max() <= tol_x and np.abs(g[16:19] - ref["pb"]).max() <= tol_x, k
        n_over += ref["phi"] < 0.0
    return n_over, len(P["type_a"]) - n_over


@pytest.mark.parametrize("types", [[(SPHERE, BOX), (BOX, SPHERE)], [(CAPSULE, BOX), (BOX, CAPSULE)], [(BOX, BOX)],
                                   [(SPHERE, SPHERE), (SPHERE, CAPSULE), (CAPSULE, CAPSULE)]])
def test_host_collide_against_oracle(host_collide, types):
    P = pairs(120, seed=100 + len(types) * 7 + types[0][0] * 3 + types[0][1], types=types)
    got = host_collide(P)
    n_over, n_apart = compare(P, got)
    assert n_over >= 10 and n_apart >= 10


@pytest.mark.parametrize("types", [[(HULL, HULL)], [(HULL, BOX), (BOX, HULL)], [(HULL, SPHERE), (CAPSULE, HULL)]])
def test_host_collide_hulls_against_oracle(host_collide, types):
    """Convex hulls (8 to 20 vertices, swept by a radius): GJK when apart, the expanding polytope
    when the cores overlap, against the oracle's hull of the whole Minkowski difference."""
    P = pairs(120, seed=300 + types[0][1] * 5 + len(types), types=types)
    got = host_collide(P)
    n_over, n_apart = compare(P, got)
    assert n_over >= 10 and n_apart >= 10


def test_host_collide_identical_shapes_at_one_pose(host_collide):
    """The degenerate overlap of a shape with its copy at the same pose: for boxes phi = -2 x the
    smallest half extent (the separating axes); for hulls, where GJK's first support difference is
    the origin itself, the enclosing tetrahedron is built by GJK's intersection iteration and EPA
    gives the oracle's phi (its normal is one of a +-m pair, as D = A - A is symmetric), with
    sb - sa = phi n."""
    P = pairs(8, seed=3, types=[(BOX, BOX), (HULL, HULL)])
    for k in range(8):
        P["type_b"][k], P["size_b"][k], P["pose_b"][k] = P["type_a"][k], P["size_a"][k], P["pose_a"][k]
    got = host_collide(P)
    assert np.isfinite(got).all()
    for k in range(8):
        phi, n, sa, sb = got[k][0], got[k][4:7], got[k][13:16], got[k][16:19]
        ref = -2.0 * P["size_a"][k].min() if P["type_a"][k] == BOX else oracle_collide(P, k)["phi"]
        assert abs(phi - ref) <= 1e-12
        assert abs(n @ n - 1.0) <= 1e-12 and np.abs(sb - sa - phi * n).max() <= 1e-12


def test_host_collide_bad_hull_range_is_nan(host_collide):
    P = pairs(3, seed=6, types=[(HULL, BOX)])
    P["size_a"][1][1] = 40.0                              # more than 32 vertices
    P["size_a"][2][0] = len(P["hull_vertices"]) - 2.0     # runs past the pool
    got = host_collide(P)
    assert np.isfinite(got[0]).all() and np.isnan(got[1]).all() and np.isnan(got[2]).all()


def test_host_collide_witness_identity_large_batch(host_collide):
    """On 20000 pairs: sb - sa = phi n and |n| = 1 for every pair (a false overlap from a flat
    GJK simplex, seen once in 262144 pairs with contracted rounding, broke the first)."""
    P = pairs(20000, seed=77)
    got = host_collide(P)
    phi, nrm, sa, sb = got[:, 0], got[:, 4:7], got[:, 13:16], got[:, 16:19]
    assert np.abs(sb - sa - phi[:, None] * nrm).max() <= 1e-12
    assert np.abs(np.einsum("ij,ij->i", nrm, nrm) - 1.0).max() <= 1e-12


def test_host_collide_unknown_type_is_nan(host_collide):
    P = pairs(2, seed=5, types=[(SPHERE, BOX)])
    P["type_b"][1] = 7
    got = host_collide(P)
    assert np.isfinite(got[0]).all() and np.isnan(got[1]).all()


PROG_SMOOTH = r'''
#include "ds_collision.cuh"
#include <cstdio>
#include <vector>
int main() {
  int ta, tb, S;
  double sigma, sa[3], sb[3], pa[12], pb[12], J[84];
  while (std::scanf("%d %lf", &S, &sigma) == 2) {
    std::vector<double> eps(12 * S);
    for (double& x : eps) std::scanf("%lf", &x);
    std::scanf("%d", &ta);
    for (double& x : sa) std::scanf("%lf", &x);
    for (double& x : pa) std::scanf("%lf", &x);
    std::scanf("%d", &tb);
    for (double& x : sb) std::scanf("%lf", &x);
    for (double& x : pb) std::scanf("%lf", &x);
    ds::cd::smoothing_jacobian(ta, sa, pa, tb, sb, pb, nullptr, 0, S, eps.data(), sigma, J);
    for (int k = 0; k < 84; ++k) std::printf("%.17g ", J[k]);
    std::printf("\n");
  }
  return 0;
}
'''


def test_host_smoothing_jacobian_against_oracle(tmp_path):
    """App. C's randomized-smoothing derivative on the device side (the poses moved by the caller's
    samples as world-frame twists, antithetic differences of (phi, c, n)) equals the oracle's
    estimator fed the same samples, pair by pair."""
    nvcc = build._nvcc()
    if not ((os.path.isabs(nvcc) and os.path.exists(nvcc)) or shutil.which(nvcc)):
        pytest.skip("nvcc not found")
    src, exe = tmp_path / "sm.cu", tmp_path / "sm"
    src.write_text(PROG_SMOOTH)
    r = subprocess.run([nvcc, "-std=c++17", "-O2", "-I" + build.INCLUDE, "-I" + build.CSRC, str(src), "-o", str(exe)],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    P = pairs(48, seed=404)
    rng = np.random.default_rng(5)
    sigma, S = 2e-3, 6
    eps = rng.normal(0.0, sigma, size=(S, 12))
    head = "%d %.17g %s" % (S, sigma, " ".join("%.17g" % x for x in eps.ravel()))
    lines = []
    for k in range(len(P["type_a"])):
        fa = " ".join("%.17g" % x for x in np.concatenate([P["size_a"][k], P["pose_a"][k]]))
        fb = " ".join("%.17g" % x for x in np.concatenate([P["size_b"][k], P["pose_b"][k]]))
        lines.append("%s %d %s %d %s" % (head, P["type_a"][k], fa, P["type_b"][k], fb))
    out = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True, text=True, timeout=300)
    got = np.array([[float(x) for x in ln.split()] for ln in out.stdout.splitlines() if ln.strip()]).reshape(-1, 7, 12)
    for k in range(len(P["type_a"])):
        sa = oracle_shape(P["type_a"][k], P["size_a"][k])
        sb = oracle_shape(P["type_b"][k], P["size_b"][k])
        pa, pb = P["pose_a"][k], P["pose_b"][k]
        ref = C.randomized_smoothing_jacobian(sa, pa[:9].reshape(3, 3), pa[9:], sb, pb[:9].reshape(3, 3), pb[9:],
                                              sigma, S, None, eps_samples=eps)
        assert np.abs(got[k] - ref).max() <= 1e-8 * max(1.0, np.abs(ref).max()), k
