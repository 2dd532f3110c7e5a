"""App. C's contact rows J_c and contact-placement terms on the device side (ds_appc.cuh), compiled
for the host with nvcc and run on the CPU, against the oracle's (oracle/collision.py pair_jc,
appc_dJcv_dq, appc_dJctlam_dq, dcd_dbody), no GPU.  The inputs (contact placement, body poses, twists, Jacobians and dCD/dM_i) come from the
oracle's kinematics and collision detection for a contact between two links of a random 7-dof arm
and between an arm link and a fixed box; the expected values are the oracle's terms, which
test_oracle_collision.py pins against central differences."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import collision as C
from oracle import rigid
from paper_2409_07107_gb300 import build

PROG = r'''
#include "ds_appc.cuh"
#include <cstdio>
#include <vector>
static void rd(double* x, int n) { for (int i = 0; i < n; ++i) if (std::scanf("%lf", &x[i]) != 1) x[i] = 0.0; }
int main() {
  int nv, has[2];
  while (std::scanf("%d %d %d", &nv, &has[0], &has[1]) == 3) {
    double Rc[9], c[3], lam[3], R[2][9], p[2][3], V[2][6], D[2][36];
    std::vector<double> J[2] = {std::vector<double>(6 * nv), std::vector<double>(6 * nv)};
    rd(Rc, 9); rd(c, 3); rd(lam, 3);
    for (int b = 0; b < 2; ++b) { rd(R[b], 9); rd(p[b], 3); rd(V[b], 6); rd(J[b].data(), 6 * nv); rd(D[b], 36); }
    std::vector<double> t1(3 * nv), t2(nv * nv), scratch(3 * nv), jc(3 * nv);
    ds::cd::pair_jc(nv, Rc, c, has[0] ? R[0] : nullptr, p[0], J[0].data(), has[1] ? R[1] : nullptr, p[1],
                    J[1].data(), jc.data());
    ds::cd::appc_dJcv_dq(nv, Rc, c, has[0] ? R[0] : nullptr, p[0], V[0], J[0].data(), D[0],
                         has[1] ? R[1] : nullptr, p[1], V[1], J[1].data(), D[1], t1.data());
    ds::cd::appc_dJctlam_dq(nv, lam, Rc, c, has[0] ? R[0] : nullptr, p[0], J[0].data(), D[0],
                            has[1] ? R[1] : nullptr, p[1], J[1].data(), D[1], scratch.data(), t2.data());
    for (double x : t1) std::printf("%.17g ", x);
    for (double x : t2) std::printf("%.17g ", x);
    for (double x : jc) std::printf("%.17g ", x);
    std::printf("\n");
  }
  return 0;
}
'''


def _arm_pair(rng, kind):
    from paper_2409_07107_gb300 import scenes
    from scipy.spatial.transform import Rotation
    model, tip = scenes.arm7(rng)
    q = rng.uniform(-np.pi, np.pi, size=7)
    v = rng.normal(size=7)
    I3 = np.eye(3)
    if kind == "self":
        pair = (C.sphere(0.05), 6, (I3, np.asarray(tip, float)), C.box(0.05, 0.08, 0.06), 2,
                (Rotation.from_rotvec(rng.normal(size=3)).as_matrix(), np.zeros(3)))
    else:
        pair = (C.capsule(0.05, 0.03), 4, (Rotation.from_rotvec(rng.normal(size=3)).as_matrix(), np.zeros(3)),
                C.box(0.3, 0.3, 0.1), -1, (I3, np.array([0.0, 0.0, -0.5])))
    return model, q, v, pair


def _line(model, q, v, pair, lam):
    Rc, c, _ = C.pair_placement(model, q, pair)
    Js = rigid.body_jacobians(model, q)
    vel = rigid.body_velocities(model, q, v)
    nv = Js[0].shape[1]
    dcd = (C.dcd_dbody(model, q, pair, 0), C.dcd_dbody(model, q, pair, 1))
    fields = [nv, int(pair[1] >= 0), int(pair[4] >= 0)]
    nums = [Rc.ravel(), c, lam]
    for which, body in ((0, pair[1]), (1, pair[4])):
        if body < 0:
            nums += [np.zeros(9), np.zeros(3), np.zeros(6), np.zeros(6 * nv), np.zeros(36)]
            continue
        R, p = C.body_pose(model, q, body)
        nums += [R.ravel(), p, vel[body], Js[body].ravel(), dcd[which].ravel()]
    ref1 = C.appc_dJcv_dq(model, q, v, pair, dcd)
    ref2 = C.appc_dJctlam_dq(model, q, lam, pair, dcd)
    ref3 = C.pair_jc(model, q, pair)
    return " ".join(str(x) for x in fields) + " " + " ".join("%.17g" % x for x in np.concatenate(nums)), ref1, ref2, ref3


@pytest.mark.parametrize("kind", ["self", "world"])
def test_appc_terms_against_oracle(tmp_path, kind):
    nvcc = build._nvcc()
    if not ((os.path.isabs(nvcc) and os.path.exists(nvcc)) or shutil.which(nvcc)):
        pytest.skip("nvcc not found")
    src, exe = tmp_path / "appc.cu", tmp_path / "appc"
    src.write_text(PROG)
    r = subprocess.run([nvcc, "-std=c++17", "-O2", "-I" + build.INCLUDE, "-I" + build.CSRC, str(src), "-o", str(exe)],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines, refs = [], []
    for seed in range(6):
        rng = np.random.default_rng(50 + seed + (0 if kind == "self" else 100))
        model, q, v, pair = _arm_pair(rng, kind)
        ln, r1, r2, r3 = _line(model, q, v, pair, rng.normal(size=3))
        lines.append(ln)
        refs.append((r1, r2, r3))
    out = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True, text=True, timeout=120)
    rows = [np.array([float(x) for x in ln.split()]) for ln in out.stdout.splitlines() if ln.strip()]
    assert len(rows) == len(refs)
    for row, (r1, r2, r3) in zip(rows, refs):
        nv = r1.shape[1]
        g1, g2 = row[:3 * nv].reshape(3, nv), row[3 * nv:3 * nv + nv * nv].reshape(nv, nv)
        g3 = row[3 * nv + nv * nv:].reshape(3, nv)
        assert np.abs(g3 - r3).max() <= 1e-13 * max(1.0, np.abs(r3).max())
        assert np.abs(r1).max() > 1e-3 and np.abs(r2).max() > 1e-3
        assert np.abs(g1 - r1).max() <= 1e-12 * max(1.0, np.abs(r1).max())
        assert np.abs(g2 - r2).max() <= 1e-12 * max(1.0, np.abs(r2).max())


def test_appc_compiles_for_sm103a(tmp_path):
    """The same functions compile as device code for sm_103a (a kernel calling them; no GPU)."""
    nvcc = build._nvcc()
    if not ((os.path.isabs(nvcc) and os.path.exists(nvcc)) or shutil.which(nvcc)):
        pytest.skip("nvcc not found")
    src = tmp_path / "appc_dev.cu"
    src.write_text(r'''
#include "ds_appc.cuh"
__global__ void k(const double* in, double* out) {
  double scratch[21];
  ds::cd::appc_dJcv_dq(7, in, in + 9, in + 12, in + 21, in + 24, in + 30, in + 72, nullptr, nullptr, nullptr,
                       nullptr, nullptr, out);
  ds::cd::appc_dJctlam_dq(7, in + 108, in, in + 9, in + 12, in + 21, in + 30, in + 72, nullptr, nullptr, nullptr,
                          nullptr, scratch, out + 21);
  ds::cd::dcd_dbody(2, in, in + 3, in + 15, 0, in + 27, in + 30, in + 42, nullptr, 0, 1, 1e-6, out + 70);
  ds::cd::dcd_dbody_smoothed(2, in, in + 3, in + 15, 0, in + 27, in + 30, in + 42, nullptr, 0, 0, 4, in + 54, 1e-4,
                             out + 106);
}
''')
    r = subprocess.run([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-I" + build.INCLUDE,
                        "-I" + build.CSRC, "-c", str(src), "-o", str(tmp_path / "appc_dev.o")],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]


PROG_DCD = r'''
#include "ds_appc.cuh"
#include <cstdio>
#include <vector>
static void rd(double* x, int n) { for (int i = 0; i < n; ++i) if (std::scanf("%lf", &x[i]) != 1) x[i] = 0.0; }
int main() {
  int ta, tb, which, S;
  while (std::scanf("%d %d %d %d", &ta, &tb, &which, &S) == 4) {
    double sa[3], sb[3], Ma[12], Mb[12], oa[12], ob[12], h, out[36];
    rd(sa, 3); rd(Ma, 12); rd(oa, 12); rd(sb, 3); rd(Mb, 12); rd(ob, 12); rd(&h, 1);
    std::vector<double> eps(6 * S + 6);
    rd(eps.data(), 6 * S);
    // S = 0: central differences with step h; S > 0: the smoothing estimate with sigma = h
    const bool ok = S == 0 ? ds::cd::dcd_dbody(ta, sa, Ma, oa, tb, sb, Mb, ob, nullptr, 0, which, h, out)
                           : ds::cd::dcd_dbody_smoothed(ta, sa, Ma, oa, tb, sb, Mb, ob, nullptr, 0, which, S,
                                                        eps.data(), h, out);
    std::printf("%d ", ok ? 1 : 0);
    for (double x : out) std::printf("%.17g ", x);
    std::printf("\n");
  }
  return 0;
}
'''


def _device_shape(shape):
    """(type, size) of the device collision detection for the oracle's sphere, capsule or box."""
    core, r = shape.core, shape.radius
    if len(core) == 1:
        return 0, [r, 0.0, 0.0]
    if len(core) == 2:
        return 1, [float(core[1][2]), r, 0.0]
    return 2, list(np.abs(core[-1]))


def test_dcd_dbody_against_oracle(tmp_path):
    """dCD/dM_i by central differences of the device collision detection, in the body's local twist,
    and by App. C's randomized smoothing fed the same samples, against the oracle's (the same
    definitions on its own collision detection): both bodies of a pair between two arm links, and
    the arm body of a pair against a fixed box."""
    nvcc = build._nvcc()
    if not ((os.path.isabs(nvcc) and os.path.exists(nvcc)) or shutil.which(nvcc)):
        pytest.skip("nvcc not found")
    src, exe = tmp_path / "dcd.cu", tmp_path / "dcd"
    src.write_text(PROG_DCD)
    r = subprocess.run([nvcc, "-std=c++17", "-O2", "-I" + build.INCLUDE, "-I" + build.CSRC, str(src), "-o", str(exe)],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines, refs = [], []
    for kind in ("self", "world"):
        for seed in range(4):
            rng = np.random.default_rng(70 + seed + (0 if kind == "self" else 100))
            model, q, _, pair = _arm_pair(rng, kind)
            sa, ba, (Ea, ra), sb, bb, (Eb, rb) = pair
            Ma = np.concatenate([np.ravel(C.body_pose(model, q, ba)[0]), C.body_pose(model, q, ba)[1]])
            Mb = np.concatenate([np.ravel(C.body_pose(model, q, bb)[0]), C.body_pose(model, q, bb)[1]])
            ta, za = _device_shape(sa)
            tb, zb = _device_shape(sb)
            for which in ((0, 1) if bb >= 0 else (0,)):
                nums = np.concatenate([za, Ma, np.ravel(Ea), ra, zb, Mb, np.ravel(Eb), rb, [1e-6]])
                lines.append("%d %d %d 0 %s" % (ta, tb, which, " ".join("%.17g" % x for x in nums)))
                refs.append(C.dcd_dbody(model, q, pair, which))
                # App. C's smoothing estimate with 8 Gaussian samples, the same on both sides
                sig = 1e-4
                eps = rng.normal(0.0, sig, size=(8, 6))
                nums = np.concatenate([za, Ma, np.ravel(Ea), ra, zb, Mb, np.ravel(Eb), rb, [sig], eps.ravel()])
                lines.append("%d %d %d 8 %s" % (ta, tb, which, " ".join("%.17g" % x for x in nums)))
                refs.append(C.dcd_dbody_smoothed(model, q, pair, which, sig, eps))
    out = subprocess.run([str(exe)], input="\n".join(lines) + "\n", capture_output=True, text=True, timeout=120)
    rows = [np.array([float(x) for x in ln.split()]) for ln in out.stdout.splitlines() if ln.strip()]
    assert len(rows) == len(refs)
    for row, ref in zip(rows, refs):
        assert row[0] == 1.0
        assert np.abs(ref).max() > 0.1
        assert np.abs(row[1:].reshape(6, 6) - ref).max() <= 1e-7 * max(1.0, np.abs(ref).max())
