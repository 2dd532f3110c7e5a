"""The checked build of the library (compiled with DS_CHECK: every tree index, work-list env index
and shared-memory group index is checked, and one out of range is counted instead of faulting)
on small batches of every workload, pipeline and fused kernels, FP64 and mixed, VJP, the PGS
iteration, the adaptive penalty, the split finish and the persistent launch: no index out of
range, and the same results as the normal build.  The counting itself
is tested with one check of an index outside and one inside its range."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MIXED_CASES = ("arm_cube_mixed", "humanoid", "humanoid_split", "uneven_persistent")  # checked_run's mixed-form cases


def test_checked_build_matches_and_finds_no_bad_index(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2409_07107_gb300 as ds
    from paper_2409_07107_gb300 import build
    from tests.checked_run import run_all
    build.build()
    checked = build.build(check=True)
    path = str(tmp_path / "checked.npz")
    env = dict(os.environ, DIFFSIM_LIB=checked)
    r = subprocess.run([sys.executable, "-m", "tests.checked_run", path], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    got = dict(np.load(path))
    assert int(got["check/self_test_outside"]) == 1 and int(got["check/self_test_inside"]) == 0
    assert int(got["check/bad_indices"]) == 0
    with pytest.raises(ds.DiffsimError):          # the normal build has no checks
        ds.check_bad_indices()
    ref = run_all()
    assert set(ref) == {k for k in got if not k.startswith("check/")}
    for k, v in ref.items():
        g = got[k]
        mixed = k.split("/")[0] in MIXED_CASES
        if v.dtype.kind in "iu":
            # the checks change no arithmetic; in the FP32 bulk of the mixed form the compiler may
            # still schedule and contract differently, which can move a convergence test
            assert np.array_equal(g, v) if not mixed else (g == v).mean() >= 0.98, k
        elif v.size:
            scale = max(float(np.max(np.abs(v))), 1e-6)
            assert float(np.max(np.abs(g - v))) <= (1e-5 if mixed else 1e-12) * scale, k
