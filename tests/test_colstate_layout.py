"""The split finish's column state overwrites an env's forward-state rows in place, and its prep
threads write the rows of the implicit part at a fixed offset, so its layout must agree in three
places: the host's row count (ds_colstate_rows, which sizes the workspace), the members the
column kernel visits (ColState::visit) and the offset of P the prep writes at
(ColState::kOffP).  Checked on the host for every compiled shape in both precisions (a small
host program compiled with nvcc; no GPU)."""
import os
import re
import shutil
import subprocess

import pytest

from paper_2409_07107_gb300 import build

PROG = r'''
#include "ds_kernel.cuh"
#include <cstdio>
#include <type_traits>
template <int NB, int NV, int NS, typename T>
void report() {
  ds::ColState<NB, NV, NS, T> cs;
  long long rows = 0, off_p = -1;
  cs.visit([&](auto* ptr, int n) {
    if ((const void*)ptr == (const void*)&cs.P[0][0]) off_p = rows;
    rows += n;
  });
  std::printf("%d %d %d %d %lld %d %d %lld %d\n", NB, NV, NS, (int)std::is_same<T, double>::value, rows,
              ds_colstate_rows(NB, NV, NS), ds::ColState<NB, NV, NS, T>::kRows, off_p,
              ds::ColState<NB, NV, NS, T>::kOffP);
}
int main() {
#define DS_SHAPE(NB, NV, NS) report<NB, NV, NS, double>(); report<NB, NV, NS, float>();
#include "ds_shapes_list.inc"
#undef DS_SHAPE
  return 0;
}
'''


def _nvcc():
    c = build._nvcc()
    return c if (os.path.isabs(c) and os.path.exists(c)) or shutil.which(c) else None


def test_colstate_rows_visit_and_offset_agree(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    src = tmp_path / "layout.cu"
    src.write_text(PROG)
    exe = tmp_path / "layout"
    r = subprocess.run([nvcc, "-std=c++17", "-I" + build.INCLUDE, "-I" + build.CSRC, str(src), "-o", str(exe)],
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60).stdout.split("\n")
    shapes = re.findall(r"DS_SHAPE\((\d+), (\d+), (\d+)\)", open(os.path.join(build.CSRC, "ds_shapes_list.inc")).read())
    lines = [ln.split() for ln in out if ln.strip()]
    assert len(lines) == 2 * len(shapes)
    for nb, nv, ns, dbl, rows, host_rows, k_rows, off_p, k_off_p in lines:
        assert int(rows) == int(host_rows) == int(k_rows), (nb, nv, ns, dbl)
        assert int(off_p) == int(k_off_p), (nb, nv, ns, dbl)
