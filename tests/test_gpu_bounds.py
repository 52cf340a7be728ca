"""The bounds-checked build (libmisr_check.so, compiled with MISR_BOUNDS_CHECK) on the odd
geometries: every tile shape, the streaming shape (its item split included) and both storage
types, ragged and one-pixel images, frame counts below f^2, f = 1, 3 and 4, the gradient and a
mixed batch; and the frame-wise pass on frame sets it alone runs (several frames per phase, far
and off-lattice shifts, binning, its three tap widths), whose adjoint gathers' tap indices and
tile slots of sums are checked too.  No shared-memory item position, global
store, tile or group index or TMA x coordinate may fail its check, and the images must equal
the normal build's bit for bit (the checks change nothing when they pass).  compute-sanitizer
is closed on this machine; this build stands in for it."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _child(lib, out):
    r = subprocess.run([sys.executable, "-m", "tests.bounds_child", lib, out, ROOT], cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_bounds_checked_build_on_odd_geometries(tmp_path):
    from paper_2108_04315_b300 import build
    checked = build.build(checked=True)
    normal = build.build()
    rec = _child(checked, str(tmp_path / "checked.npz"))
    assert rec["bits"] == 0, f"failed bounds checks: bits {rec['bits']:#x}, first {rec['first']}"
    plain = _child(normal, str(tmp_path / "normal.npz"))
    assert plain["bits"] == 0
    a, b = np.load(tmp_path / "checked.npz"), np.load(tmp_path / "normal.npz")
    assert sorted(a.files) == sorted(b.files) and len(a.files) > 50
    for k in a.files:
        assert np.array_equal(a[k], b[k]), k
