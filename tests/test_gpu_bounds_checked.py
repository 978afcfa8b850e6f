"""The GPU parity suites rerun on the bounds-checked build of the library.

In that build (LBMH_CHECK_BOUNDS) every global-memory index the step kernels
form passes a guard: an index outside its array sets a status bit and is
clamped, never faulting.  lbmh_moments then fails with LBMH_ERR_BOUNDS, which
every parity test would see.  The suites run in a child process with
LBMH_LIBRARY=checked (ragged grids, every boundary kind, 1D, 2D and 3D,
slabs), and a batch of uneven lattices is stepped there with its status bits
checked.  No compute-sanitizer is involved: this is how index arithmetic is
checked on a GPU without a memory fault.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
pytestmark = pytest.mark.gpu

BATCH_CHECK = r"""
import numpy as np
from paper_2609_18177_b300 import lbmh
from paper_2609_18177_b300 import workloads as W
assert 'bounds-checked' in lbmh.version(), lbmh.version()
cases = [W.dam_break_bump(n) for n in (37, 64, 130, 251)]
cap = sum(lbmh.Batch.footprint(pb, lbmh.FP32) for pb, _ in cases) + (8 << 20)
b = lbmh.Batch(W.SWE, precision=lbmh.FP32, capacity_bytes=cap, max_instances=8)
slots = [b.add(pb.with_(precision=1), U0, max_steps=40) for pb, U0 in cases]
b.autotune(steps_per_candidate=1)
b.step(45)
done, t, steps, status = b.poll()
assert all(int(status[s]) & 16 == 0 for s in slots), [int(status[s]) for s in slots]
b.close()
print('batch ok')
"""


def _child(args):
    env = dict(os.environ, LBMH_LIBRARY="checked")
    return subprocess.run([sys.executable, *args], cwd=ROOT, env=env, capture_output=True, text=True, timeout=1200)


def test_parity_suites_pass_on_the_bounds_checked_build():
    from paper_2609_18177_b300 import build as B
    assert os.path.exists(B.LIB_CHECKED), "bounds-checked library not built"
    r = _child(["-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider",
                "tests/test_gpu_parity.py", "tests/test_gpu_boundaries.py", "tests/test_gpu_3d.py",
                "tests/test_gpu_slab.py"])
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]


def test_batch_of_uneven_lattices_on_the_bounds_checked_build():
    r = _child(["-c", BATCH_CHECK])
    assert r.returncode == 0 and "batch ok" in r.stdout, r.stdout[-2000:] + r.stderr[-2000:]
