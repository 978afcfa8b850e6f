"""The C ABI library loads, exports every entry point include/lbmh.h declares,
and the ctypes mirrors of its structs match the C layout.  No GPU needed: only
argument validation (which fails before any CUDA call) is exercised."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2609_18177_b300 import build as B
from paper_2609_18177_b300 import lbmh
from paper_2609_18177_b300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbmh.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return lbmh.load()


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"LBMH_API\s+[\w\s\*]+?\b(lbmh_\w+)\s*\(", text)))


def exported_symbols(path):
    out = subprocess.check_output(["nm", "-D", "--defined-only", path], text=True)
    return {line.split()[-1] for line in out.splitlines() if " T " in line}


def test_every_declared_function_is_exported(lib):
    decl = declared_functions()
    assert len(decl) >= 12
    exported = exported_symbols(lbmh.LIB_PATH)
    missing = [f for f in decl if f not in exported]
    assert not missing, missing
    for f in decl:
        assert hasattr(lib, f)
    # the binding covers the whole ABI
    assert sorted(n for n, _r, _a in lbmh.SIGNATURES) == decl


def test_struct_layout_matches_header():
    src = r'''
#include <stddef.h>
#include <stdio.h>
#include "lbmh.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(lbmh_problem), offsetof(lbmh_problem, A),
         offsetof(lbmh_problem, cuda_stream), offsetof(lbmh_problem, sponge_width),
         offsetof(lbmh_problem, u_in), offsetof(lbmh_problem, nz), offsetof(lbmh_problem, adv_z),
         sizeof(lbmh_info), offsetof(lbmh_info, status), offsetof(lbmh_info, device_bytes),
         offsetof(lbmh_info, abar_z));
  return 0;
}
'''
    d = os.path.join(ROOT, "_build", "abi_check")  # git-ignored build folder
    os.makedirs(d, exist_ok=True)
    c = os.path.join(d, "t.c")
    exe = os.path.join(d, "t")
    with open(c, "w") as fh:
        fh.write(src)
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", exe, c])
    vals = [int(v) for v in subprocess.check_output([exe], text=True).split()]
    P, I = lbmh._Problem, lbmh.Info
    assert vals == [ctypes.sizeof(P), P.A.offset, P.cuda_stream.offset, P.sponge_width.offset, P.u_in.offset,
                    P.nz.offset, P.adv_z.offset, ctypes.sizeof(I), I.status.offset, I.device_bytes.offset,
                    I.abar_z.offset]


def _create(lib, pb, **kw):
    s = lbmh._c_problem(pb, kw.get("precision", 0), kw.get("kernel", 0), None)
    h = ctypes.c_void_p()
    rc = lib.lbmh_create(ctypes.byref(s), ctypes.byref(h))
    return rc, h, lib.lbmh_last_error(None).decode()


@pytest.mark.parametrize("bad,code", [
    (dict(dim=3), lbmh.ERR_INVALID_ARG),
    (dict(nx=0), lbmh.ERR_INVALID_ARG),
    (dict(bc=(0, 1, 0, 0)), lbmh.ERR_INVALID_ARG),
    (dict(cfl=0.0), lbmh.ERR_INVALID_ARG),
    (dict(system=W.LINEAR, m_linear=2), lbmh.ERR_UNSUPPORTED),
    (dict(dim=2, nx=10, ny=10, y1=2.0), lbmh.ERR_INVALID_ARG),  # dx != dy
    (dict(gamma=1.0), lbmh.ERR_INVALID_ARG),
    (dict(dim=4), lbmh.ERR_INVALID_ARG),
    (dict(system=W.SWE, dim=3, nx=8, ny=8, nz=8), lbmh.ERR_UNSUPPORTED),         # 3D: no shallow water
    (dict(dim=3, nx=8, ny=8, nz=8, bc=(W.REFLECT, W.REFLECT, 0, 0)), lbmh.ERR_UNSUPPORTED),
    (dict(dim=3, nx=8, ny=8, nz=8, z1=2.0), lbmh.ERR_INVALID_ARG),               # dz != dx
    (dict(nx=3, bc=(W.REFLECT, W.OUTFLOW, 0, 0)), lbmh.ERR_INVALID_ARG),         # < 4 nodes across
    (dict(bc=(W.OUTFLOW, W.INFLOW, 0, 0), u_in=(0.0, 0.0, 0.0)), lbmh.ERR_INVALID_ARG),  # not physical
    (dict(sponge_width=2.0), lbmh.ERR_INVALID_ARG),                                # wider than the domain
    (dict(bc=(4, 4, 0, 0)), lbmh.ERR_INVALID_ARG),
])
def test_create_rejects_invalid_problems_before_touching_the_device(lib, bad, code):
    pb = W.Problem(system=W.EULER, dim=1, nx=16).with_(**bad)
    rc, h, msg = _create(lib, pb)
    assert rc == code and not h.value and msg


def test_null_arguments(lib):
    assert lib.lbmh_create(None, None) == lbmh.ERR_INVALID_ARG
    assert lib.lbmh_step(None, 1) == lbmh.ERR_INVALID_ARG
    assert lib.lbmh_destroy(None) == lbmh.OK
    assert lib.lbmh_version().decode().startswith("lbmh")


@pytest.mark.parametrize("shape", [(5, 4, 29, 66), (5, 4, 29 * 67), (3, 4, 29, 67)])
def test_step_static_rejects_wrong_shapes_before_any_launch(shape):
    """The C entry point cannot see array sizes, so the binding refuses arrays
    that are not exactly [Q][m][ny][nx] of the problem before it reaches the
    library (here on the CPU, where no launch could happen at all)."""
    import torch
    pb = W.Problem(system=W.EULER, dim=2, nx=67, ny=29, y1=29 / 67)
    good = torch.zeros((5, 4, 29, 67), dtype=torch.float64)
    bad = torch.zeros(shape, dtype=torch.float64)
    with pytest.raises(TypeError, match="shape"):
        lbmh.step_static(pb, bad, good)
    with pytest.raises(TypeError, match="shape"):
        lbmh.step_static(pb, good, bad)
    with pytest.raises(TypeError, match="CUDA"):  # right shape, but host memory
        lbmh.step_static(pb, good, good.clone())
