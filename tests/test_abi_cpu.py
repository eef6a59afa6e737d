"""Host-side checks of the C-ABI library: it loads without a GPU, exports every function
declared in include/mch.h, validates descriptors before touching the device, and its host
level planner agrees bit for bit with the oracle's (Eq. defi_Sn and the multilinear parent
weights)."""
import ctypes
import os
import re

import numpy as np
import pytest

import mch_inputs as mi
from oracle import plan

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def mch():
    from paper_2503_01276_gb300 import build as b
    b.build()
    import paper_2503_01276_gb300 as m
    return m


def _declared():
    src = open(os.path.join(ROOT, "include", "mch.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mch_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(mch):
    lib = ctypes.CDLL(mch.LIB_PATH)
    names = _declared()
    assert "mch_solve_level" in names and "mch_backward" in names
    for nm in names:
        assert hasattr(lib, nm), nm


@pytest.mark.parametrize("interp", ["multilinear", "nearest1"])
@pytest.mark.parametrize("name", ["channel2d_4x4_n32", "channel2d_17x17_L3", "incl2d_33x33_L4",
                                  "channel3d_9x9x9_L3", "channel2d_65x65_L3_adj"])
def test_host_plan_matches_oracle(mch, name, interp):
    wl = mi.workload(name, interp=interp)
    d = mch.desc_from_workload(wl)
    pl = plan.level_plan(wl)
    for lev in range(1, wl.n_levels + 1):
        idx, pL, pP, w = mch.plan_level(d, lev)
        assert np.array_equal(idx, pl[lev - 1]["points"])
        for i, par in enumerate(pl[lev - 1]["parents"]):
            got = sorted((int(a), int(b), float(c)) for a, b, c in zip(pL[i], pP[i], w[i]) if a > 0)
            assert got == sorted(par)


def test_descriptor_validation_without_gpu(mch):
    wl = mi.workload("channel2d_17x17_L3")
    lib = mch._mch._LIB
    h = ctypes.c_void_p()
    bad = mch.desc_from_workload(wl, strides=(8, 3, 1))
    assert lib.mch_create(ctypes.byref(bad), None, ctypes.byref(h)) == 1
    bad = mch.desc_from_workload(wl, n_cont=7)
    assert lib.mch_create(ctypes.byref(bad), None, ctypes.byref(h)) == 1
    # 3D: up to three continua (12 cell functions); grids with at least 2 elements per period
    d3 = mch.desc_from_workload(mi.workload("channel3d_9x9x9_L3"), n_cont=4, periods=2)
    assert lib.mch_create(ctypes.byref(d3), None, ctypes.byref(h)) == 8
    d3 = mch.desc_from_workload(mi.workload("channel3d_9x9x9_L3"), periods=16)
    assert lib.mch_create(ctypes.byref(d3), None, ctypes.byref(h)) == 8
    bad = mch.desc_from_workload(wl, point_batch=-1)
    assert lib.mch_create(ctypes.byref(bad), None, ctypes.byref(h)) == 1
    ov = mch.desc_from_workload(wl, overs=2)          # no period left in R_p (P = 4)
    assert lib.mch_create(ctypes.byref(ov), None, ctypes.byref(h)) == 1
    ov = mch.desc_from_workload(mi.workload("channel3d_9x9x9_L3"), overs=2)   # 3D, none left
    assert lib.mch_create(ctypes.byref(ov), None, ctypes.byref(h)) == 1
    # 3 sub-blocks per side do not divide the 128-element grid: refused, not mis-solved
    # (grids 96 / 48 / 24 with 3 sub-blocks run; the kernels need a power-of-two number of
    # elements per sub-block)
    ov = mch.desc_from_workload(wl, periods=3, overs=1)
    assert lib.mch_create(ctypes.byref(ov), None, ctypes.byref(h)) == 8
    assert not h.value
    assert lib.mch_status_name(4) == b"MCH_ERR_ORDER"


def test_header_is_plain_c(tmp_path):
    """include/mch.h is a C interface: it compiles as strict C99 with no warnings."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    src = tmp_path / "use_header.c"
    src.write_text('#include "mch.h"\nint main(void) { return mch_status_name(0) == 0; }\n')
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                        "-fsyntax-only", "-I", inc, str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr

