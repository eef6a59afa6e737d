"""The allocation-free single-level entry point (mch_direct_noalloc) against the regular
path (mch_create / mch_solve_level / mch_effective_coeffs) on the same media.

Kept in a file that pytest collects last: the entry point's fixed device buffer is shared
by every call, and this test must pass both on its own in a fresh process and after the
rest of the suite. It calls the entry point twice in a row (the buffer then holds the first
call's data) and checks both results.
"""
import ctypes

import numpy as np
import pytest

import mch_inputs as mi
from util import block_rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2503_01276_gb300 as mch  # noqa: E402


@pytest.mark.parametrize("n,macro", [(32, 4), (64, 3)])
def test_direct_noalloc_matches_regular_path(n, macro):
    wl = mi.small_workload("channel2d_17x17_L3", n_fine=n, macro_n=macro, strides=(1,))
    ref_solver = mch.Solver.from_workload(wl, rtol=1e-11)
    pts = ref_solver.level_points(1)
    kap, lab = mi.media(wl, pts, n)
    k_d = torch.from_numpy(kap).cuda()
    l_d = torch.from_numpy(lab).cuda()
    ref_solver.solve_level(1, k_d, l_d)
    E_ref = ref_solver.effective_coeffs(1)
    ref_solver.close()

    R = wl.n_rhs
    for call in range(2):
        E = torch.full((len(pts), R, R), float("nan"), dtype=torch.float64, device="cuda")
        st = mch.direct_noalloc(wl.n_cont, n, wl.periods, wl.rve_len, k_d, l_d, E, rtol=1e-11)
        assert st == 0, mch._mch.STATUS.get(st, st)
        err = block_rel_err(E.cpu().numpy(), E_ref, wl.n_cont, wl.dim)
        assert err < 1e-10, (call, err)


def test_direct_noalloc_rejects_oversized_batch():
    lib = mch._mch._LIB
    # 4096 points of a 64x64 grid need far more than the fixed buffer; rejected before any
    # device work, so the pointers are never touched
    dummy = ctypes.c_void_p(16)
    st = lib.mch_direct_noalloc(2, 64, 4, 0.0625, 1, 0.0, 4096, dummy, dummy, dummy, None)
    assert mch._mch.STATUS[st] == "MCH_ERR_OOM"
