"""The allocation-free single-level entry point (mch_direct_noalloc) against the regular
path (mch_create / mch_solve_level / mch_effective_coeffs) and against the FP64 oracle.

Some callers cannot allocate device memory when they need a result (their memory is held
by another framework's caching allocator, or fixed at start-up); this entry point keeps
every intermediate in one fixed buffer compiled into the library. Kept in a file that pytest
collects last: the buffer is shared by every call, and this test must pass both on its own
in a fresh process and after the rest of the suite. Two calls in a row use different media
and batch sizes on the same grid, so data left in the buffer by the first call is not the
second call's answer; the free device memory is unchanged across the second call.
"""
import ctypes
from dataclasses import replace

import numpy as np
import pytest

import mch_inputs as mi
from oracle import cell, plan
from util import block_rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2503_01276_gb300 as mch  # noqa: E402


def _oracle_E(wl, pts):
    med = mi.media(wl, pts, wl.n_fine)
    pl = [{"points": pts, "parents": [[] for _ in range(len(pts))]}]
    return cell.run_hierarchy(wl, pl, [med], keep_phi=False)[0]["E"]


@pytest.mark.parametrize("n,macro", [(32, 4), (64, 3)])
def test_direct_noalloc_matches_regular_path_and_oracle(n, macro):
    wl = mi.small_workload("channel2d_17x17_L3", n_fine=n, macro_n=macro, strides=(1,),
                           precision="fp64")
    pts = plan.level_plan(wl)[0]["points"]
    # second call: another medium (seed and contrast) and a smaller batch on the same grid
    wl_b = replace(wl, seed=wl.seed + 17, contrast=1e3)
    pts_b = pts[: max(1, len(pts) // 2)]
    R = wl.n_rhs
    cases = []
    for w, p in ((wl, pts), (wl_b, pts_b)):
        kap, lab = mi.media(w, p, n)
        cases.append((w, p, torch.from_numpy(kap).cuda(), torch.from_numpy(lab).cuda()))

    # the regular path on the first medium
    ref_solver = mch.Solver.from_workload(wl, rtol=1e-11)
    ref_solver.solve_level(1, cases[0][2], cases[0][3])
    E_reg = ref_solver.effective_coeffs(1)
    ref_solver.close()

    for call, (w, p, k_d, l_d) in enumerate(cases):
        E = torch.full((len(p), R, R), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        st = mch.direct_noalloc(w.n_cont, n, w.periods, w.rve_len, k_d, l_d, E,
                                precision="fp64", rtol=1e-11)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        assert st == 0, mch._mch.STATUS.get(st, st)
        if call > 0:
            # the first call loaded the kernels and created the buffer; this one allocates
            # nothing
            assert free1 == free0, (free0, free1)
        Eg = E.cpu().numpy()
        err_or = block_rel_err(Eg, _oracle_E(w, p), w.n_cont, w.dim)
        assert err_or < 1e-9, (call, err_or)
        if call == 0:
            err_reg = block_rel_err(Eg, E_reg, w.n_cont, w.dim)
            assert err_reg < 1e-10, (call, err_reg)

    # mixed precision on the first medium against the regular mixed path
    ref_mixed = mch.Solver.from_workload(wl, rtol=1e-11, precision="mixed")
    ref_mixed.solve_level(1, cases[0][2], cases[0][3])
    E_rm = ref_mixed.effective_coeffs(1)
    ref_mixed.close()
    E = torch.full((len(pts), R, R), float("nan"), dtype=torch.float64, device="cuda")
    st = mch.direct_noalloc(wl.n_cont, n, wl.periods, wl.rve_len, cases[0][2], cases[0][3], E,
                            precision="mixed", rtol=1e-11)
    assert st == 0, mch._mch.STATUS.get(st, st)
    assert block_rel_err(E.cpu().numpy(), E_rm, wl.n_cont, wl.dim) < 1e-10


def test_direct_noalloc_rejects_oversized_batch():
    lib = mch._mch._LIB
    # 4096 points of a 64x64 grid need far more than the fixed buffer; rejected before any
    # device work, so the pointers are never touched
    dummy = ctypes.c_void_p(16)
    st = lib.mch_direct_noalloc(2, 64, 4, 0.0625, 1, 0.0, 4096, dummy, dummy, dummy, None)
    assert mch._mch.STATUS[st] == "MCH_ERR_OOM"
