"""Hierarchical (HMH) against direct (MH) effective coefficients on the 17x17 channel
workload: every macropoint solved directly on the 128x128 RVE grid versus the three-level
hierarchy (grids 128/64/32) with multilinear interpolation and with the single nearest S_1
parent. The block-relative difference per level is the error of the hierarchical
approximation on these media (the analogue of the paper's Type-3 comparison, which it
reports for the macroscopic solutions of its own media); it is printed, and level 1 (solved
identically by both) must agree to the solver tolerance."""
import numpy as np
import pytest

import mch_inputs as mi
from util import block_rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2503_01276_gb300 as mch  # noqa: E402


def _solve(wl):
    s = mch.Solver.from_workload(wl)
    out = {}
    for lev in range(1, wl.n_levels + 1):
        pts = s.level_points(lev)
        k, l = mi.media(wl, pts, s.n_elem(lev))
        s.solve_level(lev, torch.from_numpy(k).cuda(), torch.from_numpy(l).cuda())
        E = s.effective_coeffs(lev)
        for p, e in zip(pts, E):
            out[tuple(int(v) for v in p)] = (lev, e)
    s.close()
    return out


def test_hmh_vs_direct_report():
    base = mi.workload("channel2d_17x17_L3")
    direct = _solve(mi.workload("channel2d_17x17_L3", strides=(1,), n_levels=1))
    lines = []
    for interp in ("multilinear", "nearest1"):
        hmh = _solve(mi.workload("channel2d_17x17_L3", interp=interp))
        for lev in range(1, base.n_levels + 1):
            errs = [block_rel_err(e, direct[p][1], base.n_cont, base.dim)
                    for p, (lv, e) in hmh.items() if lv == lev]
            lines.append(f"{interp:11s} level {lev} ({len(errs)} points, grid "
                         f"{base.n_level(lev)}): block-rel diff vs direct max {max(errs):.3e} "
                         f"median {float(np.median(errs)):.3e}")
            if lev == 1:
                assert max(errs) < 1e-6
            assert np.isfinite(max(errs))
    print("\n" + "\n".join(lines))
