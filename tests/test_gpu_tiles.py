"""Launch shapes of the 2D level solve (mixed precision and FP64) and the autotuner.

Every valid shape of every grid size (16 to 256) must give the default shape's effective
coefficients (to the solver tolerance: rtol = 1e-11, compared at 1e-10), and the default
shapes are checked against the oracle by the parity tests; the autotuner must keep results
unchanged, record its choices in the cache file and reuse them."""
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

CASES = [("channel2d_17x17_L3", 128, 5, (4, 2, 1)), ("channel2d_17x17_L3", 32, 5, (2, 1))]
SHAPE_CASES = [(name, n, m, st, "mixed") for (name, n, m, st) in CASES] + [
    ("incl2d_33x33_L4", 256, 3, (1,), "mixed"),
    ("channel2d_17x17_L3", 128, 5, (4, 2, 1), "fp64"),
    ("channel2d_17x17_L3", 32, 5, (2, 1), "fp64")]


def _media(wl, s):
    out = []
    for lev in range(1, wl.n_levels + 1):
        k, l = mi.media(wl, s.level_points(lev), s.n_elem(lev))
        out.append((torch.from_numpy(k).cuda(), torch.from_numpy(l).cuda()))
    return out


def _solve(s, med, shapes=None):
    Es = []
    for lev, (k, l) in enumerate(med, start=1):
        if shapes is not None:
            s.set_variant(lev, shapes[lev - 1])
        s.solve_level(lev, k, l)
        Es.append(s.effective_coeffs(lev))
    return Es


@pytest.mark.parametrize("name,n_fine,macro,strides,precision", SHAPE_CASES)
def test_every_shape_matches_default(name, n_fine, macro, strides, precision):
    wl = mi.small_workload(name, n_fine=n_fine, macro_n=macro, strides=strides,
                           precision=precision)
    s = mch.Solver.from_workload(wl, rtol=1e-11)
    med = _media(wl, s)
    ref = _solve(s, med)
    # the default shape against the oracle, so that every shape is tied to it
    pl = plan.level_plan(wl)
    oref = cell.run_hierarchy(wl, pl, [mi.media(wl, l["points"], wl.n_level(k + 1))
                                       for k, l in enumerate(pl)], keep_phi=False)
    for lev in range(wl.n_levels):
        assert block_rel_err(ref[lev], oref[lev]["E"], wl.n_cont, wl.dim) < 1e-9, lev
    counts = [s.variant(lev)[1] for lev in range(1, wl.n_levels + 1)]
    tried = 0
    for v in range(1, max(counts)):
        shapes = []
        for lev in range(1, wl.n_levels + 1):
            ok = v < counts[lev - 1]
            if ok:
                try:
                    s.set_variant(lev, v)
                except mch.MchError:
                    ok = False
            shapes.append(v if ok else 0)
        tried += sum(1 for x in shapes if x)
        Es = _solve(s, med, shapes)
        for lev in range(wl.n_levels):
            err = block_rel_err(Es[lev], ref[lev], wl.n_cont, wl.dim)
            assert err < 1e-10, (v, lev + 1, shapes, err)
            err = block_rel_err(Es[lev], oref[lev]["E"], wl.n_cont, wl.dim)
            assert err < 1e-9, (v, lev + 1, shapes, err)
    assert tried > 0


def test_invalid_shape_rejected():
    wl = mi.small_workload("channel2d_17x17_L3", n_fine=32, macro_n=3, strides=(1,))
    s = mch.Solver.from_workload(wl)
    with pytest.raises(mch.MchError) as e:
        s.set_variant(1, 99)
    assert e.value.name == "MCH_ERR_UNSUPPORTED"


def test_autotune_and_cache(tmp_path, monkeypatch):
    name, n_fine, macro, strides = CASES[0]
    wl = mi.small_workload(name, n_fine=n_fine, macro_n=macro, strides=strides)
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("MCH_TUNE_CACHE", str(cache))
    s = mch.Solver.from_workload(wl, rtol=1e-11)
    med = _media(wl, s)
    ref = _solve(s, med)
    s2 = mch.Solver.from_workload(wl, rtol=1e-11)
    picks = []
    for lev, (k, l) in enumerate(med, start=1):
        v, ms = s2.autotune_level(lev, k, l)
        assert ms > 0.0
        picks.append(v)
        assert s2.variant(lev)[0] == v
        err = block_rel_err(s2.effective_coeffs(lev), ref[lev - 1], wl.n_cont, wl.dim)
        assert err < 1e-10, (lev, v, err)
    lines = cache.read_text().strip().splitlines()
    assert len(lines) == wl.n_levels
    s3 = mch.Solver.from_workload(wl, rtol=1e-11)
    for lev, (k, l) in enumerate(med, start=1):
        v, ms = s3.autotune_level(lev, k, l)
        assert (v, ms) == (picks[lev - 1], 0.0)
