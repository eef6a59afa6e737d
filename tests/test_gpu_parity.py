"""GPU parity: the sm_103a library through its C ABI against the FP64 oracle.

Tolerances. A level's effective coefficients are stationary in its own cell functions
(quadratic error) but depend linearly on its parents' functions, so the refinement
tolerance rtol on the projected residual sets the accuracy of every child level. With
rtol = 1e-11 both the FP64 mode and the mixed mode (FP32 PCG inside FP64 refinement) are
asserted at a block-relative error of 1e-9 on every level; with the default rtol = 1e-8
(the benchmark setting) the bound asserted is 1e-6.
"""
import numpy as np
import pytest

import mch_inputs as mi
from oracle import cell, plan
from util import block_rel_err, entry_rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2503_01276_gb300 as mch  # noqa: E402


def _run_gpu(wl, levels=None, device=True, **kw):
    s = mch.Solver.from_workload(wl, **kw)
    out = []
    L = wl.n_levels if levels is None else levels
    for lev in range(1, L + 1):
        pts = s.level_points(lev)
        kap, lab = mi.media(wl, pts, s.n_elem(lev))
        if device:
            k_t = torch.from_numpy(kap).cuda()
            l_t = torch.from_numpy(lab).cuda()
            s.solve_level(lev, k_t, l_t)
            E = torch.zeros((len(pts), s.R, s.R), dtype=torch.float64, device="cuda")
            s.effective_coeffs(lev, E)
            out.append(E.cpu().numpy())
        else:
            s.solve_level(lev, kap, lab)
            out.append(s.effective_coeffs(lev))
    return s, out


def _run_oracle(wl):
    pl = plan.level_plan(wl)
    med = [mi.media(wl, l["points"], wl.n_level(k + 1)) for k, l in enumerate(pl)]
    return cell.run_hierarchy(wl, pl, med)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("mixed", 1e-9)])
def test_level1_4x4_n32(precision, tol):
    """2D, L = 1, 4x4 macropoints, 32x32 RVEs, two continua (full size of this workload)."""
    wl = mi.workload("channel2d_4x4_n32", precision=precision)
    s, Eg = _run_gpu(wl, rtol=1e-11)
    Eo = _run_oracle(wl)
    err = block_rel_err(Eg[0], Eo[0]["E"], wl.n_cont, wl.dim)
    assert err < tol, err
    # every entry on its own, against its Cauchy-Schwarz scale
    assert entry_rel_err(Eg[0], Eo[0]["E"]) < tol


@pytest.mark.parametrize("name,n_fine,macro,strides", [
    ("channel2d_17x17_L3", 64, 5, (4, 2, 1)),
    ("channel2d_17x17_L3", 64, 9, (4, 2, 1)),
    ("incl2d_33x33_L4", 128, 5, (4, 2, 1)),
    ("channel2d_65x65_L3_adj", 64, 5, (2, 1)),
])
@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_hierarchy_small(name, n_fine, macro, strides, precision):
    wl = mi.small_workload(name, n_fine=n_fine, macro_n=macro, strides=strides,
                           precision=precision)
    s, Eg = _run_gpu(wl, rtol=1e-11)
    Eo = _run_oracle(wl)
    for lev in range(wl.n_levels):
        err = block_rel_err(Eg[lev], Eo[lev]["E"], wl.n_cont, wl.dim)
        assert err < 1e-9, (lev + 1, err)
        # every entry on its own, against its Cauchy-Schwarz scale
        err_e = entry_rel_err(Eg[lev], Eo[lev]["E"])
        assert err_e < 1e-9, (lev + 1, err_e)
    # the cell functions on the level-1 grid
    for lev in range(1, wl.n_levels + 1):
        phi = s.cell_functions(lev)
        ref = Eo[lev - 1]["Phi"]
        scale = np.abs(ref).max(axis=2, keepdims=True) + 1e-300
        assert (np.abs(phi - ref) / scale).max() < 1e-9, lev


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_hierarchy_nearest_s1(precision):
    """The single-parent interpolation variant (nearest point of S_1, weight one)."""
    wl = mi.small_workload("channel2d_17x17_L3", n_fine=64, macro_n=9, strides=(4, 2, 1),
                           precision=precision, interp="nearest1")
    s, Eg = _run_gpu(wl, rtol=1e-11)
    Eo = _run_oracle(wl)
    for lev in range(wl.n_levels):
        err = block_rel_err(Eg[lev], Eo[lev]["E"], wl.n_cont, wl.dim)
        assert err < 1e-9, (lev + 1, err)


@pytest.mark.parametrize("name,n_fine,macro,strides", [
    ("channel2d_4x4_n32", 32, None, None),
    ("channel2d_17x17_L3", 64, 5, (4, 2, 1)),
])
@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_oversampling(name, n_fine, macro, strides, precision):
    """R_p = the central 2x2 of the 4x4 periods (o = 1): centroids and E over R_p."""
    if macro is None:
        wl = mi.workload(name, precision=precision, overs=1)
    else:
        wl = mi.small_workload(name, n_fine=n_fine, macro_n=macro, strides=strides,
                               precision=precision, overs=1)
    s, Eg = _run_gpu(wl, rtol=1e-11)
    Eo = _run_oracle(wl)
    for lev in range(wl.n_levels):
        err = block_rel_err(Eg[lev], Eo[lev]["E"], wl.n_cont, wl.dim)
        assert err < 1e-9, (lev + 1, err)


def test_host_buffers_match_device_buffers():
    """Host and device buffers give the same answer. Shared-memory reductions use atomics,
    so two runs agree to the solver tolerance rather than bit for bit."""
    wl = mi.small_workload("channel2d_17x17_L3", n_fine=32, macro_n=5, strides=(2, 1))
    _, Ed = _run_gpu(wl, device=True, rtol=1e-11)
    s, Eh = _run_gpu(wl, device=False, rtol=1e-11)
    for a, b in zip(Ed, Eh):
        assert block_rel_err(a, b, wl.n_cont, wl.dim) < 1e-10
    st = s.stats(2)
    assert st["h2d_bytes"] > 0


@pytest.mark.parametrize("point_batch", [1, 7])
def test_point_batch_matches_whole_level(point_batch):
    """Solving a level in chunks of point_batch points per launch (1 = the unbatched
    per-macropoint solve) gives the same coefficients as one launch for the level."""
    wl = mi.small_workload("channel2d_17x17_L3", n_fine=64, macro_n=5, strides=(4, 2, 1),
                           precision="fp64")
    _, Ea = _run_gpu(wl, rtol=1e-11)
    s, Eb = _run_gpu(wl, rtol=1e-11, point_batch=point_batch)
    for a, b in zip(Ea, Eb):
        assert block_rel_err(a, b, wl.n_cont, wl.dim) < 1e-10
    np_l = [s.num_points(l) for l in range(1, wl.n_levels + 1)]
    assert [s.stats(l)["pcg_launches"] for l in range(1, wl.n_levels + 1)] == \
        [-(-n // point_batch) for n in np_l]


def test_prepared_levels_match_plain_solve():
    """mch_prepare_level for every level up front (setup on the side stream, overlapping the
    earlier levels' solves) gives the plain solve's coefficients; a solve with other buffers
    than the prepared ones ignores the preparation."""
    wl = mi.small_workload("channel2d_17x17_L3", n_fine=64, macro_n=9, strides=(4, 2, 1))
    _, ref = _run_gpu(wl, rtol=1e-11)
    s = mch.Solver.from_workload(wl, rtol=1e-11)
    med = []
    for lev in range(1, wl.n_levels + 1):
        k, l = mi.media(wl, s.level_points(lev), s.n_elem(lev))
        med.append((torch.from_numpy(k).cuda(), torch.from_numpy(l).cuda()))
    for lev, (k, l) in enumerate(med, start=1):
        s.prepare_level(lev, k, l)
    for lev, (k, l) in enumerate(med, start=1):
        s.solve_level(lev, k, l)
        assert block_rel_err(s.effective_coeffs(lev), ref[lev - 1], wl.n_cont, wl.dim) < 1e-10
    # prepared with a scaled copy, solved with the original: the original is used
    k2 = med[0][0] * 3.0
    s.prepare_level(1, k2, med[0][1])
    s.solve_level(1, *med[0])
    assert block_rel_err(s.effective_coeffs(1), ref[0], wl.n_cont, wl.dim) < 1e-10


def test_full_size_17x17_sampled():
    """The benchmark workload (17x17 points, RVE grids 128/64/32, mixed precision) solved in
    full on the GPU; sampled points of every level checked against the oracle, which
    computes them (and their ancestors) one by one."""
    wl = mi.workload("channel2d_17x17_L3")
    s, Eg = _run_gpu(wl)
    pl = plan.level_plan(wl)
    targets = [(1, 0), (1, 4), (2, 0), (2, 37), (3, 0), (3, 101), (3, 207)]

    def media_fn(lv, pos):
        return mi.media(wl, pl[lv - 1]["points"][pos], wl.n_level(lv))

    ref = cell.run_sampled(wl, pl, media_fn, targets)
    for (lv, i) in targets:
        err = block_rel_err(Eg[lv - 1][i], ref[(lv, i)]["E"], wl.n_cont, wl.dim)
        assert err < 1e-6, (lv, i, err)
    for lev in (1, 2, 3):
        st = s.stats(lev)
        assert st["max_relres"] < 1e-8


def test_full_size_33x33_three_continua_sampled():
    """Four levels (25/56/208/800 points on RVE grids 256/128/64/32), three continua
    (channels at contrast 1e6, lognormal inclusions, matrix), nine cell functions per
    point, mixed precision at the default tolerance: sampled points of every level, including
    points with two and with four parents, against the oracle."""
    wl = mi.workload("incl2d_33x33_L4")
    s, Eg = _run_gpu(wl)
    pl = plan.level_plan(wl)
    targets = [(1, 12), (2, 30)]
    for lv in (3, 4):
        par = pl[lv - 1]["parents"]
        two = next(i for i in range(len(par)) if len(par[i]) == 2)
        four = next(i for i in range(len(par) - 1, -1, -1) if len(par[i]) == 4)
        targets += [(lv, two), (lv, four)]

    def media_fn(lv, pos):
        return mi.media(wl, pl[lv - 1]["points"][pos], wl.n_level(lv))

    ref = cell.run_sampled(wl, pl, media_fn, targets)
    for (lv, i) in targets:
        err = block_rel_err(Eg[lv - 1][i], ref[(lv, i)]["E"], wl.n_cont, wl.dim)
        assert err < 1e-6, (lv, i, err)
    for lev in range(1, 5):
        assert s.stats(lev)["max_relres"] < 1e-8


def test_level_order_error():
    wl = mi.small_workload("channel2d_17x17_L3", n_fine=32, macro_n=5, strides=(2, 1))
    s = mch.Solver.from_workload(wl)
    pts = s.level_points(2)
    kap, lab = mi.media(wl, pts, s.n_elem(2))
    with pytest.raises(mch.MchError) as e:
        s.solve_level(2, kap, lab)
    assert e.value.name == "MCH_ERR_ORDER"


def test_invalid_medium_reported():
    wl = mi.small_workload("channel2d_17x17_L3", n_fine=32, macro_n=3, strides=(1,))
    s = mch.Solver.from_workload(wl)
    pts = s.level_points(1)
    kap, lab = mi.media(wl, pts, 32)
    kap[1, 5] = -1.0
    with pytest.raises(mch.MchError) as e:
        s.solve_level(1, kap, lab)
    assert e.value.name == "MCH_ERR_DEGENERATE"
    kap, lab = mi.media(wl, pts, 32)
    lab[:] = 1   # continuum 0 absent everywhere
    with pytest.raises(mch.MchError) as e:
        s.solve_level(1, kap, lab)
    assert e.value.name == "MCH_ERR_DEGENERATE"


def _coarse_block_workload(n_fine, macro, strides, precision, mp=6):
    """Sec. 2 and Sec. 5: R_p^+ = the coarse block K_p with l = 1 layer of neighbouring
    blocks, so the constraint sub-blocks R_q are 3 x 3 coarse blocks (P = 3, odd), R_p = K_p
    (o = 1), and the medium's period (mp per RVE side) differs from the blocks."""
    wl = mi.small_workload("channel2d_17x17_L3", n_fine=n_fine, macro_n=macro, strides=strides)
    return mi.small_workload("channel2d_17x17_L3", n_fine=n_fine, macro_n=macro,
                             strides=strides, periods=3, overs=1, medium_periods=mp,
                             rve_len=3 * wl.spacing, precision=precision)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_coarse_blocks_odd_P_single_level(precision):
    """The configuration pinned against the dense brute force in the oracle pins (48 x 48
    RVE, 3 x 3 coarse blocks, o = 1, six medium periods per side), every point of a 3 x 3
    macrogrid: E and the cell functions against the oracle."""
    wl = _coarse_block_workload(48, 3, (1,), precision)
    s, Eg = _run_gpu(wl, rtol=1e-11)
    Eo = _run_oracle(wl)
    err = block_rel_err(Eg[0], Eo[0]["E"], wl.n_cont, wl.dim)
    assert err < 1e-9, err
    phi = s.cell_functions(1)
    ref = Eo[0]["Phi"]
    scale = np.abs(ref).max(axis=2, keepdims=True) + 1e-300
    assert (np.abs(phi - ref) / scale).max() < 1e-9


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_coarse_blocks_odd_P_hierarchy(precision):
    """Three levels (RVE grids 96 / 48 / 24) with 3 x 3 coarse blocks and o = 1 on a 5 x 5
    macrogrid: every level against the oracle."""
    wl = _coarse_block_workload(96, 5, (4, 2, 1), precision)
    s, Eg = _run_gpu(wl, rtol=1e-11)
    Eo = _run_oracle(wl)
    for lev in range(wl.n_levels):
        err = block_rel_err(Eg[lev], Eo[lev]["E"], wl.n_cont, wl.dim)
        assert err < 1e-9, (lev + 1, err)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_inputs_are_read_only(precision):
    """The library reads the caller's media and loss weights and never writes them: after a
    forward pass over every level and a backward pass, the device buffers are bit-identical
    to the host originals."""
    wl = mi.small_workload("channel2d_17x17_L3", n_fine=128, macro_n=5, strides=(4, 2, 1),
                           precision=precision)
    s = mch.Solver.from_workload(wl, rtol=1e-11)
    host, dev = [], []
    for lev in range(1, wl.n_levels + 1):
        k, l = mi.media(wl, s.level_points(lev), s.n_elem(lev))
        host.append((k, l))
        dev.append((torch.from_numpy(k).cuda(), torch.from_numpy(l).cuda()))
        s.solve_level(lev, *dev[-1])
    rng = np.random.default_rng(3)
    W = [rng.standard_normal((s.num_points(l), s.R, s.R)) for l in range(1, wl.n_levels + 1)]
    Wd = [torch.from_numpy(w).cuda() for w in W]
    G = [torch.zeros((s.num_points(l), s.n_elem(l) ** 2), dtype=torch.float64, device="cuda")
         for l in range(1, wl.n_levels + 1)]
    s.backward(Wd, G)
    torch.cuda.synchronize()
    for (k, l), (kd, ld) in zip(host, dev):
        assert np.array_equal(kd.cpu().numpy(), k)
        assert np.array_equal(ld.cpu().numpy(), l)
    for w, wd in zip(W, Wd):
        assert np.array_equal(wd.cpu().numpy(), w)
    s.close()
