"""3D GPU path (hexahedral Q1 RVEs, 21-point stencil, n_c up to 128 constraint rows) against
the FP64 oracle.

The oracle's sparse LU takes ~20 s per 32^3 point, so parity is element-by-element on RVE
grids up to 16^3 for whole hierarchies (one level with 4x4x4 periods, two levels (16/8) with
2x2x2 periods and three levels with eta = 1, all 16^3 with 2x2x2 periods and parents
interpolated on the same grid), and on two points of a one-level 32^3 workload with 4x4x4
periods.
Every grid keeps at least 4 elements per period so that the quarter-period channel contains
element centroids (with 2 elements per period the channel continuum is absent and the
solve reports MCH_ERR_DEGENERATE). The full-size workload (9^3 macropoints, grids 64/32/16) is checked by properties
that hold at any size, on sampled points of every level: the constraints C Phi = G,
stationarity (P_n^T A_1 Phi lies in the range of C_n^T, checked with the oracle's sparse
stiffness and constraint rows, independent of the solver's own residual), the effective
coefficients equal to the Gram of the cell functions on the level-1 grid, and a symmetric
positive definite E."""
import numpy as np
import pytest

import mch_inputs as mi
from oracle import cell, fe, plan
from util import block_rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2503_01276_gb300 as mch  # noqa: E402

NAME = "channel3d_9x9x9_L3"


def _run_gpu(wl, **kw):
    s = mch.Solver.from_workload(wl, **kw)
    out = []
    for lev in range(1, wl.n_levels + 1):
        pts = s.level_points(lev)
        kap, lab = mi.media(wl, pts, s.n_elem(lev))
        s.solve_level(lev, torch.from_numpy(kap).cuda(), torch.from_numpy(lab).cuda())
        out.append(s.effective_coeffs(lev))
    return s, out


def _run_oracle(wl):
    pl = plan.level_plan(wl)
    med = [mi.media(wl, l["points"], wl.n_level(k + 1)) for k, l in enumerate(pl)]
    return cell.run_hierarchy(wl, pl, med)


@pytest.mark.parametrize("n_fine,macro,strides,periods,eta", [
    (16, 3, (1,), 4, 2),
    (16, 3, (2, 1), 2, 2),
    (16, 5, (4, 2, 1), 2, 1),
])
@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_3d_hierarchy_small(n_fine, macro, strides, periods, eta, precision):
    wl = mi.small_workload(NAME, n_fine=n_fine, macro_n=macro, strides=strides,
                           periods=periods, eta=eta, precision=precision)
    s, Eg = _run_gpu(wl, rtol=1e-11)
    Eo = _run_oracle(wl)
    for lev in range(wl.n_levels):
        err = block_rel_err(Eg[lev], Eo[lev]["E"], wl.n_cont, wl.dim)
        assert err < 1e-9, (lev + 1, err)
        assert s.stats(lev + 1)["max_relres"] < 1e-11
    for lev in range(1, wl.n_levels + 1):
        phi = s.cell_functions(lev)
        ref = Eo[lev - 1]["Phi"]
        scale = np.abs(ref).max(axis=2, keepdims=True) + 1e-300
        assert (np.abs(phi - ref) / scale).max() < 1e-9, lev


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_3d_oversampling(precision):
    """R_p = the central 2x2x2 of the 4x4x4 periods (o = 1): centroids and E over R_p, every
    level of a two-level hierarchy (eta = 1, 16^3) against the oracle."""
    wl = mi.small_workload(NAME, n_fine=16, macro_n=3, strides=(2, 1), periods=4, eta=1,
                           overs=1, precision=precision)
    s, Eg = _run_gpu(wl, rtol=1e-11)
    Eo = _run_oracle(wl)
    for lev in range(wl.n_levels):
        err = block_rel_err(Eg[lev], Eo[lev]["E"], wl.n_cont, wl.dim)
        assert err < 1e-9, (lev + 1, err)


def test_3d_single_level_32_against_oracle():
    """One level, 3x3x3 macropoints on 32^3 RVEs with 4x4x4 periods (the size of the 9^3
    workload's second level): two points element by element against the oracle."""
    wl = mi.small_workload(NAME, n_fine=32, macro_n=3, strides=(1,), periods=4)
    s, Eg = _run_gpu(wl, rtol=1e-11)
    phi = s.cell_functions(1)
    pl = plan.level_plan(wl)
    ops = cell.LevelOps(wl, 1)
    for i in (0, 13):
        kap, lab = mi.media(wl, pl[0]["points"][[i]], 32)
        r = cell.solve_point(ops, kap[0], lab[0])
        err = block_rel_err(Eg[0][i], r["E"], wl.n_cont, wl.dim)
        assert err < 1e-9, (i, err)
        scale = np.abs(r["Phi"]).max(axis=1, keepdims=True) + 1e-300
        assert (np.abs(phi[i] - r["Phi"]) / scale).max() < 1e-9, i


def _stationarity(ops, kf, lf, wl, Phi):
    """M^-1-weighted size of the part of P^T A_1 Phi outside the range of C_n^T (the
    multipliers), relative to P^T A_1 Phi: zero at the constrained minimiser."""
    A1 = fe.stiffness_full(ops.gf, kf)
    C1 = fe.constraint_rows(ops.gf, lf, wl.n_cont, wl.periods)
    r = ops.P.T @ (A1 @ Phi)                         # [coarse interior, R]
    Cn = (C1 @ ops.P).toarray()
    keep = np.abs(Cn).sum(axis=1) > 0
    Cn = Cn[keep]
    An = (ops.P.T @ A1 @ ops.P).tocsr()
    minv = 1.0 / An.diagonal()
    beta = np.linalg.solve((Cn * minv) @ Cn.T, (Cn * minv) @ r)
    res = r - Cn.T @ beta
    num = np.sqrt(np.einsum("kr,k,kr->r", res, minv, res))
    den = np.sqrt(np.einsum("kr,k,kr->r", r, minv, r))
    return float((num / den).max())


def test_3d_full_size_properties():
    wl = mi.workload(NAME)
    s, Eg = _run_gpu(wl)
    pl = plan.level_plan(wl)
    gf = fe.Grid(3, wl.n_fine, wl.rve_len)
    vol = wl.rve_len ** 3
    ops = {lev: cell.LevelOps(wl, lev) for lev in range(1, wl.n_levels + 1)}
    for lev in range(1, wl.n_levels + 1):
        st = s.stats(lev)
        assert st["max_relres"] < 1e-8, (lev, st)
        E = Eg[lev - 1]
        sym = np.abs(E - E.transpose(0, 2, 1)).max() / np.abs(E).max()
        assert sym < 1e-12, (lev, sym)
        assert np.all(np.linalg.eigvalsh(0.5 * (E + E.transpose(0, 2, 1))) > 0)
        phi = s.cell_functions(lev)
        npts = len(pl[lev - 1]["points"])
        n = wl.n_level(lev)
        rho = wl.n_fine // n
        for i in sorted({0, npts - 1}):
            kap, lab = mi.media(wl, pl[lev - 1]["points"][[i]], n)
            kf = cell.prolong_medium(kap[0], 3, n, rho)
            lf = cell.prolong_medium(lab[0], 3, n, rho)
            C = fe.constraint_rows(gf, lf, wl.n_cont, wl.periods)
            G = fe.targets(gf, lf, wl.n_cont, wl.periods, 0)
            Phi = phi[i].T                                   # [nodes, R]
            cres = np.abs(C @ Phi - G).max() / np.abs(G).max()
            assert cres < 1e-9, (lev, i, cres)
            A1 = fe.stiffness_full(gf, kf)
            Eh = Phi.T @ (A1 @ Phi) / vol
            err = block_rel_err(E[i], Eh, wl.n_cont, wl.dim)
            assert err < 1e-8, (lev, i, err)
            stat = _stationarity(ops[lev], kf, lf, wl, Phi)
            assert stat < 1e-6, (lev, i, stat)
