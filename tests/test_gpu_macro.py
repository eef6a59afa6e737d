"""GPU parity of the macroscopic multicontinuum problem (Sec. 2, Eq. macro_eq) against the
oracle: the source densities of every level from the cell functions (Eq. Bs_defi, b_j, with
the Gaussian source of Sec. 5), their exact value for a source constant per continuum (the
constraints fix it), and the macro solve on the coarse blocks from the library's effective
coefficients. Tolerances: the cell functions agree with the oracle to ~1e-9 at rtol 1e-11, the
source densities are linear in them; the macro solve is run to a relative residual of 1e-13."""
import numpy as np
import pytest

import mch_inputs as mi
from oracle import cell, macro, plan

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2503_01276_gb300 as mch  # noqa: E402


def _weights(N):
    # Sec. 5: eta in the low-conductivity continuum, 1 in the high one (plus a third value)
    return np.array([1e-4, 1.0, 0.3, 0.5][:N])


def _gpu(wl, **kw):
    s = mch.Solver.from_workload(wl, **kw)
    E, med = [], []
    for lev in range(1, wl.n_levels + 1):
        pts = s.level_points(lev)
        kap, lab = mi.media(wl, pts, s.n_elem(lev))
        med.append((kap, lab))
        s.solve_level(lev, torch.from_numpy(kap).cuda(), torch.from_numpy(lab).cuda())
        E.append(s.effective_coeffs(lev))
    return s, E, med


def _oracle_sources(wl, phis, med, w, c, alpha):
    pl = plan.level_plan(wl)
    out = []
    for n, lev in enumerate(pl):
        xs = mi.macro_points_xyz(wl, lev["points"])
        out.append(np.array([macro.source_point(wl, n + 1, phis[n][i], med[n][1][i], xs[i], w, c,
                                                alpha, getattr(wl, "overs", 0))
                             for i in range(len(lev["points"]))]))
    return out


CASES = [
    ("channel2d_4x4_n32", dict(n_fine=32), "fp64"),   # one level; blocks tile the unit square
    ("channel2d_17x17_L3", dict(n_fine=64, macro_n=9, strides=(4, 2, 1)), "fp64"),
    ("channel2d_17x17_L3", dict(n_fine=64, macro_n=9, strides=(4, 2, 1)), "mixed"),
    ("channel2d_17x17_L3", dict(n_fine=64, macro_n=9, strides=(4, 2, 1), overs=1), "mixed"),
    ("incl2d_33x33_L4", dict(n_fine=128, macro_n=5, strides=(4, 2, 1)), "mixed"),
    ("channel3d_9x9x9_L3", dict(n_fine=16, macro_n=3, strides=(2, 1), periods=2), "mixed"),
]


@pytest.mark.parametrize("name,kw,precision", CASES)
def test_source_and_solve_match_oracle(name, kw, precision):
    wl = mi.small_workload(name, precision=precision, **kw)
    s, E, med = _gpu(wl, rtol=1e-11)
    pl = plan.level_plan(wl)
    o = cell.run_hierarchy(wl, pl, [mi.media(wl, l["points"], wl.n_level(k + 1))
                                    for k, l in enumerate(pl)])
    d, N = wl.dim, wl.n_cont
    w, c, alpha = _weights(N), np.full(d, 0.5), 40.0
    origin = np.full(d, wl.origin)
    fb = [s.macro_source(lev, w, c, alpha, origin, wl.spacing) for lev in range(1, wl.n_levels + 1)]
    ref = _oracle_sources(wl, [x["Phi"] for x in o], med, w, c, alpha)
    for lev in range(wl.n_levels):
        err = np.abs(fb[lev] - ref[lev]).max() / np.abs(ref[lev]).max()
        assert err < 1e-8, (lev + 1, err)
    # the solve: the same coefficients and sources through the library and the oracle
    U, iters, rr = s.macro_solve(E, fb, wl.spacing, tol=1e-13)
    assert rr <= 1e-13 and iters > 0
    Eg = macro.grid_from_levels(pl, wl.macro_n, d, E)
    fg = macro.grid_from_levels(pl, wl.macro_n, d, fb)
    Uo = macro.solve(wl.macro_n, d, wl.spacing, Eg, fg)
    # two solvers of one system: the difference is bounded by cond(A) times the residual
    err = np.abs(U - Uo).max() / np.abs(Uo).max()
    assert err < 1e-7, err


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_source_constant_per_continuum(precision):
    """alpha = 0: fbar_i = w_i times the volume fraction of continuum i in R_p, fixed by the
    constraints of Eqs. (phi_avar), on every level."""
    wl = mi.small_workload("channel2d_17x17_L3", n_fine=64, macro_n=9, strides=(4, 2, 1),
                           precision=precision)
    s, E, med = _gpu(wl, rtol=1e-11)
    w = np.array([0.25, 1.5])
    for lev in range(1, wl.n_levels + 1):
        fb = s.macro_source(lev, w, np.full(2, 0.5), 0.0, np.full(2, wl.origin), wl.spacing)
        lab = med[lev - 1][1]
        frac = np.stack([(lab == j).mean(axis=1) for j in range(wl.n_cont)], axis=1)
        assert np.abs(fb - w[None, :] * frac).max() < 1e-9 * w.max(), lev


def test_bench_workload_macro_solve():
    """The 17x17 three-level workload at the default tolerance: device buffers in and out, the
    solve converges and matches the oracle's solve of the same system."""
    wl = mi.workload("channel2d_17x17_L3")
    s, E, med = _gpu(wl)
    d, N = wl.dim, wl.n_cont
    fb = []
    for lev in range(1, wl.n_levels + 1):
        out = torch.zeros((s.num_points(lev), N), dtype=torch.float64, device="cuda")
        s.macro_source(lev, _weights(N), np.full(d, 0.5), 40.0, np.full(d, wl.origin),
                       wl.spacing, out=out)
        fb.append(out)
    Et = [torch.from_numpy(e).cuda() for e in E]
    U = torch.zeros((N, (wl.macro_n + 1) ** d), dtype=torch.float64, device="cuda")
    _, iters, rr = s.macro_solve(Et, fb, wl.spacing, tol=1e-13, out=U)
    assert rr <= 1e-13
    pl = plan.level_plan(wl)
    Uo = macro.solve(wl.macro_n, d, wl.spacing,
                     macro.grid_from_levels(pl, wl.macro_n, d, E),
                     macro.grid_from_levels(pl, wl.macro_n, d, [f.cpu().numpy() for f in fb]))
    Ug = U.cpu().numpy()
    assert np.abs(Uo).max() > 0
    assert np.abs(Ug - Uo).max() < 1e-6 * np.abs(Uo).max()
