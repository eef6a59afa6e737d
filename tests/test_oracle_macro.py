"""Pins of the oracle's macroscopic multicontinuum problem (Sec. 2, Eq. macro_eq).

None of these re-types an oracle formula: the assembly is compared with a tensor-product
(Kronecker) construction from 1D element integrals, the discretisation with the second-order
convergence of a manufactured solution, the source with the exact identity that the
constraints of Eqs. (phi_avar) impose on the constant cell functions.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import mch_inputs as mi
from oracle import cell, macro, plan


def _oned(M, H):
    """Global 1D Q1 matrices on M elements of length H: mass, stiffness and
    D[a, b] = int phi_a' phi_b."""
    n = M + 1
    Mg = np.zeros((n, n))
    Kg = np.zeros((n, n))
    Dg = np.zeros((n, n))
    me = H / 6 * np.array([[2.0, 1.0], [1.0, 2.0]])
    ke = 1 / H * np.array([[1.0, -1.0], [-1.0, 1.0]])
    de = np.array([[-0.5, -0.5], [0.5, 0.5]])   # (d/dx N_a) * int N_b
    for e in range(M):
        idx = [e, e + 1]
        Mg[np.ix_(idx, idx)] += me
        Kg[np.ix_(idx, idx)] += ke
        Dg[np.ix_(idx, idx)] += de
    return Mg, Kg, Dg


def _spd(R, rng):
    A = rng.standard_normal((R, R))
    return A @ A.T + R * np.eye(R)


@pytest.mark.parametrize("N", [1, 2])
def test_assembly_matches_kronecker(N):
    """Constant coefficients (2D): the element-loop assembly equals the sum over the blocks
    of E of Kronecker products of 1D mass, stiffness and derivative matrices."""
    rng = np.random.default_rng(7)
    d, M, H = 2, 5, 0.2
    R = N * (1 + d)
    E = _spd(R, rng)
    A, _, g = macro.assemble(M, d, H, np.repeat(E[None], M ** d, axis=0), np.zeros((M ** d, N)))
    Mg, Kg, Dg = _oned(M, H)
    nn = (M + 1) ** d

    def w_op(r, s):
        # int w_r(V) w_s(U) with V, U in one continuum each, lattice index iy * (M+1) + ix
        def kind(t):
            return ("val", None) if t < N else ("der", (t - N) % d)
        kr, kv = kind(r), kind(s)
        if kr[0] == "val" and kv[0] == "val":
            return np.kron(Mg, Mg)
        if kr[0] == "val":                       # V, d_m U
            return np.kron(Mg, Dg.T) if kv[1] == 0 else np.kron(Dg.T, Mg)
        if kv[0] == "val":                       # d_n V, U
            return np.kron(Mg, Dg) if kr[1] == 0 else np.kron(Dg, Mg)
        n_, m_ = kr[1], kv[1]
        if n_ == 0 and m_ == 0:
            return np.kron(Mg, Kg)
        if n_ == 1 and m_ == 1:
            return np.kron(Kg, Mg)
        if n_ == 0 and m_ == 1:
            return np.kron(Dg.T, Dg)
        return np.kron(Dg, Dg.T)

    def cont(t):
        return t if t < N else (t - N) // d

    ref = np.zeros((N * nn, N * nn))
    for r in range(R):
        for s in range(R):
            j, i = cont(r), cont(s)
            ref[j * nn:(j + 1) * nn, i * nn:(i + 1) * nn] += E[r, s] * w_op(r, s)
    Ad = A.toarray()
    assert np.abs(Ad - ref).max() < 1e-12 * np.abs(ref).max()
    assert np.abs(Ad - Ad.T).max() < 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("d,Ms", [(2, (16, 32, 64)), (3, (8, 16))])
def test_manufactured_solution_second_order(d, Ms):
    """c U - k Laplace U = F with U = prod sin(pi x_a / L), midpoint source per block: the
    nodal error falls by ~4 per halving of H (second-order Q1 with exact integration)."""
    c, k, L = 3.0, 2.0, 1.0
    errs = []
    for M in Ms:
        H = L / M
        E = np.diag([c] + [k] * d)
        cen = (np.stack(np.meshgrid(*[np.arange(M)] * d, indexing="ij")[::-1], -1)
               .reshape(-1, d) + 0.5) * H
        F = (c + d * k * np.pi ** 2 / L ** 2) * np.prod(np.sin(np.pi * cen / L), axis=1)
        U = macro.solve(M, d, H, np.repeat(E[None], M ** d, axis=0), F[:, None])
        g = (np.stack(np.meshgrid(*[np.arange(M + 1)] * d, indexing="ij")[::-1], -1)
             .reshape(-1, d)) * H
        Ue = np.prod(np.sin(np.pi * g / L), axis=1)
        errs.append(np.abs(U[0] - Ue).max())
    for a, b in zip(errs[:-1], errs[1:]):
        assert 3.6 < a / b < 4.4, errs


def test_decoupled_continua():
    """Block-diagonal coefficients (no exchange, no cross terms): each continuum solves its
    own single-continuum problem."""
    rng = np.random.default_rng(3)
    d, M, H, N = 2, 6, 1 / 6, 2
    R = N * (1 + d)
    Es = np.zeros((M ** d, R, R))
    singles = [np.zeros((M ** d, 1 + d, 1 + d)) for _ in range(N)]
    for e in range(M ** d):
        for j in range(N):
            B = _spd(1 + d, rng)
            idx = [j] + [N + j * d + m for m in range(d)]
            Es[e][np.ix_(idx, idx)] = B
            singles[j][e] = B
    f = rng.random((M ** d, N))
    U = macro.solve(M, d, H, Es, f)
    for j in range(N):
        Uj = macro.solve(M, d, H, singles[j], f[:, j:j + 1])
        assert np.abs(U[j] - Uj[0]).max() < 1e-12 * np.abs(Uj).max()


def test_source_constant_per_continuum_is_volume_fraction():
    """alpha = 0 (f = s_j in continuum j): the constraints int_{R_q} psi_j phi_i =
    delta_ij |R_q cap Omega_j| make fbar_i = s_i |R_p cap Omega_i| / |R_p| exactly, on every
    level of the hierarchy."""
    wl = mi.small_workload("channel2d_17x17_L3", n_fine=64, macro_n=9)
    pl = plan.level_plan(wl)
    med = [mi.media(wl, lev["points"], wl.n_level(n + 1)) for n, lev in enumerate(pl)]
    out = cell.run_hierarchy(wl, pl, med)
    s = np.array([0.25, 1.5])
    for n, lev in enumerate(pl):
        for i in range(0, len(lev["points"]), 5):
            x_p = mi.macro_points_xyz(wl, lev["points"][i:i + 1])[0]
            fb = macro.source_point(wl, n + 1, out[n]["Phi"][i], med[n][1][i], x_p, s,
                                    np.full(wl.dim, 0.5), 0.0)
            frac = np.array([(med[n][1][i] == j).mean() for j in range(wl.n_cont)])
            assert np.abs(fb - s * frac).max() < 1e-12 * s.max()


def test_macro_system_spd_with_hierarchy_coefficients():
    """With the effective coefficients of a hierarchy (symmetric positive definite per
    block), the macro matrix is symmetric positive definite (Cholesky succeeds)."""
    wl = mi.small_workload("channel2d_17x17_L3", n_fine=64, macro_n=9)
    pl = plan.level_plan(wl)
    med = [mi.media(wl, lev["points"], wl.n_level(n + 1)) for n, lev in enumerate(pl)]
    out = cell.run_hierarchy(wl, pl, med)
    M, d = wl.macro_n, wl.dim
    E = macro.grid_from_levels(pl, M, d, [o["E"] for o in out])
    A, _, g = macro.assemble(M, d, wl.spacing, E, np.zeros((M ** d, wl.n_cont)))
    nn = g.n_nodes
    interior = np.nonzero(np.all((g.ncoord > 0) & (g.ncoord < M), axis=1))[0]
    dof = np.concatenate([j * nn + interior for j in range(wl.n_cont)])
    Ai = A[dof][:, dof].toarray()
    assert np.abs(Ai - Ai.T).max() < 1e-12 * np.abs(Ai).max()
    np.linalg.cholesky(0.5 * (Ai + Ai.T))


def test_grid_from_levels_places_points_by_macro_index():
    """Per-level arrays land at the flat macro index of their points (x fastest), and the
    levels of the plan cover every macropoint exactly once."""
    for name in ("channel2d_17x17_L3", "channel3d_9x9x9_L3"):
        wl = mi.workload(name)
        pl = plan.level_plan(wl)
        M, d = wl.macro_n, wl.dim
        vals = [np.asarray(lev["points"], dtype=np.float64) for lev in pl]   # value = index
        g = macro.grid_from_levels(pl, M, d, vals)
        want = np.stack(np.meshgrid(*[np.arange(M)] * d, indexing="ij")[::-1], -1).reshape(-1, d)
        assert np.array_equal(g, want)
        assert sum(len(lev["points"]) for lev in pl) == M ** d

