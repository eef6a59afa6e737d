"""Macroscopic multicontinuum problem (oracle; test infrastructure only).

Sec. 2, Eq. (macro_eq): for N continua, with coefficients constant on every coarse block,
    B_ji U_i + B^m_ji d_m U_i - d_n (Bbar^n_ji U_i) - d_n (B^mn_ji d_m U_i) = b_j,
the coefficients and the source being the cell-function integrals of Eq. (Bs_defi).

The paper prints no discretisation of this system; the readings taken here:
  * Coarse blocks K_p = x_p + [-H/2, H/2]^d around every macropoint of T_L (H = the macro
    spacing); Sec. 5 treats every coarse block as an RVE (R_p = K_p). The macro mesh is
    these blocks, U_j is Q1 on their (M+1)^d vertices (x fastest), zero Dirichlet data on
    the outer boundary.
  * Coefficients and source as densities on K_p: E_p (E_rs = (1/|R_p|) int_{R_p} kappa
    grad Phi_r . grad Phi_s, the library's output; B = |K_p| E_p) and
    fbar_j(p) = (1/|R_p|) int_{R_p} f phi_j.
  * Weak form: sum_p int_{K_p} w(V)^T E_p w(U) dx = sum_p int_{K_p} sum_j fbar_j(p) V_j dx,
    w(U) = (U_0, .., U_{N-1}, d_0 U_0, .., d_{d-1} U_0, .., d_{d-1} U_{N-1}) in the order of
    the cell functions (r = i, r = N + i d + m); integrated exactly (2 Gauss points per axis).
  * Source (Sec. 5): f = s_j exp(-alpha |x - c|^2) in continuum j (there s = (eta, 1) for
    the low- and high-conductivity continua, alpha = 40, c = the domain centre), sampled at
    the centroids of the level-1-grid elements of the RVE; for a point of level n an
    element's continuum is that of the level-n element containing it (the child's medium,
    prolonged piecewise constantly). int_{R_p} f phi_j = sum_e f_e int_e phi_j is exact for
    this piecewise-constant f and the Q1 phi_j (int_e N_b = h^d / 2^d per corner).
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spl

from . import fe
from .cell import prolong_medium

_GAUSS = (0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0))   # 2-point Gauss on [0,1]


def source_point(wl, level: int, phi, labels, x_p, weights, center, alpha: float,
                 overs: int = 0):
    """fbar [N] of one macropoint: phi [>= N, (n_1+1)^d] its cell functions on the level-1
    lattice (the first N are phi_i), labels [n_n^d] its level-n labels, x_p its position."""
    d, N = wl.dim, wl.n_cont
    gf = fe.Grid(d, wl.n_fine, wl.rve_len)
    n_c = wl.n_level(level)
    lf = prolong_medium(np.asarray(labels), d, n_c, wl.n_fine // n_c).astype(np.int64)
    x = np.asarray(x_p, dtype=np.float64)[None, :] + gf.ecent
    G = np.exp(-alpha * np.sum((x - np.asarray(center, dtype=np.float64)[None, :]) ** 2,
                               axis=1))
    f = np.asarray(weights, dtype=np.float64)[lf] * G
    reg = gf.region_mask(wl.periods, overs)
    f = np.where(reg, f, 0.0)
    vol = reg.sum() * gf.h ** d
    corner_w = gf.h ** d / 2 ** d
    out = np.zeros(N)
    for j in range(N):
        out[j] = np.sum(f * corner_w * phi[j][gf.enodes].sum(axis=1)) / vol
    return out


def _ref_tables(d: int):
    """Q1 shape values [g, b] and reference gradients [g, b, a] at the 2^d Gauss points,
    and the Gauss weights [g] (of the unit cube)."""
    cs = fe.corners(d)
    gps = list(itertools.product(range(2), repeat=d))
    val = np.zeros((len(gps), len(cs)))
    grad = np.zeros((len(gps), len(cs), d))
    for g, qp in enumerate(gps):
        xi = [_GAUSS[i] for i in qp]
        for b, c in enumerate(cs):
            v, gr = fe._shape(xi, c)
            val[g, b] = v
            grad[g, b] = gr
    return val, grad, np.full(len(gps), 0.5 ** d)


def assemble(M: int, d: int, H: float, E_grid, fbar_grid):
    """Global matrix on the (M+1)^d vertex lattice x N continua (unknown (node, j) at
    j * (M+1)^d + node) and load vector, before the boundary conditions. E_grid [M^d, R, R]
    and fbar_grid [M^d, N] in macro order (x fastest)."""
    E_grid = np.asarray(E_grid, dtype=np.float64)
    fbar_grid = np.asarray(fbar_grid, dtype=np.float64)
    R = E_grid.shape[1]
    N = R // (1 + d)
    g = fe.Grid(d, M, M * H)
    nn = g.n_nodes
    val, grad, wq = _ref_tables(d)
    vol = H ** d
    nb = 2 ** d
    # W[g][s, (b, i)]: the value of w_s(U) at Gauss point g for U = N_b in continuum i
    W = np.zeros((len(wq), R, nb * N))
    for q in range(len(wq)):
        for b in range(nb):
            for i in range(N):
                W[q, i, b * N + i] = val[q, b]
                for m in range(d):
                    W[q, N + i * d + m, b * N + i] = grad[q, b, m] / H
    rows, cols, vals = [], [], []
    rhs = np.zeros(N * nn)
    for e in range(g.n_el):
        Ke = np.zeros((nb * N, nb * N))
        for q in range(len(wq)):
            Ke += wq[q] * vol * (W[q].T @ E_grid[e] @ W[q])
        dofs = np.array([i * nn + g.enodes[e, b] for b in range(nb) for i in range(N)])
        rows.append(np.repeat(dofs, nb * N))
        cols.append(np.tile(dofs, nb * N))
        vals.append(Ke.ravel())
        for b in range(nb):
            for i in range(N):
                rhs[i * nn + g.enodes[e, b]] += fbar_grid[e, i] * vol / nb
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(N * nn, N * nn))
    return A, rhs, g


def solve(M: int, d: int, H: float, E_grid, fbar_grid):
    """U [N, (M+1)^d] with zero boundary values."""
    A, rhs, g = assemble(M, d, H, E_grid, fbar_grid)
    N = np.asarray(E_grid).shape[1] // (1 + d)
    nn = g.n_nodes
    interior = np.all((g.ncoord > 0) & (g.ncoord < M), axis=1)
    dof = np.concatenate([i * nn + np.nonzero(interior)[0] for i in range(N)])
    U = np.zeros(N * nn)
    U[dof] = spl.spsolve(A[dof][:, dof].tocsc(), rhs[dof])
    return U.reshape(N, nn)


def grid_from_levels(plan, M: int, d: int, per_level):
    """Arranges per-level arrays [npts_n, ...] into macro order [M^d, ...] using the level
    plan's macro indices."""
    first = np.asarray(per_level[0])
    out = np.zeros((M ** d,) + first.shape[1:])
    for lev, arr in zip(plan, per_level):
        pts = np.asarray(lev["points"])
        flat = sum(pts[:, a] * M ** a for a in range(d))
        out[flat] = np.asarray(arr)
    return out
