"""Constrained cell problems, hierarchy and effective coefficients (oracle).

Sec. 2, Eqs. (phi_avar), (phi_grad), in the energy form of Sec. 3,
Eq. (phi_abstract): for each macropoint and each cell function r,
minimise 1/2 int kappa |grad v|^2 over Q1 functions vanishing on the RVE
boundary subject to int_{R_q} psi_j v = G[(j,q), r] for every continuum j and
sub-block R_q. The stationarity conditions are the saddle-point system
    A x - C^T beta = b,   C x = g
(b = 0, g = G at level 1). It is solved here with a sparse LU of A, the
Schur complement S = C A^-1 C^T, and FP64 iterative refinement of the full
saddle-point residual.

Sec. 3.3, Eqs. (PhiXiI), (phiXiI_all), (phi_avar_corrector),
(phi_grad_corrector): at level n > 1, Phi = I + Xi with I = sum_t c_t Phi_t
(same-index parent functions on the level-1 grid) and Xi in V_n (the level-n
Q1 space embedded by the nested prolongation P_n). Substituting into the
energy form gives the correction problem, written out literally:
    min (I + P Xi)^T A_1 (I + P Xi)  s.t.  C_1 (I + P Xi) = G,
i.e. the saddle system with matrix P^T A_1 P, constraint C_1 P, right-hand
side b = -P^T A_1 I and targets g' = G - C_1 I.

Sec. 2, Eq. (Bs_defi): the effective coefficients are the energy Gram of the
cell functions over R_p, reported as E_rs = (1/|R_p|) int_{R_p} kappa
grad Phi_r . grad Phi_s (the caller multiplies by |K_p|). Block layout:
B_ji = E[j][i], B^m_ji = E[j][N+i d+m], Bbar^n_ji = E[N+j d+n][i],
B^{mn}_ji = E[N+j d+n][N+i d+m].
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spl

from . import fe


def saddle_solve(A, C, b, g, tol=1e-14, max_refine=6):
    """Solve [A -C^T; C 0][x; beta] = [b; g] for several right-hand sides.
    Sparse LU of A, dense Cholesky of the Schur complement S = C A^-1 C^T,
    then FP64 iterative refinement on both block rows."""
    lu = spl.splu(A.tocsc())
    Cd = C.toarray() if sp.issparse(C) else np.asarray(C)
    W = lu.solve(np.ascontiguousarray(Cd.T))
    S = Cd @ W
    cho = sla.cho_factor(0.5 * (S + S.T))

    def apply_inv(f1, f2):
        x0 = lu.solve(f1)
        beta = sla.cho_solve(cho, f2 - Cd @ x0)
        return x0 + W @ beta, beta

    x, beta = apply_inv(b, g)
    nb = max(np.linalg.norm(b), np.linalg.norm(A @ x)) + 1e-300
    ng = np.linalg.norm(g) + 1e-300
    for _ in range(max_refine):
        r1 = b - (A @ x - Cd.T @ beta)
        r2 = g - Cd @ x
        if np.linalg.norm(r1) <= tol * nb and np.linalg.norm(r2) <= tol * ng:
            break
        dx, db = apply_inv(r1, r2)
        x += dx
        beta += db
    return x, beta


def prolong_medium(values: np.ndarray, d: int, n_coarse: int, rho: int) -> np.ndarray:
    """Piecewise-constant prolongation of an element field from the level-n
    grid to the level-1 grid (reading of Sec. 3.2 for the child's medium)."""
    if rho == 1:
        return values.copy()
    shape = (n_coarse,) * d
    v = values.reshape(shape[::-1])            # array axes (z, y, x)
    for ax in range(d):
        v = np.repeat(v, rho, axis=ax)
    return v.reshape(-1)


class LevelOps:
    """Grids and the nested prolongation for one level (independent of the point)."""

    def __init__(self, wl, level: int):
        self.wl = wl
        self.level = level
        self.n_c = wl.n_level(level)
        self.n_f = wl.n_fine
        self.rho = self.n_f // self.n_c
        self.gc = fe.Grid(wl.dim, self.n_c, wl.rve_len)
        self.gf = fe.Grid(wl.dim, self.n_f, wl.rve_len)
        Pfull = fe.prolongation(self.gc, self.gf) if self.rho > 1 else sp.identity(
            self.gf.n_nodes, format="csr")
        self.P = Pfull[:, self.gc.interior_nodes].tocsr()     # fine full lattice <- coarse interior
        self.region = self.gf.region_mask(wl.periods, 0)


def solve_point(ops: LevelOps, kappa, labels, I=None, overs: int = 0):
    """One macropoint of one level: returns dict with Phi (fine full lattice,
    [R, (n_1+1)^d]), Xi (coarse interior, [R, (n-1)^d]), beta, kept rows,
    targets and E [R, R]."""
    wl = ops.wl
    d, N = wl.dim, wl.n_cont
    R = N * (1 + d)
    gf, gc, P = ops.gf, ops.gc, ops.P
    kf = prolong_medium(kappa, d, ops.n_c, ops.rho)
    lf = prolong_medium(labels, d, ops.n_c, ops.rho)
    A1 = fe.stiffness_full(gf, kf)
    C1 = fe.constraint_rows(gf, lf, N, wl.periods)
    G = fe.targets(gc, labels, N, wl.periods, overs)
    if I is None:
        I = np.zeros((gf.n_nodes, R))
    AX = (P.T @ A1 @ P).tocsr()
    CX = (C1 @ P).tocsr()
    keep = np.asarray(abs(CX).sum(axis=1)).ravel() > 0
    CX = CX[keep]
    b = -(P.T @ (A1 @ I))
    g = G[keep] - C1[keep] @ I
    Xi, beta = saddle_solve(AX, CX, b, g)
    Phi = I + P @ Xi
    if overs:
        reg = gf.region_mask(wl.periods, overs)
        ARp = fe.stiffness_full(gf, kf * reg)
        vol = reg.sum() * gf.h ** d
    else:
        ARp = A1
        vol = wl.rve_len ** d
    E = Phi.T @ (ARp @ Phi) / vol
    return {"Phi": Phi.T.copy(), "Xi": Xi.T.copy(), "beta": beta, "keep": keep,
            "G": G, "E": E, "n_dropped": int((~keep).sum()),
            "kappa_fine": kf, "labels_fine": lf}


def run_hierarchy(wl, plan, media_levels, keep_phi=True, points=None):
    """Algorithm 1, lines 3-8: levels in order, points of each level in order.
    media_levels[n] = (kappa [npts, n_n^d], labels [npts, n_n^d]).
    Returns per level a dict with E [npts, R, R] and (if keep_phi) Phi."""
    out = []
    phis = []
    for n, lev in enumerate(plan):
        ops = LevelOps(wl, n + 1)
        kap, lab = media_levels[n]
        npts = len(lev["points"])
        R = wl.n_rhs
        E = np.zeros((npts, R, R))
        Phi = np.zeros((npts, R, ops.gf.n_nodes)) if (keep_phi or n + 1 < len(plan)) else None
        res = []
        for i in range(npts):
            if points is not None and n + 1 == len(plan) and i not in points:
                continue
            I = None
            if n > 0:
                I = np.zeros((ops.gf.n_nodes, R))
                for (lv, pos, w) in lev["parents"][i]:
                    I += w * phis[lv - 1][pos].T
            r = solve_point(ops, kap[i], lab[i], I, overs=getattr(wl, "overs", 0))
            E[i] = r["E"]
            if Phi is not None:
                Phi[i] = r["Phi"]
            res.append(r)
        phis.append(Phi)
        out.append({"E": E, "Phi": Phi})
    return out


def ancestors(plan, level: int, idx: int, acc=None):
    """Set of (level, position) pairs needed to compute point `idx` of `level` (itself
    and, recursively, its parents)."""
    if acc is None:
        acc = set()
    if (level, idx) in acc:
        return acc
    acc.add((level, idx))
    if level > 1:
        for (lv, pos, _) in plan[level - 1]["parents"][idx]:
            ancestors(plan, lv, pos, acc)
    return acc


def run_sampled(wl, plan, media_fn, targets):
    """Algorithm 1 restricted to the listed (level, position) targets and their ancestors,
    levels in order. media_fn(level, positions) -> (kappa, labels) for those points.
    Returns {(level, position): solve_point result}."""
    need = set()
    for (lv, i) in targets:
        ancestors(plan, lv, i, need)
    out = {}
    for lv in range(1, len(plan) + 1):
        pos = sorted(i for (l, i) in need if l == lv)
        if not pos:
            continue
        ops = LevelOps(wl, lv)
        kap, lab = media_fn(lv, pos)
        for k, i in enumerate(pos):
            I = None
            if lv > 1:
                I = np.zeros((ops.gf.n_nodes, wl.n_rhs))
                for (pl, pp, w) in plan[lv - 1]["parents"][i]:
                    I += w * out[(pl, pp)]["Phi"].T
            out[(lv, i)] = solve_point(ops, kap[k], lab[k], I, overs=getattr(wl, "overs", 0))
    return out
