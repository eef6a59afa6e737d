"""Gradient of a loss of the effective coefficients with respect to kappa (oracle).

Loss L = sum over levels and points of sum_rs W_p[r,s] E_p[r,s], with E_p the effective
coefficients of Sec. 2, Eq. (Bs_defi) computed through the hierarchy of Sec. 3 (Eqs.
PhiXiI, phiXiI_all, phi_avar_corrector, phi_grad_corrector). The paper has no gradient;
this is the adjoint of the oracle's own forward computation, derived from the energy form
of Sec. 3, Eq. (phi_abstract), and written with the same sparse operators:

For a point p of level n with seed V_r = dL/dPhi_r collected from its children, and
What = (W + W^T) / |R_p|:
  * adjoint constrained solve on the level-n grid (only the seeds need one):
        A_n mu_r + C_n^T nu_r = P^T V_r,   C_n mu_r = 0;
  * kappa gradient of every level-n element E (A_1 depends on kappa_E through the fine
    elements e inside E, each contributing Khat to its nodes):
        dL/dkappa_E = sum_{e in E} [ sum_rs W_rs Phi_r|e^T Khat Phi_s|e / |R_p|
                                     - sum_r (P mu_r)|e^T Khat Phi_r|e ];
  * seed for the parents t (weights c_t), on the level-1 grid:
        U_r = V_r + sum_s What_rs (A_1 Phi_s - C_1^T beta_s) - A_1 P mu_r - C_1^T nu_r,
        V_t,r += c_t U_r,
with beta the multipliers of the forward solve (A_n Xi - C_n^T beta = b). Levels are
processed from L down to 1. Checked against central finite differences and the Euler
identity sum_e kappa_e dL/dkappa_e = L (E is 1-homogeneous in kappa jointly over levels).
"""
from __future__ import annotations

import numpy as np

from . import cell, fe


def forward(wl, plan, media_levels):
    """Forward pass keeping every point's solve result (Phi, Xi, beta, keep, E)."""
    res = []
    for n, lev in enumerate(plan):
        ops = cell.LevelOps(wl, n + 1)
        kap, lab = media_levels[n]
        out = []
        for i in range(len(lev["points"])):
            I = None
            if n > 0:
                I = np.zeros((ops.gf.n_nodes, wl.n_rhs))
                for (lv, pos, w) in lev["parents"][i]:
                    I += w * res[lv - 1][pos]["Phi"].T
            out.append(cell.solve_point(ops, kap[i], lab[i], I, overs=getattr(wl, "overs", 0)))
        res.append(out)
    return res


def loss(fwd, weights):
    return float(sum(np.sum(weights[n][i] * r["E"]) for n, lev in enumerate(fwd)
                     for i, r in enumerate(lev)))


def _point_adjoint(wl, ops, kap, lab, r, W, V):
    """One point of level n (ops) in the reverse sweep: its kappa gradient per level-n element
    and, for n > 1, the seed U pushed to its parents (None at level 1)."""
    if getattr(wl, "overs", 0):
        return _point_adjoint_region(wl, ops, kap, lab, r, W, V)
    d, R = wl.dim, wl.n_rhs
    vol = wl.rve_len ** d
    Kh, _ = fe.unit_element_matrices(d)
    gf, P = ops.gf, ops.P
    What = (W + W.T) / vol
    kf = cell.prolong_medium(kap, d, ops.n_c, ops.rho)
    lf = cell.prolong_medium(lab, d, ops.n_c, ops.rho)
    A1 = fe.stiffness_full(gf, kf)
    C1 = fe.constraint_rows(gf, lf, wl.n_cont, wl.periods)[r["keep"]]
    AX = (P.T @ A1 @ P).tocsr()
    CX = (C1 @ P).tocsr()
    Phi = r["Phi"].T                                   # [nodes, R]
    f = P.T @ V
    if np.any(f):
        mu, nu_neg = cell.saddle_solve(AX, CX, f, np.zeros((CX.shape[0], R)))
        nu = -nu_neg                                   # A mu + C^T nu = f
    else:
        mu = np.zeros((P.shape[1], R))
        nu = np.zeros((CX.shape[0], R))
    Pmu = P @ mu
    # kappa gradient per fine element, summed over the fine elements of each E
    Pe = Phi[gf.enodes]                                # [ne, 2^d, R]
    Me = Pmu[gf.enodes]
    KP = np.einsum("ab,ebr->ear", Kh, Pe)              # Khat Phi on each element
    ge = (np.einsum("rs,ear,eas->e", W / vol, Pe, KP) -
          np.einsum("ear,ear->e", Me, KP)) * gf.h ** (d - 2)
    ec = gf.ecoord // ops.rho
    idx = sum(ec[:, a] * ops.n_c ** a for a in range(d))
    g = np.bincount(idx, weights=ge, minlength=ops.n_c ** d)
    if ops.level == 1:
        return g, None
    beta = r["beta"]
    U = V + (A1 @ Phi - C1.T @ beta) @ What.T - A1 @ Pmu - C1.T @ nu
    U[~np.isin(np.arange(gf.n_nodes), gf.interior_nodes)] = 0.0
    return g, U


def _point_adjoint_region(wl, ops, kap, lab, r, W, V):
    """The same step when E is integrated over R_p, the central (P - 2o)^d periods
    (oversampling). E_R = Phi^T A_{1,R} Phi / |R_p| is no longer stationary in Phi (the cell
    problem minimises the energy over the whole RVE), so the level's own term enters as an
    adjoint source instead of through the envelope form:
        V_tot,r = V_r + sum_s What_rs A_{1,R} Phi_s,   What = (W + W^T) / |R_p|
        A_n mu_r + C_n^T nu_r = P^T V_tot,r,   C_n mu_r = 0
        dL/dkappa_E = sum_{e in E} [ [e in R_p] sum_rs W_rs Phi_r|e^T Khat Phi_s|e / |R_p|
                                     - sum_r (P mu_r)|e^T Khat Phi_r|e ]
        U_r = V_tot,r - A_1 P mu_r - C_1^T nu_r.
    With R_p = Y+ this reduces to the envelope form of _point_adjoint."""
    d, R = wl.dim, wl.n_rhs
    Kh, _ = fe.unit_element_matrices(d)
    gf, P = ops.gf, ops.P
    reg = gf.region_mask(wl.periods, wl.overs)
    vol = reg.sum() * gf.h ** d
    What = (W + W.T) / vol
    kf = cell.prolong_medium(kap, d, ops.n_c, ops.rho)
    lf = cell.prolong_medium(lab, d, ops.n_c, ops.rho)
    A1 = fe.stiffness_full(gf, kf)
    AR = fe.stiffness_full(gf, kf * reg)
    C1 = fe.constraint_rows(gf, lf, wl.n_cont, wl.periods)[r["keep"]]
    AX = (P.T @ A1 @ P).tocsr()
    CX = (C1 @ P).tocsr()
    Phi = r["Phi"].T                                   # [nodes, R]
    interior = np.isin(np.arange(gf.n_nodes), gf.interior_nodes)
    Vt = V + (AR @ Phi) @ What.T
    Vt[~interior] = 0.0
    f = P.T @ Vt
    if np.any(f):
        mu, nu_neg = cell.saddle_solve(AX, CX, f, np.zeros((CX.shape[0], R)))
        nu = -nu_neg                                   # A mu + C^T nu = f
    else:
        mu = np.zeros((P.shape[1], R))
        nu = np.zeros((CX.shape[0], R))
    Pmu = P @ mu
    Pe = Phi[gf.enodes]                                # [ne, 2^d, R]
    Me = Pmu[gf.enodes]
    KP = np.einsum("ab,ebr->ear", Kh, Pe)
    ge = (reg * np.einsum("rs,ear,eas->e", W / vol, Pe, KP) -
          np.einsum("ear,ear->e", Me, KP)) * gf.h ** (d - 2)
    ec = gf.ecoord // ops.rho
    idx = sum(ec[:, a] * ops.n_c ** a for a in range(d))
    g = np.bincount(idx, weights=ge, minlength=ops.n_c ** d)
    if ops.level == 1:
        return g, None
    U = Vt - A1 @ Pmu - C1.T @ nu
    U[~interior] = 0.0
    return g, U


def backward(wl, plan, media_levels, fwd, weights):
    """dL/dkappa per level, [npts, n_n^d], for L = sum W * E."""
    R = wl.n_rhs
    L = len(plan)
    nf_nodes = fe.Grid(wl.dim, wl.n_fine, wl.rve_len).n_nodes
    seeds = [np.zeros((len(plan[n]["points"]), nf_nodes, R)) for n in range(L)]
    grads = [None] * L
    for n in range(L - 1, -1, -1):
        ops = cell.LevelOps(wl, n + 1)
        kap, lab = media_levels[n]
        npts = len(plan[n]["points"])
        g_lev = np.zeros((npts, ops.n_c ** wl.dim))
        for i in range(npts):
            g_lev[i], U = _point_adjoint(wl, ops, kap[i], lab[i], fwd[n][i], weights[n][i],
                                         seeds[n][i])
            if n > 0:
                for (lv, pos, w) in plan[n]["parents"][i]:
                    seeds[lv - 1][pos] += w * U
        grads[n] = g_lev
    return grads


def backward_sampled(wl, plan, media_fn, weights):
    """The same gradient for a loss whose weights vanish outside a few points.

    weights: {(level, position): W [R, R]}. Only those points and their ancestors carry
    seeds, so the forward and reverse sweeps run over that closure alone (Algorithm 1
    restricted to it). media_fn(level, positions) -> (kappa, labels). Returns
    ({(level, position): dL/dkappa [n_n^d]}, loss)."""
    R = wl.n_rhs
    fwd = cell.run_sampled(wl, plan, media_fn, list(weights))
    nf_nodes = fe.Grid(wl.dim, wl.n_fine, wl.rve_len).n_nodes
    seeds = {k: np.zeros((nf_nodes, R)) for k in fwd}
    zero = np.zeros((R, R))
    loss_val = float(sum(np.sum(W * fwd[k]["E"]) for k, W in weights.items()))
    grads = {}
    for n in range(len(plan), 0, -1):
        pos = sorted(i for (l, i) in fwd if l == n)
        if not pos:
            continue
        ops = cell.LevelOps(wl, n)
        kap, lab = media_fn(n, pos)
        for k, i in enumerate(pos):
            grads[(n, i)], U = _point_adjoint(wl, ops, kap[k], lab[k], fwd[(n, i)],
                                              weights.get((n, i), zero), seeds[(n, i)])
            if n > 1:
                for (lv, pp, w) in plan[n - 1]["parents"][i]:
                    seeds[(lv, pp)] += w * U
    return grads, loss_val
