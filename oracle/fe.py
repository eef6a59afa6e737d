"""Q1 finite-element building blocks on a uniform RVE grid (oracle, FP64).

Sec. 2, Eq. (weak_galerkin): bilinear (2D) / trilinear (3D) elements on
rectangles for the energy int kappa grad u . grad v, zero Dirichlet data on
the RVE boundary. Sec. 2, Eqs. (phi_avar), (phi_grad): the constraint
functionals int_{R_q} psi_j v and their targets.

Grid conventions: an RVE Y+ = [-l/2, l/2]^d is split into n^d elements of
size h = l/n; element (e_0, .., e_{d-1}) has flat index sum_a e_a n^a (x
fastest); nodes are indexed the same way on the (n+1)^d lattice and the
unknowns are the (n-1)^d interior nodes, also x fastest.
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp

_GAUSS = (0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0))   # 2-point Gauss on [0,1]


def corners(d: int):
    """Local corner offsets of a unit element, corner c <-> bits of c."""
    return [tuple((c >> a) & 1 for a in range(d)) for c in range(2 ** d)]


def _shape(xi, b):
    """Q1 shape function of corner b at reference point xi and its gradient."""
    d = len(xi)
    f1 = [xi[a] if b[a] else 1.0 - xi[a] for a in range(d)]
    df1 = [1.0 if b[a] else -1.0 for a in range(d)]
    val = float(np.prod(f1))
    grad = []
    for a in range(d):
        g = df1[a]
        for o in range(d):
            if o != a:
                g *= f1[o]
        grad.append(g)
    return val, np.array(grad)


def unit_element_matrices(d: int):
    """Unit-cube Q1 element stiffness Khat (int grad N_b . grad N_c) and the
    element moments int N_b, int N_b xi_a, all by 2-point Gauss quadrature
    per axis (exact for these polynomial degrees)."""
    cs = corners(d)
    nc = len(cs)
    K = np.zeros((nc, nc))
    mom0 = np.zeros(nc)
    for qp in itertools.product(range(2), repeat=d):
        xi = [_GAUSS[i] for i in qp]
        w = 0.5 ** d
        vals, grads = zip(*[_shape(xi, b) for b in cs])
        for i in range(nc):
            mom0[i] += w * vals[i]
            for j in range(nc):
                K[i, j] += w * float(grads[i] @ grads[j])
    return K, mom0


class Grid:
    """Index maps of an n^d RVE grid."""

    def __init__(self, d: int, n: int, rve_len: float):
        self.d, self.n, self.l = d, n, rve_len
        self.h = rve_len / n
        self.n_el = n ** d
        self.n_nodes = (n + 1) ** d
        e = np.arange(self.n_el)
        self.ecoord = np.stack([(e // n ** a) % n for a in range(d)], axis=1)   # [ne, d]
        cs = corners(d)
        self.enodes = np.stack(
            [sum((self.ecoord[:, a] + b[a]) * (n + 1) ** a for a in range(d)) for b in cs],
            axis=1)                                                             # [ne, 2^d]
        k = np.arange(self.n_nodes)
        self.ncoord = np.stack([(k // (n + 1) ** a) % (n + 1) for a in range(d)], axis=1)
        interior = np.all((self.ncoord > 0) & (self.ncoord < n), axis=1)
        self.interior_nodes = np.nonzero(interior)[0]
        self.n_int = self.interior_nodes.size
        self.node_to_int = -np.ones(self.n_nodes, dtype=np.int64)
        self.node_to_int[self.interior_nodes] = np.arange(self.n_int)
        # element centroids in local coordinates y in [-l/2, l/2]^d
        self.ecent = -rve_len / 2 + (self.ecoord + 0.5) * self.h

    def block_of_element(self, periods: int) -> np.ndarray:
        """Sub-block index q of each element (R_q = the P^d periods)."""
        m = self.n // periods
        qa = self.ecoord // m
        return sum(qa[:, a] * periods ** a for a in range(self.d))

    def region_mask(self, periods: int, overs: int) -> np.ndarray:
        """Elements of the integration region R_p: the central (P-2o)^d periods."""
        m = self.n // periods
        lo, hi = overs * m, (periods - overs) * m
        return np.all((self.ecoord >= lo) & (self.ecoord < hi), axis=1)


def stiffness_full(g: Grid, kappa: np.ndarray) -> sp.csr_matrix:
    """A = sum_e kappa_e h^(d-2) Khat on all (n+1)^d nodes (Eq. weak_galerkin)."""
    K, _ = unit_element_matrices(g.d)
    nc = K.shape[0]
    scale = kappa * g.h ** (g.d - 2)
    rows = np.repeat(g.enodes, nc, axis=1).ravel()
    cols = np.tile(g.enodes, (1, nc)).ravel()
    vals = (scale[:, None] * K.ravel()[None, :]).ravel()
    return sp.csr_matrix((vals, (rows, cols)), shape=(g.n_nodes, g.n_nodes))


def stiffness(g: Grid, kappa: np.ndarray) -> sp.csr_matrix:
    """Interior block of the stiffness matrix (zero Dirichlet data)."""
    A = stiffness_full(g, kappa)
    ii = g.interior_nodes
    return A[ii][:, ii].tocsr()


def constraint_rows(g: Grid, labels: np.ndarray, n_cont: int, periods: int):
    """Constraint functionals of Eqs. (phi_avar)/(phi_grad) on the full node
    lattice: row (j, q) is v -> int_{R_q} psi_j v, i.e. sum over elements of
    block q with label j of int_e N_b = h^d/2^d per corner. Returns the
    (N * P^d) x (n+1)^d matrix, rows ordered j * P^d + q."""
    _, mom0 = unit_element_matrices(g.d)
    nq = periods ** g.d
    blk = g.block_of_element(periods)
    row_of_el = labels.astype(np.int64) * nq + blk
    nc = mom0.size
    rows = np.repeat(row_of_el, nc)
    cols = g.enodes.ravel()
    vals = np.tile(mom0 * g.h ** g.d, g.n_el)
    return sp.csr_matrix((vals, (rows, cols)), shape=(n_cont * nq, g.n_nodes))


def centroids(g: Grid, labels: np.ndarray, n_cont: int, periods: int, overs: int):
    """c_mj with int_{R_p} (y_m - c_mj) psi_j = 0 (Eq. phi_grad; the region is
    read as R_p). Falls back to the whole RVE, then to 0, for an absent
    continuum."""
    reg = g.region_mask(periods, overs)
    c = np.zeros((g.d, n_cont))
    for j in range(n_cont):
        sel = reg & (labels == j)
        if not sel.any():
            sel = labels == j
        if sel.any():
            c[:, j] = g.ecent[sel].mean(axis=0)
    return c


def targets(g: Grid, labels: np.ndarray, n_cont: int, periods: int, overs: int):
    """Right-hand sides of the constraints (Eqs. phi_avar, phi_grad), one
    column per cell function r: r = i for phi_i, r = N + i d + m for phi_i^m.
    G[(j,q), i] = delta_ij int_{R_q} psi_j;
    G[(j,q), N+id+m] = delta_ij int_{R_q} (y_m - c_mj) psi_j (exact per element
    as |e| times the centroid offset)."""
    d, N = g.d, n_cont
    nq = periods ** d
    R = N * (1 + d)
    blk = g.block_of_element(periods)
    c = centroids(g, labels, N, periods, overs)
    vol = g.h ** d
    G = np.zeros((N * nq, R))
    for e in range(g.n_el):
        j = int(labels[e])
        row = j * nq + blk[e]
        G[row, j] += vol
        for m in range(d):
            G[row, N + j * d + m] += vol * (g.ecent[e, m] - c[m, j])
    return G


def prolongation(gc: Grid, gf: Grid) -> sp.csr_matrix:
    """Nested Q1 prolongation from the coarse lattice to the fine lattice
    (full node sets): value at a fine node = multilinear interpolation of the
    coarse nodal values (Sec. 3.2, V_n subset of V_1)."""
    rho = gf.n // gc.n
    d = gf.d
    rows, cols, vals = [], [], []
    for kf in range(gf.n_nodes):
        cf = gf.ncoord[kf]
        base = cf // rho
        frac = (cf - base * rho) / rho
        for b in itertools.product(range(2), repeat=d):
            w = 1.0
            cc = []
            for a in range(d):
                w *= frac[a] if b[a] else 1.0 - frac[a]
                cc.append(min(base[a] + b[a], gc.n))
            if w == 0.0:
                continue
            kc = sum(cc[a] * (gc.n + 1) ** a for a in range(d))
            rows.append(kf)
            cols.append(kc)
            vals.append(w)
    return sp.csr_matrix((vals, (rows, cols)), shape=(gf.n_nodes, gc.n_nodes))
