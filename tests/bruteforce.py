"""Dense brute-force restatement of the cell problems for tiny grids.

Written independently of ``oracle``: the element stiffness comes from the
closed-form integrals of products of 1D hat functions (not quadrature), the
coarse-to-fine embedding is built by evaluating the coarse Q1 basis at fine
node coordinates, the constraint functionals are integrated element by
element in closed form, and the saddle-point system is solved as one dense
linear system with numpy.linalg.solve. Used only to pin the oracle.
"""
from __future__ import annotations

import itertools

import numpy as np


def khat_closed_form(d):
    """int_{[0,1]^d} grad N_a . grad N_b in closed form: per axis, the 1D
    stiffness is [[1,-1],[-1,1]] and the 1D mass [[1/3,1/6],[1/6,1/3]]."""
    k1 = np.array([[1.0, -1.0], [-1.0, 1.0]])
    m1 = np.array([[1 / 3, 1 / 6], [1 / 6, 1 / 3]])
    cs = list(itertools.product(range(2), repeat=d))
    K = np.zeros((len(cs), len(cs)))
    for i, a in enumerate(cs):
        for j, b in enumerate(cs):
            tot = 0.0
            for ax in range(d):
                t = k1[a[ax], b[ax]]
                for o in range(d):
                    if o != ax:
                        t *= m1[a[o], b[o]]
                tot += t
            K[i, j] = tot
    return cs, K


def node_id(c, n):
    return sum(c[a] * (n + 1) ** a for a in range(len(c)))


def el_id(e, n):
    return sum(e[a] * n ** a for a in range(len(e)))


def in_region(e, n, P, overs):
    """Element e lies in the central (P - 2 overs)^d periods."""
    m = n // P
    return all(overs * m <= e[a] < (P - overs) * m for a in range(len(e)))


def dense_system(d, n, L, kappa, labels, N, P, overs=0):
    """Dense A on all (n+1)^d nodes, constraint rows C (all (j,q) rows) and
    targets G (all rows), plus the interior mask. kappa/labels are flat with
    x fastest. With overs > 0 the centroids are taken over the central
    (P - 2 overs)^d periods (over the whole RVE if a continuum is absent there)."""
    h = L / n
    cs, K = khat_closed_form(d)
    nn = (n + 1) ** d
    A = np.zeros((nn, nn))
    nq = P ** d
    m = n // P
    C = np.zeros((N * nq, nn))
    vol = h ** d
    sums = np.zeros((N, d))
    cnt = np.zeros(N)
    sums_all = np.zeros((N, d))
    cnt_all = np.zeros(N)
    for e in itertools.product(range(n), repeat=d):
        eid = el_id(e, n)
        j = int(labels[eid])
        y = np.array([-L / 2 + (e[a] + 0.5) * h for a in range(d)])
        sums_all[j] += y
        cnt_all[j] += 1
        if in_region(e, n, P, overs):
            sums[j] += y
            cnt[j] += 1
    use = cnt > 0
    sums = np.where(use[:, None], sums, sums_all)
    cnt = np.where(use, cnt, cnt_all)
    cen = np.where(cnt[:, None] > 0, sums / np.maximum(cnt, 1)[:, None], 0.0)
    G = np.zeros((N * nq, N * (1 + d)))
    for e in itertools.product(range(n), repeat=d):
        eid = el_id(e, n)
        ids = [node_id(tuple(e[a] + c[a] for a in range(d)), n) for c in cs]
        A[np.ix_(ids, ids)] += kappa[eid] * h ** (d - 2) * K
        j = int(labels[eid])
        q = sum((e[a] // m) * P ** a for a in range(d))
        row = j * nq + q
        for i in ids:
            C[row, i] += vol / 2 ** d
        G[row, j] += vol
        y = np.array([-L / 2 + (e[a] + 0.5) * h for a in range(d)])
        for mm in range(d):
            G[row, N + j * d + mm] += vol * (y[mm] - cen[j, mm])
    mask = np.zeros(nn, dtype=bool)
    for c in itertools.product(range(n + 1), repeat=d):
        if all(0 < c[a] < n for a in range(d)):
            mask[node_id(c, n)] = True
    return A, C, G, mask


def coarse_basis_at_fine(d, nc, nf):
    """Matrix whose column k is the coarse Q1 basis function of coarse node k
    evaluated at every fine node (both full lattices)."""
    Pm = np.zeros(((nf + 1) ** d, (nc + 1) ** d))
    for cf in itertools.product(range(nf + 1), repeat=d):
        xf = np.array(cf, dtype=float) / nf
        for cc in itertools.product(range(nc + 1), repeat=d):
            xc = np.array(cc, dtype=float) / nc
            w = np.prod(np.maximum(0.0, 1.0 - np.abs(xf - xc) * nc))
            if w:
                Pm[node_id(cf, nf), node_id(cc, nc)] = w
    return Pm


def kkt_solve(A, C, b, g):
    """One dense solve of [A -C^T; C 0][x; beta] = [b; g]."""
    n, k = A.shape[0], C.shape[0]
    K = np.zeros((n + k, n + k))
    K[:n, :n] = A
    K[:n, n:] = -C.T
    K[n:, :n] = C
    sol = np.linalg.solve(K, np.vstack([b, g]))
    return sol[:n], sol[n:]


def cell_E(d, n, L, kappa, labels, N, P, overs=0):
    """Level-1 effective coefficients by the dense KKT solve; with overs > 0 the energy is
    integrated over the central (P - 2 overs)^d periods and divided by their volume."""
    A, C, G, mask = dense_system(d, n, L, kappa, labels, N, P, overs)
    Ai = A[np.ix_(mask, mask)]
    Ci = C[:, mask]
    keep = np.abs(Ci).sum(axis=1) > 0
    x, beta = kkt_solve(Ai, Ci[keep], np.zeros((mask.sum(), G.shape[1])), G[keep])
    Phi = np.zeros((A.shape[0], G.shape[1]))
    Phi[mask] = x
    if overs == 0:
        return Phi.T @ A @ Phi / L ** d, Phi
    h = L / n
    cs, K = khat_closed_form(d)
    Ar = np.zeros_like(A)
    ne = 0
    for e in itertools.product(range(n), repeat=d):
        if not in_region(e, n, P, overs):
            continue
        ne += 1
        ids = [node_id(tuple(e[a] + c[a] for a in range(d)), n) for c in cs]
        Ar[np.ix_(ids, ids)] += kappa[el_id(e, n)] * h ** (d - 2) * K
    return Phi.T @ Ar @ Phi / (ne * h ** d), Phi


def child_E(d, nf, nc, L, kappa_c, labels_c, N, P, I):
    """Correction problem of a child with a coarse grid nc and interpolant I
    (fine full lattice, [nodes, R]) by a dense KKT solve on the fine grid:
    min (I + Pm xi)^T A_f (I + Pm xi) subject to C_f (I + Pm xi) = G."""
    rho = nf // nc
    # child's medium prolonged piecewise-constantly to the fine grid
    kf = np.zeros(nf ** d)
    lf = np.zeros(nf ** d, dtype=np.int64)
    for e in itertools.product(range(nf), repeat=d):
        ec = tuple(e[a] // rho for a in range(d))
        kf[el_id(e, nf)] = kappa_c[el_id(ec, nc)]
        lf[el_id(e, nf)] = labels_c[el_id(ec, nc)]
    Af, Cf, Gf, maskf = dense_system(d, nf, L, kf, lf, N, P)
    Pm = coarse_basis_at_fine(d, nc, nf)
    _, _, _, maskc = dense_system(d, nc, L, kappa_c, labels_c, N, P)
    Pm = Pm[:, maskc]
    AX = Pm.T @ Af @ Pm
    CX = Cf @ Pm
    keep = np.abs(CX).sum(axis=1) > 1e-300
    b = -Pm.T @ Af @ I
    g = (Gf - Cf @ I)[keep]
    xi, beta = kkt_solve(AX, CX[keep], b, g)
    Phi = I + Pm @ xi
    return Phi.T @ Af @ Phi / L ** d, Phi
