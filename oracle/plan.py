"""Level plan of the hierarchical macrogrid (oracle).

Sec. 3.1, Eq. (defi_Sn): nested macrogrids T_1 c T_2 c ... c T_L = T, here
T_n = the macro indices that are multiples of stride_n along every axis, and
S_1 = T_1, S_n = T_n minus T_{n-1}. Points of S_n are listed lexicographically
with x fastest.

Sec. 3.3, Eq. (phiXiI_all): a point of S_n (n > 1) inherits from neighbouring
points of the earlier levels with weights c_t summing to one. Reading taken
here: the neighbours are the vertices of the T_{n-1} cell that contains the
point, with multilinear interpolation weights; along an axis where the point
lies on a T_{n-1} grid line only that line's vertex is used.
"""
from __future__ import annotations

import itertools

import numpy as np


def macro_indices(M: int, d: int) -> np.ndarray:
    """All macro indices of the M^d grid, x fastest."""
    grids = [np.arange(M)] * d
    pts = np.array(list(itertools.product(*grids[::-1])))[:, ::-1]
    return pts.astype(np.int64)


def level_plan(wl):
    """Returns a list over levels n = 1..L of dicts with
    'points': int [npts, d] macro indices of S_n,
    'parents': list per point of [(level, position, weight)] (empty at n = 1).
    """
    M, d, strides = wl.macro_n, wl.dim, tuple(wl.strides)
    if strides[-1] != 1:
        raise ValueError("the last level must contain every macropoint (stride 1)")
    for s_prev, s in zip(strides[:-1], strides[1:]):
        if s_prev % s:
            raise ValueError("strides must be nested")
    if (M - 1) % strides[0]:
        raise ValueError("the coarsest macrogrid must cover the whole index range")
    allp = macro_indices(M, d)
    levels = []
    where = {}
    prev_mask = np.zeros(len(allp), dtype=bool)
    for n, s in enumerate(strides):
        mask_T = np.all(allp % s == 0, axis=1)
        mask_S = mask_T & ~prev_mask
        pts = allp[mask_S]
        for pos, p in enumerate(pts):
            where[tuple(p)] = (n + 1, pos)
        parents = []
        if n > 0 and getattr(wl, "interp", "multilinear") == "nearest1":
            # Sec. 3.3, the choice of the numerical experiments: I_p = Phi_t with x_t the
            # nearest point of S_1 (= T_1), weight one; ties to the lower index
            s1 = strides[0]
            for p in pts:
                q = tuple(int((i // s1) * s1 + (s1 if 2 * (i % s1) > s1 else 0)) for i in p)
                lev, pos = where[q]
                parents.append([(lev, pos, 1.0)])
        elif n > 0:
            sp_ = strides[n - 1]
            for p in pts:
                axes = []
                for a in range(d):
                    i = int(p[a])
                    if i % sp_ == 0:
                        axes.append([(i, 1.0)])
                    else:
                        lo = (i // sp_) * sp_
                        f = (i - lo) / sp_
                        axes.append([(lo, 1.0 - f), (lo + sp_, f)])
                plist = []
                for combo in itertools.product(*axes):
                    q = tuple(c[0] for c in combo)
                    w = float(np.prod([c[1] for c in combo]))
                    lev, pos = where[q]
                    plist.append((lev, pos, w))
                parents.append(plist)
        levels.append({"points": pts, "parents": parents})
        prev_mask = mask_T
    return levels
