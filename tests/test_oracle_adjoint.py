"""Pins of the oracle's gradient: central finite differences of the loss on elements of
every level (the loss is recomputed through the whole hierarchy, so a parent's kappa
reaches its children's coefficients), and the Euler identity sum kappa dL/dkappa = L, which
holds because every effective coefficient is 1-homogeneous in kappa jointly over levels
(scaling all kappa leaves every cell function unchanged, Sec. 3, Eq. phi_abstract)."""
import numpy as np
import pytest

import mch_inputs as mi
from oracle import adjoint, plan


def _setup(strides, n_fine, macro, seed=7, overs=0):
    wl = mi.small_workload("channel2d_17x17_L3", n_fine=n_fine, macro_n=macro,
                           strides=strides, overs=overs)
    pl = plan.level_plan(wl)
    med = [mi.media(wl, l["points"], wl.n_level(k + 1)) for k, l in enumerate(pl)]
    rng = np.random.default_rng(seed)
    W = [rng.standard_normal((len(l["points"]), wl.n_rhs, wl.n_rhs)) for l in pl]
    return wl, pl, med, W


def _loss(wl, pl, med, W):
    return adjoint.loss(adjoint.forward(wl, pl, med), W)


@pytest.mark.parametrize("strides,n_fine,macro,overs", [((1,), 16, 3, 0), ((2, 1), 16, 3, 0),
                                                        ((4, 2, 1), 64, 5, 0),
                                                        ((1,), 16, 3, 1), ((2, 1), 32, 3, 1)])
def test_euler_identity(strides, n_fine, macro, overs):
    wl, pl, med, W = _setup(strides, n_fine, macro, overs=overs)
    fwd = adjoint.forward(wl, pl, med)
    Lv = adjoint.loss(fwd, W)
    g = adjoint.backward(wl, pl, med, fwd, W)
    s = sum(float(np.sum(med[n][0] * g[n])) for n in range(len(pl)))
    assert abs(s - Lv) <= 1e-10 * abs(Lv)


@pytest.mark.parametrize("strides,n_fine,macro,overs", [((1,), 16, 3, 0), ((2, 1), 16, 3, 0),
                                                        ((4, 2, 1), 64, 5, 0),
                                                        ((1,), 16, 3, 1), ((2, 1), 32, 3, 1)])
def test_central_differences(strides, n_fine, macro, overs):
    """Central differences with relative step 1e-6 on three elements of every level. The
    oracle solves its saddle systems to ~1e-14 (FP64 refinement), so a loss value is accurate
    to ~1e-14 sum |W||E| and a central difference to ~1e-14 sum |W||E| / h; the allowance is
    100 times that (the Euler identity does not pin the hierarchical part of the gradient:
    scaling every kappa leaves the cell functions unchanged, so the terms through the parents'
    functions cancel in it; these differences do)."""
    wl, pl, med, W = _setup(strides, n_fine, macro, overs=overs)
    fwd = adjoint.forward(wl, pl, med)
    g = adjoint.backward(wl, pl, med, fwd, W)
    swe = sum(float(np.sum(np.abs(W[n]) * np.abs(np.array([r["E"] for r in fwd[n]]))))
              for n in range(len(pl)))
    rng = np.random.default_rng(11)
    checked = 0
    for n in range(len(pl)):
        kap, lab = med[n]
        npts, ne = kap.shape
        for _ in range(3):
            i = int(rng.integers(npts))
            e = int(rng.integers(ne))
            h = 1e-6 * kap[i, e]
            out = []
            for sgn in (+1, -1):
                k2 = [m[0].copy() for m in med]
                k2[n][i, e] += sgn * h
                out.append(_loss(wl, pl, [(k2[q], med[q][1]) for q in range(len(pl))], W))
            fd = (out[0] - out[1]) / (2 * h)
            scale = max(abs(g[n][i, e]), 1e-6 * np.abs(g[n]).max())
            assert abs(fd - g[n][i, e]) <= 1e-5 * scale + 1e-12 * swe / h, (n, i, e, fd, g[n][i, e])
            checked += 1
    assert checked == 3 * len(pl)


def test_sampled_backward_matches_full_backward():
    """The closure-restricted reverse sweep (weights on two points only) reproduces the full
    sweep's gradient on every point of the closure and zero elsewhere."""
    wl = mi.small_workload("channel2d_17x17_L3", n_fine=32, macro_n=5, strides=(4, 2, 1),
                           precision="fp64")
    pl = plan.level_plan(wl)
    med = [mi.media(wl, l["points"], wl.n_level(k + 1)) for k, l in enumerate(pl)]
    rng = np.random.default_rng(3)
    R = wl.n_rhs
    picks = {(3, 5): rng.standard_normal((R, R)), (2, 1): rng.standard_normal((R, R))}
    W = [np.zeros((len(l["points"]), R, R)) for l in pl]
    for (lv, i), w in picks.items():
        W[lv - 1][i] = w
    fwd = adjoint.forward(wl, pl, med)
    full = adjoint.backward(wl, pl, med, fwd, W)

    def media_fn(lv, pos):
        return mi.media(wl, pl[lv - 1]["points"][pos], wl.n_level(lv))

    samp, loss_s = adjoint.backward_sampled(wl, pl, media_fn, picks)
    assert abs(loss_s - adjoint.loss(fwd, W)) <= 1e-12 * abs(loss_s)
    for lv in range(1, 4):
        for i in range(len(pl[lv - 1]["points"])):
            g = full[lv - 1][i]
            if (lv, i) in samp:
                assert np.abs(samp[(lv, i)] - g).max() <= 1e-10 * np.abs(g).max()
            else:
                assert not np.any(g)
