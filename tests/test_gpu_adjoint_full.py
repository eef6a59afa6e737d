"""Backward pass at full size: the 2D channel medium at contrast 1e5 on 65x65 macropoints,
three levels (289/800/3136 points on RVE grids 128/64/32), mixed precision.

Loss L = sum over all points of sum W[r,s] E[r,s] with seeded N(0,1) weights on the upper
triangles of the exchange block (N x N) and of the permeability block (Nd x Nd). Checked:
the Euler identity; checkpointed vs recomputed cell functions; the oracle's gradient on the
closure of a few weighted points; central differences on 64 seeded elements, stratified by
continuum and spread over the levels."""
import numpy as np
import pytest

import mch_inputs as mi
from oracle import adjoint, plan

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2503_01276_gb300 as mch  # noqa: E402

WL = mi.workload("channel2d_65x65_L3_adj")
RTOL = 1e-11


@pytest.fixture(scope="module")
def case():
    pl = plan.level_plan(WL)
    med = [mi.media(WL, l["points"], WL.n_level(k + 1)) for k, l in enumerate(pl)]
    N, d, R = WL.n_cont, WL.dim, WL.n_rhs
    mask = np.zeros((R, R))
    mask[np.triu_indices(N)] = 1.0
    iu = np.triu_indices(N * d)
    mask[N + iu[0], N + iu[1]] = 1.0
    rng = np.random.default_rng(7)
    W = [rng.standard_normal((len(l["points"]), R, R)) * mask for l in pl]
    return pl, med, W, mask


def _solve(s, med):
    Es = []
    for lev in range(1, WL.n_levels + 1):
        k, l = med[lev - 1]
        s.solve_level(lev, k, l)
        E = torch.zeros((k.shape[0], s.R, s.R), dtype=torch.float64, device="cuda")
        s.effective_coeffs(lev, E)
        Es.append(E)
    return Es


def _grad(s, W):
    Wd = [torch.from_numpy(w).cuda() for w in W]
    G = [torch.zeros((w.shape[0], s.n_elem(l + 1) ** 2), dtype=torch.float64, device="cuda")
         for l, w in enumerate(W)]
    s.backward(Wd, G)
    return [g.cpu().numpy() for g in G]


def _dev_media(med):
    return [(torch.from_numpy(k).cuda(), torch.from_numpy(l).cuda()) for k, l in med]


def test_euler_identity_and_recompute(case):
    pl, med, W, _ = case
    md = _dev_media(med)
    s = mch.Solver.from_workload(WL, rtol=RTOL, keep_parents=1)
    Es = _solve(s, md)
    loss = sum(float((torch.from_numpy(w).cuda() * e).sum()) for w, e in zip(W, Es))
    g1 = _grad(s, W)
    euler = sum(float((k * g).sum()) for (k, _), g in zip(med, g1))
    assert abs(euler - loss) <= 1e-8 * abs(loss), (euler, loss)
    s.close()

    # recompute: the level-1-grid cell functions are freed after the last level and rebuilt
    # from the level-grid solutions for the backward pass
    s2 = mch.Solver.from_workload(WL, rtol=RTOL, keep_parents=0)
    _solve(s2, md)
    g2 = _grad(s2, W)
    for a, b in zip(g1, g2):
        assert np.abs(a - b).max() <= 1e-9 * np.abs(a).max()
    # after mch_backward the cell functions are freed again; reading them rebuilds them
    torch.cuda.synchronize()
    free_released = torch.cuda.mem_get_info()[0]
    phi1 = np.empty((s2.num_points(1), s2.R, (WL.n_fine + 1) ** 2))
    s2.cell_functions(1, phi1)
    torch.cuda.synchronize()
    free_restored = torch.cuda.mem_get_info()[0]
    phi_bytes = sum(s2.num_points(l) for l in (1, 2, 3)) * s2.R * (WL.n_fine + 1) ** 2 * 8
    assert 0.9 * phi_bytes <= free_released - free_restored <= 1.2 * phi_bytes + (64 << 20)
    s2.close()


def test_oracle_gradient_on_sampled_closure(case):
    pl, med, W, mask = case
    rng = np.random.default_rng(13)
    par3 = pl[2]["parents"]
    p3 = next(i for i in range(len(par3) // 2, len(par3)) if len(par3[i]) == 4)
    par2 = pl[1]["parents"]
    p2 = next(i for i in range(len(par2) // 3, len(par2)) if len(par2[i]) == 4)
    picks = {(3, p3): rng.standard_normal((WL.n_rhs, WL.n_rhs)) * mask,
             (2, p2): rng.standard_normal((WL.n_rhs, WL.n_rhs)) * mask,
             (1, 100): rng.standard_normal((WL.n_rhs, WL.n_rhs)) * mask}
    Wp = [np.zeros_like(w) for w in W]
    for (lv, i), w in picks.items():
        Wp[lv - 1][i] = w

    def media_fn(lv, pos):
        return mi.media(WL, pl[lv - 1]["points"][pos], WL.n_level(lv))

    ref, loss_ref = adjoint.backward_sampled(WL, pl, media_fn, picks)
    s = mch.Solver.from_workload(WL, rtol=RTOL)
    Es = _solve(s, _dev_media(med))
    loss = sum(float((torch.from_numpy(w).cuda() * e).sum()) for w, e in zip(Wp, Es))
    assert abs(loss - loss_ref) <= 1e-9 * abs(loss_ref)
    g = _grad(s, Wp)
    for lv in range(1, 4):
        for i in range(len(pl[lv - 1]["points"])):
            if (lv, i) in ref:
                r = ref[(lv, i)]
                err = np.abs(g[lv - 1][i] - r).max() / np.abs(r).max()
                assert err <= 1e-8, (lv, i, err)
            else:
                assert not np.any(g[lv - 1][i]), (lv, i)
    s.close()


def _descendants(pl):
    kids = {}
    for n in range(1, len(pl)):
        for i, par in enumerate(pl[n]["parents"]):
            for (lv, pos, _) in par:
                kids.setdefault((lv, pos), []).append((n + 1, i))

    def closure(key):
        out, stack = {key}, [key]
        while stack:
            for c in kids.get(stack.pop(), []):
                if c not in out:
                    out.add(c)
                    stack.append(c)
        return out
    return closure


@pytest.mark.parametrize("h,trunc,informative_min,informative_frac", [
    (1e-4, 1e-5, 24, 1e-3), (1e-6, 1e-6, 8, 1e-2)])
def test_central_differences_64_elements(case, h, trunc, informative_min, informative_frac):
    """Relative steps 1e-4 (the O(h^2) truncation is ~1e-8 of the derivative) and 1e-6 (the
    step of the workload's description; the truncation is negligible, the solves' noise is
    100x larger relative to the signal). Only the perturbed point and its descendants are
    re-read. The solves run at rtol 1e-12; a child's coefficients inherit about rtol of its
    parents' cell functions, so the allowance for the noise of the difference of two solves
    is 2 rtol of the affected weighted coefficients sum |W||E|, plus `trunc` of the
    derivative; a minimum number of the 64 elements must have a noise allowance below
    `informative_frac` of their derivative."""
    pl, med, W, _ = case
    closure = _descendants(pl)
    rng = np.random.default_rng(11)
    picks = []
    for lv, cnt in ((1, 22), (2, 21), (3, 21)):
        k, lab = med[lv - 1]
        for c in range(cnt):
            want = c % 2           # alternate channel (label 0) and matrix (label 1)
            while True:
                p = int(rng.integers(k.shape[0]))
                e = int(rng.integers(k.shape[1]))
                if lab[p, e] == want:
                    break
            picks.append((lv, p, e))
    rtol_fd = 1e-12
    s = mch.Solver.from_workload(WL, rtol=rtol_fd)
    md = _dev_media(med)
    _solve(s, md)
    g = _grad(s, W)
    rel = []
    for (lv, p, e) in picks:
        aff = closure((lv, p))
        vals = []
        for sgn in (1.0, -1.0):
            kp = md[lv - 1][0].clone()
            kp[p, e] *= 1.0 + sgn * h
            Ev = {}
            for lev in range(lv, WL.n_levels + 1):
                kk = kp if lev == lv else md[lev - 1][0]
                s.solve_level(lev, kk, md[lev - 1][1])
                E = s.effective_coeffs(lev)
                for (l2, i2) in aff:
                    if l2 == lev:
                        Ev[(l2, i2)] = E[i2]
            vals.append(Ev)
        for lev in range(lv, WL.n_levels + 1):
            s.solve_level(lev, *md[lev - 1])
        dL = sum(float(np.sum(W[l2 - 1][i2] * (vals[0][(l2, i2)] - vals[1][(l2, i2)])))
                 for (l2, i2) in aff)
        scale = sum(float(np.sum(np.abs(W[l2 - 1][i2] * vals[0][(l2, i2)]))) for (l2, i2) in aff)
        kap = med[lv - 1][0][p, e]
        fd = dL / (2 * h * kap)
        ad = g[lv - 1][p, e]
        noise = 2 * rtol_fd * scale / (2 * h * kap)
        rel.append((lv, int(med[lv - 1][1][p, e]), fd, ad, noise))
        assert abs(fd - ad) <= trunc * abs(ad) + noise, (lv, p, e, fd, ad, noise)
    informative = sum(1 for (_, _, fd, ad, nz) in rel if nz < informative_frac * abs(ad))
    print(f"h {h}: FD elements where the noise floor is below {informative_frac} of the "
          f"derivative: {informative} of {len(rel)}")
    for r in rel:
        print("level %d label %d fd %.6e ad %.6e noise %.1e" % r)
    assert informative >= informative_min
    s.close()
