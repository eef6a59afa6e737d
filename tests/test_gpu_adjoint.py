"""GPU backward pass (mch_backward) against the oracle's gradient and the Euler identity.

Loss L = sum over levels and points of sum_rs W[r,s] E[r,s] with seeded N(0,1) weights.
Forward and adjoint solves run to rtol = 1e-11, so the gradients are compared at 1e-8
relative (per level, in the max norm over elements)."""
import numpy as np
import pytest

import mch_inputs as mi
from oracle import adjoint, plan

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2503_01276_gb300 as mch  # noqa: E402


def _case(strides, n_fine, macro, precision, name="channel2d_17x17_L3"):
    wl = mi.small_workload(name, n_fine=n_fine, macro_n=macro, strides=strides,
                           precision=precision)
    pl = plan.level_plan(wl)
    med = [mi.media(wl, l["points"], wl.n_level(k + 1)) for k, l in enumerate(pl)]
    rng = np.random.default_rng(7)
    W = [rng.standard_normal((len(l["points"]), wl.n_rhs, wl.n_rhs)) for l in pl]
    return wl, pl, med, W


def _gpu_grad(wl, med, W, device=True):
    s = mch.Solver.from_workload(wl, rtol=1e-11)
    Es = []
    for lev in range(1, wl.n_levels + 1):
        k, l = med[lev - 1]
        s.solve_level(lev, torch.from_numpy(k).cuda(), torch.from_numpy(l).cuda())
        Es.append(s.effective_coeffs(lev))
    if device:
        Wd = [torch.from_numpy(w).cuda() for w in W]
        G = [torch.zeros(m[0].shape, dtype=torch.float64, device="cuda") for m in med]
        s.backward(Wd, G)
        G = [g.cpu().numpy() for g in G]
    else:
        G = [np.zeros(m[0].shape) for m in med]
        s.backward(W, G)
    return Es, G


@pytest.mark.parametrize("strides,n_fine,macro,precision", [
    ((1,), 32, 3, "mixed"),
    ((2, 1), 32, 3, "mixed"),
    ((4, 2, 1), 64, 5, "mixed"),
    ((4, 2, 1), 64, 5, "fp64"),
])
def test_gradient_matches_oracle(strides, n_fine, macro, precision):
    wl, pl, med, W = _case(strides, n_fine, macro, precision)
    Es, G = _gpu_grad(wl, med, W)
    fwd = adjoint.forward(wl, pl, med)
    Go = adjoint.backward(wl, pl, med, fwd, W)
    for n in range(wl.n_levels):
        err = np.abs(G[n] - Go[n]).max() / np.abs(Go[n]).max()
        assert err < 1e-8, (n + 1, err)
    # Euler identity on the GPU's own loss and gradient
    Lg = sum(float(np.sum(W[n] * Es[n])) for n in range(wl.n_levels))
    sk = sum(float(np.sum(med[n][0] * G[n])) for n in range(wl.n_levels))
    assert abs(sk - Lg) <= 1e-8 * abs(Lg)


def test_gradient_host_buffers():
    wl, pl, med, W = _case((2, 1), 32, 3, "mixed")
    _, Gd = _gpu_grad(wl, med, W, device=True)
    _, Gh = _gpu_grad(wl, med, W, device=False)
    for a, b in zip(Gd, Gh):
        assert np.abs(a - b).max() <= 1e-9 * np.abs(b).max()


def test_three_continua_gradient():
    wl, pl, med, W = _case((2, 1), 64, 3, "mixed", name="incl2d_33x33_L4")
    _, G = _gpu_grad(wl, med, W)
    fwd = adjoint.forward(wl, pl, med)
    Go = adjoint.backward(wl, pl, med, fwd, W)
    for n in range(wl.n_levels):
        err = np.abs(G[n] - Go[n]).max() / np.abs(Go[n]).max()
        assert err < 1e-8, (n + 1, err)


def test_autograd_directional_derivative():
    """loss.backward() through torch.autograd against a central difference of the loss
    along a random direction (all levels' kappa perturbed together)."""
    wl, pl, med, W = _case((2, 1), 32, 3, "mixed")
    s = mch.Solver.from_workload(wl, rtol=1e-11)
    kap = [torch.from_numpy(m[0]).cuda().requires_grad_(True) for m in med]
    lab = [torch.from_numpy(m[1]).cuda() for m in med]
    Wt = [torch.from_numpy(w).cuda() for w in W]
    Es = mch.homogenize(s, kap, lab)
    loss = sum((w * e).sum() for w, e in zip(Wt, Es))
    loss.backward()
    rng = np.random.default_rng(5)
    dirs = [torch.from_numpy(rng.standard_normal(m[0].shape)).cuda() * k.detach()
            for m, k in zip(med, kap)]
    h = 1e-6
    vals = []
    for sgn in (+1, -1):
        kp = [(k.detach() + sgn * h * dv) for k, dv in zip(kap, dirs)]
        Ep = mch.homogenize(s, kp, lab)
        vals.append(float(sum((w * e).sum() for w, e in zip(Wt, Ep))))
    fd = (vals[0] - vals[1]) / (2 * h)
    ad = float(sum((k.grad * dv).sum() for k, dv in zip(kap, dirs)))
    assert abs(fd - ad) <= 1e-5 * abs(ad)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
@pytest.mark.parametrize("strides,n_fine,macro", [((1,), 32, 3), ((2, 1), 32, 3)])
def test_gradient_with_oversampling(strides, n_fine, macro, precision):
    """E over R_p (o = 1): the level's own term is an adjoint source; oracle gradient and the
    Euler identity."""
    wl = mi.small_workload("channel2d_17x17_L3", n_fine=n_fine, macro_n=macro, strides=strides,
                           precision=precision, overs=1)
    pl = plan.level_plan(wl)
    med = [mi.media(wl, l["points"], wl.n_level(k + 1)) for k, l in enumerate(pl)]
    rng = np.random.default_rng(7)
    W = [rng.standard_normal((len(l["points"]), wl.n_rhs, wl.n_rhs)) for l in pl]
    Es, g = _gpu_grad(wl, med, W)
    loss = sum(float(np.sum(w * e)) for w, e in zip(W, Es))
    euler = sum(float(np.sum(m[0] * gg)) for m, gg in zip(med, g))
    assert abs(euler - loss) <= 1e-8 * abs(loss)
    fwd = adjoint.forward(wl, pl, med)
    ref = adjoint.backward(wl, pl, med, fwd, W)
    for lev in range(wl.n_levels):
        err = np.abs(g[lev] - ref[lev]).max() / np.abs(ref[lev]).max()
        assert err < 1e-8, (lev + 1, err)
