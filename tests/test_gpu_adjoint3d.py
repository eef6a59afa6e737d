"""3D backward pass against the oracle's gradient and the Euler identity (grids 16/8,
2x2x2 periods, mixed and FP64, rtol 1e-11; and with oversampling, o = 1 of 4x4x4 periods,
where the level's own term is an adjoint source)."""
import numpy as np
import pytest

import mch_inputs as mi
from oracle import adjoint, plan

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2503_01276_gb300 as mch  # noqa: E402


@pytest.mark.parametrize("precision,overs", [("mixed", 0), ("fp64", 0), ("mixed", 1),
                                             ("fp64", 1)])
def test_3d_gradient_vs_oracle(precision, overs):
    if overs:
        wl = mi.small_workload("channel3d_9x9x9_L3", n_fine=16, macro_n=3, strides=(2, 1),
                               periods=4, eta=1, overs=1, precision=precision)
    else:
        wl = mi.small_workload("channel3d_9x9x9_L3", n_fine=16, macro_n=3, strides=(2, 1),
                               periods=2, precision=precision)
    pl = plan.level_plan(wl)
    med = [mi.media(wl, l["points"], wl.n_level(k + 1)) for k, l in enumerate(pl)]
    rng = np.random.default_rng(7)
    W = [rng.standard_normal((len(l["points"]), wl.n_rhs, wl.n_rhs)) for l in pl]
    s = mch.Solver.from_workload(wl, rtol=1e-11)
    loss = 0.0
    for lev in range(1, wl.n_levels + 1):
        k, l = med[lev - 1]
        s.solve_level(lev, torch.from_numpy(k).cuda(), torch.from_numpy(l).cuda())
        loss += float(np.sum(W[lev - 1] * s.effective_coeffs(lev)))
    Wd = [torch.from_numpy(w).cuda() for w in W]
    G = [torch.zeros(m[0].shape, dtype=torch.float64, device="cuda") for m in med]
    s.backward(Wd, G)
    g = [t.cpu().numpy() for t in G]
    euler = sum(float(np.sum(m[0] * gg)) for m, gg in zip(med, g))
    assert abs(euler - loss) <= 1e-8 * abs(loss)
    fwd = adjoint.forward(wl, pl, med)
    ref = adjoint.backward(wl, pl, med, fwd, W)
    for lev in range(wl.n_levels):
        err = np.abs(g[lev] - ref[lev]).max() / np.abs(ref[lev]).max()
        assert err < 1e-8, (lev + 1, err)
