"""The seeded input generator (mch_inputs): a medium is one global function of position, so
RVEs that overlap see the same element values, draws are reproducible from the seed, and
labels stay below the number of continua. Both the oracle and the GPU tests rely on this."""
import numpy as np
import pytest

import mch_inputs as mi


def _overlap_pair(name, n):
    """Two neighbouring macropoints whose RVEs (side = 2 x spacing) overlap by half along x."""
    sp = 1.0 / 8
    wl = mi.small_workload(name, n_fine=n, macro_n=9, strides=(1,), rve_len=2 * sp,
                           spacing=sp, origin=0.0)
    d = wl.dim
    a = np.array([[2] * d])
    b = a.copy()
    b[0, 0] += 1
    return wl, a, b


@pytest.mark.parametrize("name,n", [("channel2d_17x17_L3", 32), ("incl2d_33x33_L4", 32),
                                    ("channel3d_9x9x9_L3", 16)])
def test_overlapping_rves_see_the_same_medium(name, n):
    wl, a, b = _overlap_pair(name, n)
    d = wl.dim
    ka, la = mi.media(wl, a, n)
    kb, lb = mi.media(wl, b, n)
    shape = (n,) * d
    ka, la = ka.reshape(shape), la.reshape(shape)     # array axes (z, y, x): x last
    kb, lb = kb.reshape(shape), lb.reshape(shape)
    half = n // 2
    # b is shifted by half an RVE along x: a's right half is b's left half
    assert np.array_equal(ka[..., half:], kb[..., :half])
    assert np.array_equal(la[..., half:], lb[..., :half])


def test_reproducible_and_seed_dependent():
    wl = mi.small_workload("channel2d_17x17_L3", n_fine=32, macro_n=9, strides=(1,))
    idx = np.array([[1, 2], [4, 4], [7, 0]])
    k1, l1 = mi.media(wl, idx, 32)
    k2, l2 = mi.media(wl, idx, 32)
    assert np.array_equal(k1, k2) and np.array_equal(l1, l2)
    k3, l3 = mi.media(mi.small_workload("channel2d_17x17_L3", n_fine=32, macro_n=9,
                                        strides=(1,), seed=wl.seed + 1), idx, 32)
    assert not np.array_equal(l1, l3)      # the per-period channel offsets are redrawn


@pytest.mark.parametrize("name", ["channel2d_17x17_L3", "incl2d_33x33_L4", "channel3d_9x9x9_L3"])
def test_labels_and_conductivities_valid(name):
    wl = mi.workload(name)
    n = 16 if wl.dim == 3 else 32
    idx = np.array([[0] * wl.dim, [wl.macro_n - 1] * wl.dim])
    k, lab = mi.media(wl, idx, n)
    assert lab.max() < wl.n_cont and lab.min() >= 0
    assert np.all(k > 0) and np.all(np.isfinite(k))
    for j in range(wl.n_cont):
        assert (lab == j).any(), f"continuum {j} absent"


def test_misaligned_rve_is_refused():
    wl = mi.small_workload("channel2d_17x17_L3", n_fine=32, macro_n=9, strides=(1,),
                           origin=0.01)
    with pytest.raises(ValueError):
        mi.media(wl, np.array([[1, 1]]), 32)


def test_entry_rel_err_sees_a_small_entry():
    """The entry-wise comparison of Gram matrices flags an error in an entry that is small
    next to its block (which the block-relative norm can hide)."""
    import numpy as np
    from util import block_rel_err, entry_rel_err
    rng = np.random.default_rng(0)
    B = rng.standard_normal((6, 6))
    E = B @ B.T + 6 * np.eye(6)
    E[0, 1] = E[1, 0] = 1e-6 * np.sqrt(E[0, 0] * E[1, 1])   # a small entry
    F = E.copy()
    F[0, 1] = F[1, 0] = E[0, 1] + 1e-8 * np.sqrt(E[0, 0] * E[1, 1])
    assert entry_rel_err(E, E) == 0.0
    assert abs(entry_rel_err(F, E) - 1e-8) < 1e-12
    # the same error is below a block norm's reach at this size (2 continua, d = 2: the 2x2
    # exchange block holds the entry together with its large diagonal)
    assert block_rel_err(F[None], E[None], 2, 2) < 2e-8
