"""A hierarchy split over ranks, through the library (mch_solve_level_range and
mch_set_cell_functions): two and three handles on this GPU stand for the ranks and run in
lockstep in one process, each solving its contiguous point range of every level and
importing the other ranges' cell functions before the next level (the exchange step of
paper_2503_01276_gb300.shard, here by host copies between the handles; no kernel of one
handle waits for another). The gathered coefficients equal the single-handle hierarchy and
the oracle."""
import numpy as np
import pytest

import mch_inputs as mi
from oracle import cell, plan
from paper_2503_01276_gb300 import shard
from util import block_rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2503_01276_gb300 as mch  # noqa: E402


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_sharded_handles_match_single_handle(world, precision):
    wl = mi.small_workload("channel2d_17x17_L3", n_fine=64, macro_n=9, strides=(4, 2, 1),
                           precision=precision)
    pl = plan.level_plan(wl)

    def media(level, p0, p1):
        k, l = mi.media(wl, pl[level - 1]["points"][p0:p1], wl.n_level(level))
        return torch.from_numpy(k).cuda(), torch.from_numpy(l).cuda()

    single = mch.Solver.from_workload(wl, rtol=1e-11)
    E1 = []
    for lev in range(1, wl.n_levels + 1):
        single.solve_level(lev, *media(lev, 0, len(pl[lev - 1]["points"])))
        E1.append(single.effective_coeffs(lev))
    single.close()

    handles = [mch.Solver.from_workload(wl, rtol=1e-11) for _ in range(world)]
    shards = [shard.ShardedHierarchy(shard.LibraryBackend(h), wl.n_levels, world, r, media)
              for r, h in enumerate(handles)]
    for lev in range(1, wl.n_levels + 1):
        items = [s.solve_own(lev) for s in shards]
        if lev < wl.n_levels:
            for s in shards:
                s.import_level(lev, items)
    E = shard.assemble([s.own_coeffs() for s in shards], wl.n_levels)
    med = [mi.media(wl, l["points"], wl.n_level(k + 1)) for k, l in enumerate(pl)]
    ref = cell.run_hierarchy(wl, pl, med, keep_phi=False)
    for lev in range(wl.n_levels):
        assert block_rel_err(E[lev], E1[lev], wl.n_cont, wl.dim) < 1e-9, lev
        assert block_rel_err(E[lev], ref[lev]["E"], wl.n_cont, wl.dim) < 1e-9, lev
    # the backward pass needs every point on one handle
    with pytest.raises(mch.MchError):
        R = wl.n_rhs
        W = [torch.zeros((len(l["points"]), R, R), dtype=torch.float64, device="cuda")
             for l in pl]
        G = [torch.zeros((len(l["points"]), wl.n_level(k + 1) ** 2), dtype=torch.float64,
                         device="cuda") for k, l in enumerate(pl)]
        handles[0].backward(W, G)
    for h in handles:
        h.close()
