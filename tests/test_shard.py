"""A hierarchy split over ranks (paper_2503_01276_gb300.shard) on CPU: contiguous balanced
point ranges per level, one all-gather of the level's cell functions per level, the
coefficients gathered at the end. Two and three gloo ranks, each solving its ranges with the
FP64 oracle as the per-rank backend, reproduce the single-process oracle hierarchy exactly
(the exchange and the import must deliver every parent's cell functions to the rank that
needs them)."""
import os
import socket
import sys

import numpy as np
import pytest

import mch_inputs as mi
from oracle import cell, plan
from paper_2503_01276_gb300 import shard

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _workload():
    return mi.small_workload("channel2d_17x17_L3", n_fine=64, macro_n=9, strides=(4, 2, 1),
                             precision="fp64")


class OracleBackend:
    """The oracle's per-point solve behind the backend interface of the sharded driver."""

    def __init__(self, wl):
        self.wl = wl
        self.pl = plan.level_plan(wl)
        self.phi, self.E = {}, {}

    def _arrays(self, level):
        n = len(self.pl[level - 1]["points"])
        nodes = (self.wl.n_fine + 1) ** self.wl.dim
        R = self.wl.n_rhs
        if level not in self.phi:
            self.phi[level] = np.zeros((n, R, nodes))
            self.E[level] = np.full((n, R, R), np.nan)
        return self.phi[level], self.E[level]

    def num_points(self, level):
        return len(self.pl[level - 1]["points"])

    def solve_range(self, level, p0, p1, kappa, labels):
        phi, E = self._arrays(level)
        if p1 == p0:
            return
        ops = cell.LevelOps(self.wl, level)
        for k, i in enumerate(range(p0, p1)):
            I = None
            if level > 1:
                I = sum(w * self.phi[a][b].T for (a, b, w) in self.pl[level - 1]["parents"][i])
            r = cell.solve_point(ops, kappa[k], labels[k], I)
            phi[i], E[i] = r["Phi"], r["E"]

    def cell_functions(self, level, p0, p1):
        return self.phi[level][p0:p1].copy()

    def set_cell_functions(self, level, p0, p1, phi):
        self._arrays(level)[0][p0:p1] = phi

    def effective_coeffs(self, level, p0, p1):
        return self.E[level][p0:p1].copy()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl = _workload()
    be = OracleBackend(wl)
    pl = be.pl

    def media(level, p0, p1):
        return mi.media(wl, pl[level - 1]["points"][p0:p1], wl.n_level(level))

    sh = shard.ShardedHierarchy(be, wl.n_levels, world, rank, media)
    E = sh.run(shard.TorchComm())
    # what this rank imported: every point of the earlier levels has cell functions
    imported = all(np.abs(be.phi[l]).sum(axis=(1, 2)).min() > 0 for l in range(1, wl.n_levels))
    out.put((rank, E, imported))
    dist.barrier()
    dist.destroy_process_group()


def test_partition_is_contiguous_and_balanced():
    for n, w in [(9, 2), (72, 3), (208, 8), (3, 4), (0, 2)]:
        r = shard.partition(n, w)
        assert r[0][0] == 0 and r[-1][1] == n
        assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
        sizes = [p1 - p0 for p0, p1 in r]
        assert max(sizes) - min(sizes) <= 1


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_oracle_matches_serial(world):
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    wl = _workload()
    pl = plan.level_plan(wl)
    med = [mi.media(wl, l["points"], wl.n_level(k + 1)) for k, l in enumerate(pl)]
    ref = cell.run_hierarchy(wl, pl, med, keep_phi=False)
    for rank, E, imported in res:
        assert imported, rank
        for lev in range(wl.n_levels):
            Er = ref[lev]["E"]
            assert E[lev].shape == Er.shape
            assert np.abs(E[lev] - Er).max() <= 1e-12 * np.abs(Er).max(), (rank, lev)
