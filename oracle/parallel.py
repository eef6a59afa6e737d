"""Algorithm 1 of the oracle run on all host cores (test infrastructure).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: used by the test suite and by
the CPU legs of the benchmark, never by the product path.

Algorithm 1 visits the levels in order, and within a level the macropoints are
independent (each one needs only the cell functions of its parents, Eq. phiXiI_all).
``OraclePool`` therefore solves the points of one level at a time on a pool of worker
processes (spawn start method, one BLAS thread each), levels in order. Each worker runs
``cell.solve_point`` unchanged, so the arithmetic is exactly the serial oracle's.

Media and the parents' cell functions live in memory-mapped files in a temporary
directory: the main process writes every needed point's kappa and labels before any
timing, a worker writes the cell functions of the point it solved (levels 1..L-1 only;
the children read them), and the tasks and results carry only indices, effective
coefficients and times.
"""
from __future__ import annotations

import os
import pickle
import shutil
import tempfile
import time

import numpy as np

from . import cell, plan as plan_mod

_THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS",
                "VECLIB_MAXIMUM_THREADS", "NUMEXPR_NUM_THREADS")

# per worker process: job directory -> opened job state
_JOBS: dict = {}


def host_cores() -> int:
    """Cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _open_job(jobdir: str):
    st = _JOBS.get(jobdir)
    if st is not None:
        return st
    with open(os.path.join(jobdir, "job.pkl"), "rb") as f:
        meta = pickle.load(f)
    wl = meta["wl"]
    st = {"wl": wl, "plan": plan_mod.level_plan(wl), "ops": {}, "kap": {}, "lab": {},
          "phi": {}}
    for lv, (npts, ne) in meta["media_shape"].items():
        st["kap"][lv] = np.memmap(os.path.join(jobdir, f"kap{lv}.bin"), np.float64, "r",
                                  shape=(npts, ne))
        st["lab"][lv] = np.memmap(os.path.join(jobdir, f"lab{lv}.bin"), np.uint8, "r",
                                  shape=(npts, ne))
    for lv, shape in meta["phi_shape"].items():
        st["phi"][lv] = np.memmap(os.path.join(jobdir, f"phi{lv}.bin"), np.float64, "r+",
                                  shape=shape)
    _JOBS[jobdir] = st
    return st


def _solve_task(task):
    """One macropoint of one level: (level, position, E, seconds of the solve including
    the interpolation of the parents' cell functions)."""
    jobdir, lv, i, write_phi = task
    st = _open_job(jobdir)
    wl = st["wl"]
    ops = st["ops"].get(lv)
    if ops is None:
        ops = st["ops"][lv] = cell.LevelOps(wl, lv)
    kap = np.array(st["kap"][lv][i])
    lab = np.array(st["lab"][lv][i])
    t0 = time.perf_counter()
    I = None
    if lv > 1:
        I = np.zeros((ops.gf.n_nodes, wl.n_rhs))
        for (pl, pp, w) in st["plan"][lv - 1]["parents"][i]:
            I += w * st["phi"][pl][pp].T
    r = cell.solve_point(ops, kap, lab, I, overs=getattr(wl, "overs", 0))
    if write_phi and lv in st["phi"]:
        st["phi"][lv][i] = r["Phi"]
    dt = time.perf_counter() - t0
    return lv, i, r["E"], dt


class OraclePool:
    """Runs the oracle over chosen points of a workload's hierarchy on `procs` processes."""

    def __init__(self, procs: int | None = None):
        import multiprocessing as mp
        self.procs = int(procs or host_cores())
        saved = {k: os.environ.get(k) for k in _THREAD_VARS}
        for k in _THREAD_VARS:
            os.environ[k] = "1"
        try:
            self._pool = mp.get_context("spawn").Pool(self.procs)
        finally:
            for k, v in saved.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        self._dirs = []

    def close(self):
        if self._pool is not None:
            self._pool.close()
            self._pool.join()
            self._pool = None
        for d in self._dirs:
            shutil.rmtree(d, ignore_errors=True)
        self._dirs = []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def job(self, wl, needed: dict, media_fn):
        """Prepares a job: `needed` maps level -> positions to solve (callers include every
        ancestor); media_fn(level, positions) -> (kappa, labels) of those points. Writes the
        media files (untimed) and sizes the cell-function files of levels 1..L-1."""
        jobdir = tempfile.mkdtemp(prefix="mch_oracle_")
        self._dirs.append(jobdir)
        pl = plan_mod.level_plan(wl)
        media_shape, phi_shape = {}, {}
        nf = (wl.n_fine + 1) ** wl.dim
        for lv, pos in needed.items():
            pos = sorted(pos)
            npts = len(pl[lv - 1]["points"])
            ne = wl.n_level(lv) ** wl.dim
            media_shape[lv] = (npts, ne)
            kap = np.memmap(os.path.join(jobdir, f"kap{lv}.bin"), np.float64, "w+",
                            shape=(npts, ne))
            lab = np.memmap(os.path.join(jobdir, f"lab{lv}.bin"), np.uint8, "w+",
                            shape=(npts, ne))
            for s in range(0, len(pos), 256):
                chunk = pos[s:s + 256]
                k, l_ = media_fn(lv, chunk)
                kap[chunk] = k
                lab[chunk] = l_
            kap.flush()
            lab.flush()
            del kap, lab
            if lv < wl.n_levels:
                phi_shape[lv] = (npts, wl.n_rhs, nf)
                f = np.memmap(os.path.join(jobdir, f"phi{lv}.bin"), np.float64, "w+",
                              shape=phi_shape[lv])
                del f
        with open(os.path.join(jobdir, "job.pkl"), "wb") as f:
            pickle.dump({"wl": wl, "media_shape": media_shape, "phi_shape": phi_shape}, f)
        return jobdir

    def run(self, jobdir: str, wl, needed: dict, write_phi: bool = True):
        """Solves the needed points, levels in order (each level's points in parallel).
        Returns ({(level, position): E}, wall seconds, summed per-point solve seconds,
        wall seconds per level)."""
        E = {}
        t_sum = 0.0
        walls = []
        t0 = time.perf_counter()
        for lv in range(1, wl.n_levels + 1):
            pos = sorted(needed.get(lv, ()))
            if not pos:
                walls.append(0.0)
                continue
            t1 = time.perf_counter()
            tasks = [(jobdir, lv, i, write_phi) for i in pos]
            for (l_, i, e, dt) in self._pool.imap_unordered(_solve_task, tasks, chunksize=1):
                E[(l_, i)] = e
                t_sum += dt
            walls.append(time.perf_counter() - t1)
        return E, time.perf_counter() - t0, t_sum, walls


def closure(wl, targets) -> dict:
    """level -> positions: the targets and all their ancestors (Eq. phiXiI_all)."""
    pl = plan_mod.level_plan(wl)
    acc = set()
    for (lv, i) in targets:
        cell.ancestors(pl, lv, i, acc)
    out: dict = {}
    for (lv, i) in acc:
        out.setdefault(lv, set()).add(i)
    return {lv: sorted(v) for lv, v in out.items()}


def all_points(wl) -> dict:
    pl = plan_mod.level_plan(wl)
    return {lv + 1: list(range(len(l["points"]))) for lv, l in enumerate(pl)}
