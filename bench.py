"""Benchmark: cell-problem right-hand sides solved per second on the 2D four-level
hierarchy with three continua (33x33 macropoints, levels of 25/56/208/800 points on RVE
grids 256/128/64/32, nine cell functions per point, channel contrast 1e6, FP32 PCG inside
FP64 refinement), the largest single-GPU workload of the suite.

One step solves every level of the hierarchy through the library (mch_prepare_level and
mch_solve_level per level: constraint data, interpolation and correction right-hand sides,
batched constrained solves, cell-function assembly and effective coefficients), with the
media already resident in device memory. The L2 cache is flushed (a 512 MB device write,
outside the timed event pairs) before every timed step.

JSON line keys beyond the base contract:
  roofline      the persistent level kernel k_level2d (the time sink; all of a level's
                (point, function) units in one launch): the algorithmic bytes of its
                multi-RHS stencil applies, n^d 4 B of FP32 kappa per apply shared by the R
                functions plus (n-1)^d x 2 x 4 B of FP32 vector in and out per function, over
                its CUDA-event time, against the measured HBM copy bandwidth. The kernel keeps
                its state on chip, so this is the rate an HBM-streaming apply would need to
                match it; DRAM traffic per launch from ncu is beside it, and "alu" gives the
                FP32 flop rate against the FP32 FMA rate.
  cpu_baseline  the FP64 oracle (SciPy sparse LU + Schur complement + FP64 refinement) over
                EVERY point of the workload, levels in order, on all host cores (one worker
                process per core, one BLAS thread each); `single_core_s` is the sum of the
                per-point solve times measured inside the workers.
  accuracy      largest final projected-residual ratio, and the block-relative error of the
                GPU coefficients against the oracle over every point.
  e2e           the same step through the public API with pinned host buffers (media copied
                in, effective coefficients copied out) inside the timed region.
  configs       one record per other workload of the suite (2D single level FP64; 2D three
                levels FP64 and mixed; 3D three levels; the 65x65 adjoint workload with its
                backward pass): RHS/s, e2e, roofline, accuracy against the oracle (every point,
                or sampled points of every level with 1, 2 and 4 parents), and for the adjoint
                workload the backward time with checkpointed and recomputed parents.
  plain_fp64_per_point  the unbatched comparator on the 17x17 workload: FP64 PCG, one
                macropoint per constrained-solve launch (point_batch = 1).
  macro         the macroscopic problem (Eq. macro_eq) from the last step's coefficients,
                outside the timed region.

Multi-GPU (torchrun): every rank solves an independent hierarchy (a different medium
seed, i.e. another macroscopic region) with no collective on the data path; weak scaling.
The per-workload records and the CPU legs run at N = 1 only.

--impl reference: the oracle as it stands on all host cores. Before timing, the whole
hierarchy is solved once (untimed) so that every parent's cell functions exist; each step
then re-solves the same stratified sample of every level (a fixed fraction of each level's
points, sized so that the warm-up and timed steps end within about three minutes).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import mch_inputs as mi  # noqa: E402

METRIC = "cell-problem RHS solved/s at 1e-6 rel. accuracy; stencil HBM GB/s vs peak"
WORKLOAD = "incl2d_33x33_L4"   # the benchmark workload (--workload selects others)
# refinement tolerance of every solve: the projected-residual ratio at which the effective
# coefficients of every level are within 1e-6 (block-relative) of the oracle on every workload
# of the suite, checked by the oracle legs
RTOL = 3e-9
# the other workloads of the suite, each reported as a record of "configs"
SUB_RECORDS = (("channel2d_4x4_n32", "fp64"), ("channel2d_17x17_L3", "fp64"),
               ("channel2d_17x17_L3", "mixed"), ("channel3d_9x9x9_L3", "mixed"),
               ("channel2d_65x65_L3_adj", "mixed"))
ADJOINT_WORKLOAD = "channel2d_65x65_L3_adj"
PLAIN_WORKLOAD = "channel2d_17x17_L3"
# algorithmic FP32 flops per interior node of one inner stencil application of the 2D level
# kernel with its vector work: the 9-point stencil 17, M^-1 products, Chebyshev or PCG
# updates and the dot products 8
FLOPS_PER_NODE_APPLY = 25
# FP32 FMA throughput of this GPU type measured with a register-resident FMA loop
# (34.7e12 FMA/s), in flops
FP32_MEASURED_TFLOPS = 69.4
FP32_LANES = 128
# algorithmic HBM bytes of one inner PCG iteration of the 3D level kernel per interior node of
# a (point, function) unit, FP32 vectors: q = A p pass reads p and r and writes q (12 B); the
# update pass reads p, q and r, reads and writes delta and r, writes p (28 B); per-point data
# (kappa 4 B, labels 1 B and M^-1 4 B in the first pass, labels and M^-1 in the second: 14 B)
# is shared by the point's R functions
BYTES3D_PER_NODE_ITER_UNIT, BYTES3D_PER_NODE_ITER_POINT = 40, 14
# DRAM bytes (read + write) per k_level2d launch from ncu captures, per workload, keyed by
# (grid n, launch shape) so that either of the autotuner's usual picks is covered. Valid
# only for the kernel sources they were taken on: null is reported when the sources' hash
# differs or a level ran a shape without a capture.
LEVEL_TRAFFIC = {
    # ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum
    #     --clock-control none -k regex:k_level2d -s 12 -c 4 python bench.py --no-configs
    #     --no-cpu --no-plain --steps 1 --warmup 3 --tiles T   (the timed step's launches;
    #     T = 2,5,9,5 and 4,7,9,5)
    "incl2d_33x33_L4": {"sha256_16": "e75087f419c9503d", "bytes_per_launch": {
        (256, 2): 252.150e6, (128, 5): 209.942e6, (64, 9): 110.006e6, (32, 5): 187.339e6,
        (256, 4): 253.313e6, (128, 7): 211.140e6}},
}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.samples = []
        self._stop = threading.Event()
        self._thr = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(
                    ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                     "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=5)
                vals = [v.strip() for v in out.stdout.strip().split(",")]
                if len(vals) == 7:
                    self.samples.append(vals)
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._thr = threading.Thread(target=self._run, daemon=True)
        self._thr.start()
        return self

    def __exit__(self, *exc):
        self._stop.set()
        self._thr.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4)
                          if s[3 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


def _sources_hash():
    import hashlib
    h = hashlib.sha256()
    for f in ("k_level.cuh", "common.cuh", "k_level_f32.cu", "k_level_f32_alt.cu",
              "k_level_f32_alt2.cu", "k_level_shapes.h"):
        with open(os.path.join(ROOT, "paper_2503_01276_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _level_traffic(wl, tiles):
    rec = LEVEL_TRAFFIC.get(wl.name)
    if not rec or rec["sha256_16"] != _sources_hash() or not tiles:
        return None, None
    b = [rec["bytes_per_launch"].get((wl.n_level(k + 1), v)) for k, v in enumerate(tiles)]
    if any(x is None for x in b):
        return None, None
    return float(np.mean(b)), b


def max_over_ranks(t_local: float, dist, device) -> float:
    """Largest of the ranks' timed-region durations (every rank gets it)."""
    import torch
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(t_local)
    t = torch.tensor([float(t_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank_step: int, world: int, steps: int, t_max: float) -> float:
    """Units all ranks processed / the slowest rank's time (weak scaling: every rank solves
    its own hierarchy of the same size)."""
    return units_per_rank_step * world * steps / t_max


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def _hbm_peak():
    p = _peaks()
    for k in ("hbm_gbs", "hbm_GBs", "hbm_copy_gbs"):
        if isinstance(p.get(k), (int, float)) and p[k] > 0:
            return float(p[k]), "measured copy bandwidth (MEASURED_PEAKS.json)"
    return 6800.0, "fallback 6.8 TB/s (MEASURED_PEAKS.json absent)"


def _sm_count():
    import torch
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


def _level_sizes(wl):
    from oracle import plan
    return [len(l["points"]) for l in plan.level_plan(wl)]


def _config(wl, precision):
    return {"workload": wl.name,
            "macropoints": "x".join([str(wl.macro_n)] * wl.dim),
            "levels": _level_sizes(wl), "rve_grids": [wl.n_level(k + 1) for k in range(wl.n_levels)],
            "rhs_per_point": wl.n_rhs, "n_cont": wl.n_cont, "contrast": wl.contrast,
            "precision": precision,
            "l2": "flushed before every timed step (512 MB write, untimed)"}


# ----------------------------------------------------------------------------------------
# oracle legs (no CUDA in these processes)
# ----------------------------------------------------------------------------------------

def _media_fn(wl):
    from oracle import plan
    pl = plan.level_plan(wl)
    return lambda lv, pos: mi.media(wl, pl[lv - 1]["points"][list(pos)], wl.n_level(lv))


def sample_targets(wl, per_group=2):
    """Sampled (level, position) pairs: the first and last point of level 1 and, on every
    later level, up to `per_group` points with each parent count (1, 2, 4 in 2D)."""
    from oracle import plan
    pl = plan.level_plan(wl)
    out = []
    n1 = len(pl[0]["points"])
    out += [(1, 0), (1, n1 - 1)] if n1 > 1 else [(1, 0)]
    for lv in range(2, wl.n_levels + 1):
        groups = {}
        for i, par in enumerate(pl[lv - 1]["parents"]):
            groups.setdefault(len(par), []).append(i)
        for k in sorted(groups):
            g = groups[k]
            picks = sorted({g[0], g[-1]})[:per_group]
            out += [(lv, i) for i in picks]
    return out


def cpu_leg_main(spec_file):
    """Runs the oracle for every record of the spec (one process pool for all of them) and
    prints one JSON line with, per record, the all-core time, the summed single-core solve
    time and the block-relative error of the GPU coefficients."""
    from oracle import parallel
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from util import block_rel_err
    with open(spec_file) as f:
        spec = json.load(f)
    results = {}
    with parallel.OraclePool() as pool:
        for rec in spec["records"]:
            wl = mi.workload(rec["workload"], precision=rec["precision"])
            z = np.load(rec["npz"])
            Eg = [z[f"E{i}"] for i in range(wl.n_levels)]
            if rec["mode"] == "all":
                need = parallel.all_points(wl)
                targets = [(lv, i) for lv, ps in need.items() for i in ps]
            else:
                targets = sample_targets(wl)
                need = parallel.closure(wl, targets)
            jd = pool.job(wl, need, _media_fn(wl))
            E, wall, tsum, walls = pool.run(jd, wl, need)
            errs = {}
            for (lv, i) in targets:
                e = block_rel_err(Eg[lv - 1][i], E[(lv, i)], wl.n_cont, wl.dim)
                errs[lv] = max(errs.get(lv, 0.0), e)
            err = max(errs.values())
            n_solved = sum(len(v) for v in need.values())
            results[rec["tag"]] = {
                "err": err, "err_by_level": [errs.get(lv) for lv in range(1, wl.n_levels + 1)],
                "points_checked": len(targets), "points_solved": n_solved,
                "wall_s": wall, "single_core_s": tsum, "level_wall_s": walls,
                "rhs_solved": n_solved * wl.n_rhs, "cores": pool.procs}
    print(json.dumps({"cpu": results}), flush=True)


def run_cpu_leg(records, timeout=900):
    """records: dicts with tag, workload, precision, mode ("all" | "sample") and the GPU
    coefficients E (list per level). Runs cpu_leg_main in a fresh process without CUDA."""
    with tempfile.TemporaryDirectory() as td:
        spec = {"records": []}
        for k, r in enumerate(records):
            fn = os.path.join(td, f"e{k}.npz")
            np.savez(fn, **{f"E{i}": e for i, e in enumerate(r["E"])})
            spec["records"].append({kk: r[kk] for kk in ("tag", "workload", "precision", "mode")}
                                   | {"npz": fn})
        sf = os.path.join(td, "spec.json")
        with open(sf, "w") as f:
            json.dump(spec, f)
        env = dict(os.environ)
        for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
            env.pop(k, None)
        out = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-leg", sf],
                             capture_output=True, text=True, env=env, timeout=timeout)
        try:
            return json.loads(out.stdout.strip().splitlines()[-1])["cpu"]
        except Exception:
            return {"error": (out.stderr or out.stdout)[-600:]}


def run_reference(args, rank, world):
    """The oracle arm on all host cores (rank 0 only)."""
    if rank != 0:
        return
    from oracle import parallel
    wl = mi.workload(args.workload, precision="fp64")
    need_all = parallel.all_points(wl)
    with parallel.OraclePool() as pool:
        jd = pool.job(wl, need_all, _media_fn(wl))
        # every parent's cell functions, once, untimed
        _, t_full, _, _ = pool.run(jd, wl, need_all)
        k_total = max(args.steps, 1) + max(args.warmup, 0)
        frac = min(1.0, 150.0 / max(k_total * t_full, 1e-9))
        sample = {}
        for lv, pos in need_all.items():
            cnt = max(1, int(round(frac * len(pos))))
            sample[lv] = sorted(set(np.linspace(0, len(pos) - 1, cnt).round().astype(int).tolist()))
        n_rhs = sum(len(v) for v in sample.values()) * wl.n_rhs
        for _ in range(args.warmup):
            pool.run(jd, wl, sample, write_phi=False)
        times, tsum = [], 0.0
        for _ in range(args.steps):
            _, w, ts, _ = pool.run(jd, wl, sample, write_phi=False)
            times.append(w)
            tsum += ts
        cores = pool.procs
    t = float(np.sum(times))
    v = n_rhs * args.steps / t
    desc = (f"every level's points re-solved as a stratified sample of {100 * frac:.0f}% "
            f"({sum(len(s) for s in sample.values())} of {sum(len(s) for s in need_all.values())} "
            f"points per step, levels in order) after one untimed full pass "
            f"({t_full:.1f} s on {cores} cores)")
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "RHS/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t / max(args.steps, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(_config(wl, "fp64"), rhs_per_step=n_rhs,
                           l2="not applicable (host cores)"),
            "cpu_baseline": {"value": v, "unit": "RHS/s", "cores": cores, "kind": "oracle",
                             "sample": desc, "single_core_value": n_rhs * args.steps / tsum},
            "e2e": {"value": v, "unit": "RHS/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------------------
# GPU legs
# ----------------------------------------------------------------------------------------

class GpuRun:
    """One workload on the GPU: handle, resident and pinned media, timed steps."""

    def __init__(self, wl, dev, stream, tiles=None, autotune=True, rtol=RTOL, **solver_kw):
        import torch
        import paper_2503_01276_gb300 as mch
        self.wl, self.dev, self.stream = wl, dev, stream
        self.s = mch.Solver.from_workload(wl, stream=stream.cuda_stream, rtol=rtol, **solver_kw)
        self.s.set_timing(True)
        self.L = wl.n_levels
        self.med_host, self.med_dev = [], []
        for lev in range(1, self.L + 1):
            k, lb = mi.media(wl, self.s.level_points(lev), self.s.n_elem(lev))
            kh = torch.from_numpy(k).pin_memory()
            lh = torch.from_numpy(lb).pin_memory()
            self.med_host.append((kh, lh))
            self.med_dev.append((kh.to(dev), lh.to(dev)))
        R = self.s.R
        self.E_dev = [torch.zeros((self.s.num_points(l), R, R), dtype=torch.float64, device=dev)
                      for l in range(1, self.L + 1)]
        self.E_host = [torch.zeros((self.s.num_points(l), R, R), dtype=torch.float64).pin_memory()
                       for l in range(1, self.L + 1)]
        self.rhs_per_step = sum(self.s.num_points(l) for l in range(1, self.L + 1)) * R
        self.tiles = []
        if tiles:
            for lev, v in enumerate(tiles, start=1):
                self.s.set_variant(lev, v)
            self.tiles = list(tiles)
        elif autotune and wl.dim == 2:
            for lev in range(1, self.L + 1):
                v, _ = self.s.autotune_level(lev, *self.med_dev[lev - 1])
                self.tiles.append(v)
        else:
            self.tiles = [self.s.variant(lev)[0] for lev in range(1, self.L + 1)]

    def step(self, device_inputs=True):
        med = self.med_dev if device_inputs else self.med_host
        # constraint data of every level on the library's side stream, so that the later
        # levels' setup overlaps the level-1 solve
        for lev in range(1, self.L + 1):
            self.s.prepare_level(lev, *med[lev - 1])
        for lev in range(1, self.L + 1):
            k, lb = med[lev - 1]
            self.s.solve_level(lev, k, lb)
            self.s.effective_coeffs(lev, self.E_dev[lev - 1] if device_inputs
                                    else self.E_host[lev - 1])

    def timed(self, steps, warmup, flush, dist=None, world=1):
        """Device-resident steps timed with CUDA events; returns the record pieces."""
        import torch
        for _ in range(max(warmup, 3)):
            self.step()
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        L = self.L
        lv = [{"pcg_ms": 0.0, "node_iters": 0, "node_applies": 0, "launches": 0,
               "setup_ms": 0.0, "interp_ms": 0.0, "final_ms": 0.0} for _ in range(L)]
        launches = 0
        relres = 0.0
        with ClockSampler(self.dev.index or 0) as clk:
            torch.cuda.synchronize()
            for i in range(steps):
                flush.zero_()
                evs[i][0].record(self.stream)
                self.step()
                evs[i][1].record(self.stream)
                for lev in range(1, L + 1):
                    st = self.s.stats(lev)
                    lv[lev - 1]["pcg_ms"] += st["pcg_ms"]
                    for key in ("setup_ms", "interp_ms", "final_ms"):
                        lv[lev - 1][key] += st[key]
                    lv[lev - 1]["node_iters"] += st["pcg_node_iters"]
                    lv[lev - 1]["node_applies"] += st["pcg_node_applies"]
                    lv[lev - 1]["launches"] += st["pcg_launches"]
                    launches += st["gpu_launches"]
                    relres = max(relres, st["max_relres"])
            torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        step_ms = [a.elapsed_time(b) for a, b in evs]
        return {"step_ms": step_ms, "levels": lv, "launches": launches, "relres": relres,
                "clocks": clk.summary()}

    def e2e(self, steps, flush, dist=None):
        """Host-buffer steps through the public API, host clock; seconds in total."""
        import torch
        self.step(device_inputs=False)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        tt = 0.0
        for _ in range(steps):
            flush.zero_()
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            self.step(device_inputs=False)
            torch.cuda.synchronize()
            tt += time.perf_counter() - t1
        h2d = sum(k.numel() * k.element_size() + lb.numel() * lb.element_size()
                  for k, lb in self.med_host)
        d2h = sum(e.numel() * e.element_size() for e in self.E_host)
        return tt, h2d, d2h

    def E_numpy(self):
        return [e.cpu().numpy() for e in self.E_dev]

    def close(self):
        self.s.close()


def roofline(wl, R, t, steps, tiles):
    """Roofline of the dominant kernel from the timed steps' per-level records."""
    hbm, hbm_src = _hbm_peak()
    pcg_ms = sum(l["pcg_ms"] for l in t["levels"])
    total_ms = float(np.sum(t["step_ms"]))
    share = pcg_ms / total_ms if total_ms > 0 else None
    sm_mhz = t["clocks"].get("sm_mhz") or 2070.0
    if wl.dim == 2:
        by_level = []
        tot_bytes = 0.0
        for k, l in enumerate(t["levels"]):
            n = wl.n_level(k + 1)
            unit_applies = l["node_applies"] / float((n - 1) ** 2)
            b = unit_applies * ((n - 1) ** 2 * 2 * 4 + n * n * 4.0 / R)
            tot_bytes += b
            by_level.append({"n": n, "ms_per_step": l["pcg_ms"] / steps,
                             "gbs": (b / (l["pcg_ms"] / 1e3) / 1e9) if l["pcg_ms"] > 0 else None,
                             "launches_per_step": l["launches"] / steps,
                             # the level's other phases (library event timing, ms per step):
                             # constraint data (on the side stream, overlapping earlier
                             # levels), level-1-grid interpolation and right-hand sides, and
                             # coefficients plus cell-function assembly
                             "other_ms": {k[:-3]: l.get(k, 0.0) / steps
                                          for k in ("setup_ms", "interp_ms", "final_ms")}})
        gbs = tot_bytes / (pcg_ms / 1e3) / 1e9 if pcg_ms > 0 else None
        flops = sum(l["node_applies"] for l in t["levels"]) * FLOPS_PER_NODE_APPLY
        tfl = flops / (pcg_ms / 1e3) / 1e12 if pcg_ms > 0 else None
        derived = _sm_count() * FP32_LANES * 2 * sm_mhz * 1e6 / 1e12
        traffic, traffic_levels = _level_traffic(wl, tiles)
        launches = sum(l["launches"] for l in t["levels"])
        return {"bound": "hbm", "kernel": "k_level2d (persistent level solve)",
                "achieved": gbs, "peak": hbm, "unit": "GB/s",
                "frac": (gbs / hbm) if gbs else None,
                "traffic": traffic, "traffic_per_launch_by_level": traffic_levels,
                "peak_source": hbm_src,
                "bytes_model": "per multi-RHS stencil apply: n^2 x 4 B FP32 kappa shared by the "
                               "R functions + R x (n-1)^2 x 2 x 4 B FP32 vector in and out; "
                               "applies = inner stencil applications (PCG iterations x "
                               "Chebyshev steps)",
                "algorithmic_bytes_per_step": tot_bytes / steps,
                "by_level": by_level, "kernel_share_of_step": share,
                "launches_timed": launches,
                "alu": {"achieved_tflops": tfl, "flops_per_node_apply": FLOPS_PER_NODE_APPLY,
                        "peak_measured_tflops": FP32_MEASURED_TFLOPS,
                        "frac_of_measured": (tfl / FP32_MEASURED_TFLOPS) if tfl else None,
                        "peak_derived_tflops": derived,
                        "peak_derived_source": "SMs x 128 FP32 lanes x 2 x sampled SM clock"}}
    bpn = BYTES3D_PER_NODE_ITER_UNIT + BYTES3D_PER_NODE_ITER_POINT / R
    node_iters = sum(l["node_iters"] for l in t["levels"])
    by_level = []
    for k, l in enumerate(t["levels"]):
        by_level.append({"n": wl.n_level(k + 1), "ms_per_step": l["pcg_ms"] / steps,
                         "gbs": (l["node_iters"] * bpn / (l["pcg_ms"] / 1e3) / 1e9)
                         if l["pcg_ms"] > 0 else None,
                         "other_ms": {k_[:-3]: l.get(k_, 0.0) / steps
                                      for k_ in ("setup_ms", "interp_ms", "final_ms")}})
    gbs = node_iters * bpn / (pcg_ms / 1e3) / 1e9 if pcg_ms > 0 else None
    return {"bound": "hbm", "kernel": "k_level3d (cooperative level solve)",
            "achieved": gbs, "peak": hbm, "unit": "GB/s",
            "frac": (gbs / hbm) if gbs else None, "traffic": None, "peak_source": hbm_src,
            "bytes_model": "per inner PCG iteration and interior node: 40 B of FP32 vectors "
                           "per function + 14 B of per-point data shared by the R functions",
            "bytes_per_node_iteration": bpn, "by_level": by_level,
            "kernel_share_of_step": share,
            "launches_timed": sum(l["launches"] for l in t["levels"])}


def macro_leg(s, wl, E_dev, stream):
    """Source densities (mch_macro_source, the Gaussian source of Sec. 5: weights 1/contrast
    and 1 for the other continua, alpha 40, centre of the unit domain) and the macroscopic
    solve (mch_macro_solve) from device coefficients; times of each, the CG record and the
    size."""
    import torch
    d, N = wl.dim, wl.n_cont
    w = np.ones(N)
    w[0] = 1.0 / wl.contrast
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    fb = [torch.zeros((s.num_points(lev), N), dtype=torch.float64, device=E_dev[0].device)
          for lev in range(1, wl.n_levels + 1)]
    U = torch.zeros((N, (wl.macro_n + 1) ** d), dtype=torch.float64, device=E_dev[0].device)
    ev[0].record(stream)
    for lev in range(1, wl.n_levels + 1):
        s.macro_source(lev, w, np.full(d, 0.5), 40.0, np.full(d, wl.origin), wl.spacing,
                       out=fb[lev - 1])
    ev[1].record(stream)
    _, iters, rr = s.macro_solve(E_dev, fb, wl.spacing, tol=1e-12, out=U)
    ev[2].record(stream)
    torch.cuda.synchronize()
    return {"source_ms": ev[0].elapsed_time(ev[1]), "solve_ms": ev[1].elapsed_time(ev[2]),
            "cg_iters": iters, "relres": rr, "unknowns": int(N * (wl.macro_n - 1) ** d),
            "max_abs_u": float(U.abs().max().item())}


def plain_fp64_leg(wl, med_dev, flush, steps, stream, rtol=RTOL):
    """The unbatched FP64 comparator: same workload and media, FP64 PCG, one macropoint per
    constrained-solve launch. Returns RHS/s, ms per step and the largest residual ratio."""
    import torch
    import paper_2503_01276_gb300 as mch
    s = mch.Solver.from_workload(wl, stream=stream.cuda_stream, precision="fp64",
                                 point_batch=1, rtol=rtol)
    L = wl.n_levels
    E = [torch.zeros((s.num_points(l), s.R, s.R), dtype=torch.float64, device=flush.device)
         for l in range(1, L + 1)]

    def step():
        for lev in range(1, L + 1):
            s.solve_level(lev, *med_dev[lev - 1])
            s.effective_coeffs(lev, E[lev - 1])

    step()
    torch.cuda.synchronize()
    ms = []
    relres = 0.0
    launches = 0
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
        for lev in range(1, L + 1):
            st = s.stats(lev)
            relres = max(relres, st["max_relres"])
            launches += st["pcg_launches"]
    rhs = sum(s.num_points(l) for l in range(1, L + 1)) * s.R
    out = {"value": rhs / (np.mean(ms) / 1e3), "unit": "RHS/s", "ms_per_step": float(np.mean(ms)),
           "steps": steps, "solve_launches_per_step": launches // steps, "max_relres": relres,
           "kind": "FP64 PCG, one macropoint per constrained-solve launch (point_batch=1)"}
    s.close()
    return out, E


def backward_leg(wl, dev, stream, flush, reps=2, rtol=RTOL):
    """Forward then backward of the loss L = sum_p sum W[p] . E[p] (seeded N(0,1) weights on
    the upper triangles of the exchange and permeability blocks, seed 7), with the cell
    functions of the parents checkpointed (keep_parents = 1) or recomputed (0). Times the
    backward call alone (CUDA events); checks the Euler identity sum kappa dL/dkappa = L and
    the agreement of the two gradients."""
    import torch
    import paper_2503_01276_gb300 as mch
    N, d, R = wl.n_cont, wl.dim, wl.n_rhs
    mask = np.zeros((R, R))
    mask[np.triu_indices(N)] = 1.0
    iu = np.triu_indices(N * d)
    mask[N + iu[0], N + iu[1]] = 1.0
    rng = np.random.default_rng(7)
    out = {}
    grads = {}
    for kp in (1, 0):
        s = mch.Solver.from_workload(wl, stream=stream.cuda_stream, keep_parents=kp,
                                     rtol=rtol)
        L = wl.n_levels
        med = []
        for lev in range(1, L + 1):
            k, lb = mi.media(wl, s.level_points(lev), s.n_elem(lev))
            med.append((torch.from_numpy(k).to(dev), torch.from_numpy(lb).to(dev)))
        if not grads:
            Wn = [rng.standard_normal((s.num_points(l), R, R)) * mask for l in range(1, L + 1)]
        Wd = [torch.from_numpy(w).to(dev) for w in Wn]
        E = [torch.zeros((s.num_points(l), R, R), dtype=torch.float64, device=dev)
             for l in range(1, L + 1)]
        G = [torch.zeros((s.num_points(l), s.n_elem(l) ** d), dtype=torch.float64, device=dev)
             for l in range(1, L + 1)]
        ms = []
        for rep in range(reps + 1):
            for lev in range(1, L + 1):
                s.solve_level(lev, *med[lev - 1])
                s.effective_coeffs(lev, E[lev - 1])
            flush.zero_()
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            s.backward(Wd, G)
            b.record(stream)
            torch.cuda.synchronize()
            if rep > 0:
                ms.append(a.elapsed_time(b))
        loss = sum(float((w * e).sum()) for w, e in zip(Wd, E))
        euler = sum(float((k * g).sum()) for (k, _), g in zip(med, G))
        grads[kp] = [g.cpu().numpy() for g in G]
        out[f"keep_parents_{kp}"] = {"backward_ms": float(np.mean(ms)), "reps": reps,
                                     "euler_rel_residual": abs(euler - loss) / abs(loss)}
        s.close()
    num = max(float(np.abs(a - b).max()) for a, b in zip(grads[1], grads[0]))
    den = max(float(np.abs(a).max()) for a in grads[1])
    out["checkpoint_vs_recompute_max_rel"] = num / den
    return out


def gpu_record(wl, dev, stream, flush, steps, warmup, e2e_steps, rtol=RTOL):
    """A per-workload record (N = 1): RHS/s, e2e, roofline, launches, residual."""
    g = GpuRun(wl, dev, stream, rtol=rtol)
    t = g.timed(steps, warmup, flush)
    total = float(np.sum(t["step_ms"])) / 1e3
    value = g.rhs_per_step * steps / total
    tt, h2d, d2h = g.e2e(e2e_steps, flush)
    rec = {"workload": wl.name, "precision": wl.precision,
           "config": dict(_config(wl, wl.precision), rhs_per_step=g.rhs_per_step,
                          level_tiles=g.tiles),
           "value": value, "unit": "RHS/s", "ms_per_step": float(np.mean(t["step_ms"])),
           "steps": steps, "roofline": roofline(wl, g.s.R, t, steps, g.tiles),
           "e2e": {"value": g.rhs_per_step * e2e_steps / tt, "unit": "RHS/s",
                   "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
           "gpu_launches": t["launches"], "clocks": t["clocks"],
           "max_relres": t["relres"]}
    E = g.E_numpy()
    med_dev = g.med_dev
    g.close()
    return rec, E, med_dev


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mch", choices=["mch", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle legs")
    ap.add_argument("--no-plain", action="store_true",
                    help="skip the unbatched per-macropoint FP64 comparator")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the records of the other workloads")
    ap.add_argument("--workload", default=WORKLOAD,
                    help="workload of mch_inputs (default: the benchmark workload)")
    ap.add_argument("--rtol", type=float, default=RTOL,
                    help="refinement tolerance of the solves (the accuracy the metric names "
                         "is checked against the oracle)")
    ap.add_argument("--inner-tol", type=float, default=0.0,
                    help="per-sweep reduction of the inner PCG (0: the library default)")
    ap.add_argument("--tiles", default=None,
                    help="comma-separated launch shapes per level instead of autotuning "
                         "(fixed launch counts, for profiling)")
    ap.add_argument("--macro-n", type=int, default=None,
                    help="reduced copy of the workload: macropoints per axis (with --strides; "
                         "for profiling a small case)")
    ap.add_argument("--strides", default=None,
                    help="comma-separated level strides of the reduced copy")
    ap.add_argument("--cpu-leg", default=None, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.cpu_leg is not None:
        cpu_leg_main(args.cpu_leg)
        return

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    wl = mi.workload(args.workload, precision=args.precision,
                     seed=mi.workload(args.workload).seed + rank)
    if args.macro_n is not None:
        strides = tuple(int(v) for v in args.strides.split(",")) if args.strides else (1,)
        wl = mi.small_workload(args.workload, n_fine=wl.n_fine, macro_n=args.macro_n,
                               strides=strides, precision=args.precision, seed=wl.seed)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    tiles = [int(v) for v in args.tiles.split(",")] if args.tiles else None

    g = GpuRun(wl, dev, stream, tiles=tiles, rtol=args.rtol, inner_tol=args.inner_tol)
    t = g.timed(args.steps, args.warmup, flush, dist if world > 1 else None, world)
    t_total = max_over_ranks(float(np.sum(t["step_ms"])) / 1e3, dist if world > 1 else None, dev)
    value = whole_job_rate(g.rhs_per_step, world, args.steps, t_total)
    e2e_steps = max(3, args.steps // 2)
    tt, h2d, d2h = g.e2e(e2e_steps, flush, dist if world > 1 else None)
    tt = max_over_ranks(tt, dist if world > 1 else None, dev)
    e2e_value = whole_job_rate(g.rhs_per_step, world, e2e_steps, tt)
    try:
        macro_info = macro_leg(g.s, wl, g.E_dev, stream)
    except Exception as ex:  # an auxiliary record must not cost the benchmark line
        macro_info = {"error": f"{type(ex).__name__}: {ex}"[:300]}
    E_main = g.E_numpy()
    rf = roofline(wl, g.s.R, t, args.steps, g.tiles)
    main_tiles = g.tiles
    g.close()
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    configs = []
    cpu_records = [{"tag": "main", "workload": wl.name, "precision": wl.precision,
                    "mode": "all", "E": E_main}]
    plain = None
    if world == 1 and not args.no_configs:
        for name, prec in SUB_RECORDS:
            if name == wl.name and prec == wl.precision:
                continue
            swl = mi.workload(name, precision=prec)
            sub_steps = max(3, min(args.steps, 5 if swl.dim == 3 else 10))
            try:
                rec, E, med_dev = gpu_record(swl, dev, stream, flush, sub_steps, 3,
                                             max(3, sub_steps // 2), rtol=args.rtol)
            except Exception as ex:
                configs.append({"workload": name, "precision": prec,
                                "error": f"{type(ex).__name__}: {ex}"[:300]})
                continue
            tag = f"{name}:{prec}"
            rec["tag"] = tag
            if swl.dim == 2:
                cpu_records.append({"tag": tag, "workload": name, "precision": prec,
                                    "mode": "all" if name != ADJOINT_WORKLOAD else "sample",
                                    "E": E})
            else:
                rec["accuracy"] = {
                    "vs_oracle": None,
                    "why": "the oracle's sparse LU of a 64^3 level-1 RVE does not finish in "
                           "bounded time; the 3D path is checked against the oracle on "
                           "reduced grids in the tests"}
            if name == ADJOINT_WORKLOAD:
                try:
                    rec["backward"] = backward_leg(swl, dev, stream, flush, rtol=args.rtol)
                except Exception as ex:
                    rec["backward"] = {"error": f"{type(ex).__name__}: {ex}"[:300]}
            if name == PLAIN_WORKLOAD and prec == "mixed" and not args.no_plain:
                plain, E_plain = plain_fp64_leg(swl, med_dev, flush, 2, stream, args.rtol)
                plain["workload"] = name
                plain["speedup_of_mixed_batched"] = rec["value"] / plain["value"]
                sys.path.insert(0, os.path.join(ROOT, "tests"))
                from util import block_rel_err
                plain["block_rel_diff_vs_batched"] = max(
                    block_rel_err(a, b.cpu().numpy(), swl.n_cont, swl.dim)
                    for a, b in zip(E, E_plain))
            del med_dev
            configs.append(rec)
            torch.cuda.empty_cache()

    cpu = None
    acc_err = acc_levels = None
    if not args.no_cpu:
        res = run_cpu_leg(cpu_records)
        if "error" in res:
            cpu = res
        else:
            m = res.get("main", {})
            acc_err = m.get("err")
            acc_levels = m.get("err_by_level")
            if m:
                cpu = {"value": m["rhs_solved"] / m["wall_s"], "unit": "RHS/s",
                       "cores": m["cores"], "kind": "oracle",
                       "sample": f"the whole workload ({m['points_solved']} points, levels in "
                                 f"order) on {m['cores']} worker processes, one BLAS thread "
                                 f"each",
                       "wall_s": m["wall_s"], "level_wall_s": m["level_wall_s"],
                       "single_core_s": m["single_core_s"],
                       "single_core_value": m["rhs_solved"] / m["single_core_s"]}
            for rec in configs:
                r = res.get(rec.get("tag"))
                if r:
                    rec["accuracy"] = {"block_rel_err_vs_oracle": r["err"],
                                       "block_rel_err_by_level": r["err_by_level"],
                                       "points_checked": r["points_checked"]}
                    rec["cpu_baseline"] = {"value": r["rhs_solved"] / r["wall_s"],
                                           "unit": "RHS/s", "cores": r["cores"],
                                           "kind": "oracle",
                                           "points_solved": r["points_solved"],
                                           "single_core_value": r["rhs_solved"] /
                                           r["single_core_s"]}
    line = {"metric": METRIC, "value": value, "unit": "RHS/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(args.warmup, 3),
            "ms_per_step": float(np.mean(t["step_ms"])), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
            "config": dict(_config(wl, args.precision), rhs_per_step=g.rhs_per_step,
                           level_tiles=main_tiles),
            "roofline": rf, "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "RHS/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": t["launches"], "clocks": t["clocks"],
            "accuracy": {"max_relres": t["relres"], "rtol": args.rtol,
                         "block_rel_err_vs_oracle": acc_err,
                         "block_rel_err_by_level": acc_levels,
                         "points_checked": "all" if acc_err is not None else 0},
            "configs": configs, "plain_fp64_per_point": plain, "macro": macro_info}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
