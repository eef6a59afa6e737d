"""Benchmark: cell-problem right-hand sides solved per second on the 2D three-level
hierarchy (17x17 macropoints, levels of 9/72/208 points on RVE grids 128/64/32, two
continua, six cell functions per point, contrast 1e4, FP32 PCG inside FP64 refinement).

One step solves every level of the hierarchy through the library (mch_solve_level per
level: constraint data, interpolation and correction right-hand sides, batched
constrained solves, cell-function assembly and effective coefficients), with the media
already resident in device memory. The L2 cache is flushed (a 512 MB device write,
outside the timed event pairs) before every timed step.

JSON line keys beyond the base contract:
  roofline      the persistent level kernel k_level2d (the time sink; FP32 PCG sweeps
                inside FP64 refinement steps, all of a level's points in one launch):
                algorithmic FP32 flops of the PCG iterations it ran / its CUDA-event time,
                against the FP32 ALU peak 152 SMs x 128 FP32 lanes x 2 flops x the sampled
                SM clock. The kernel keeps its whole state in shared memory, so DRAM traffic
                is small and the bound is the ALU (and the FP64 refinement steps).
  plain_fp64_per_point  the unbatched comparator: the same workload solved in FP64 with one
                macropoint per constrained-solve launch (point_batch = 1).
  cpu_baseline  the FP64 oracle (SciPy) on one host core, timed on a sample of points per
                level and extrapolated to the whole workload.
  e2e           the same step through the public API with pinned host buffers (media
                copied in, effective coefficients copied out) inside the timed region.
  accuracy      largest final projected-residual ratio, and the block-relative error of
                the sampled points against the oracle.
  macro         the macroscopic problem (Eq. macro_eq) from the last step's coefficients,
                outside the timed region: source densities of every level and the solve on
                the coarse blocks, their CUDA-event times and the CG record.

Multi-GPU (torchrun): every rank solves an independent hierarchy (a different medium
seed, i.e. another macroscopic region) with no collective on the data path; weak scaling.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import mch_inputs as mi  # noqa: E402

METRIC = "cell-problem RHS solved/s at 1e-6 rel. accuracy; stencil HBM GB/s vs peak"
WORKLOAD = "channel2d_17x17_L3"   # the benchmark workload (--workload selects others)
# algorithmic FP32 flops of one PCG iteration per interior node: stencil 17, four dot
# products 8, x/r/p updates 6, M^-1 r and M^-1 q 2, Ct^T lambda gather 4, two Ct scatters 8
FLOPS_PER_NODE_ITER = 45
SMS, FP32_LANES = 152, 128
# algorithmic HBM bytes of one inner PCG iteration of the 3D level kernel per interior node of
# a (point, function) unit, FP32 vectors: q = A p pass reads p and r and writes q (12 B); the
# update pass reads p, q and r, reads and writes delta and r, writes p (28 B); per-point data
# (kappa 4 B, labels 1 B and M^-1 4 B in the first pass, labels and M^-1 in the second: 14 B)
# is shared by the point's R functions
BYTES3D_PER_NODE_ITER_UNIT, BYTES3D_PER_NODE_ITER_POINT = 40, 14
# DRAM bytes (read + write) per k_level2d launch of this workload (levels 1, 2, 3), from one
# ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) of
#   python bench.py --steps 1 --warmup 3 --no-cpu --no-plain
# Valid only for the kernel source it was taken on: the JSON reports null when the
# sources' hash differs.
LEVEL_TRAFFIC = {"sha256_16": ("43c91844b0a8140f", "3e24044d01b04bd2", "d8d56e737f1a3b53"),
                 "bytes_per_launch": (2.832128e6, 20.505088e6, 16.83456e6)}


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


def _level_traffic():
    import hashlib
    got = []
    for f in ("k_level.cuh", "k_level_f32.cu", "k_level_f32_alt.cu"):
        with open(os.path.join(ROOT, "paper_2503_01276_gb300", "csrc", f), "rb") as fh:
            got.append(hashlib.sha256(fh.read()).hexdigest()[:16])
    if tuple(got) != LEVEL_TRAFFIC["sha256_16"]:
        return None, None
    b = LEVEL_TRAFFIC["bytes_per_launch"]
    return float(np.mean(b)), list(b)


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


def cpu_baseline(wl, Eg_by_level, per_level=2, budget_s=25.0):
    """FP64 oracle on one host core: per level, time `per_level` points (their ancestors are
    computed untimed first), extrapolate the whole workload; also returns the block-relative
    error of the GPU result on those points."""
    from oracle import cell, plan
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from util import block_rel_err
    pl = plan.level_plan(wl)
    per_point = []
    errs = []
    cache = {}
    t_used = 0.0
    for lv in range(1, wl.n_levels + 1):
        npts = len(pl[lv - 1]["points"])
        picks = sorted(set(np.linspace(0, npts - 1, per_level).astype(int).tolist()))
        ops = cell.LevelOps(wl, lv)
        times = []
        for i in picks:
            need = sorted(cell.ancestors(pl, lv, i) - {(lv, i)})
            for (l2, p2) in need:
                if (l2, p2) in cache:
                    continue
                o2 = cell.LevelOps(wl, l2)
                k, lb = mi.media(wl, pl[l2 - 1]["points"][[p2]], wl.n_level(l2))
                I = None
                if l2 > 1:
                    I = sum(w * cache[(a, b)]["Phi"].T for (a, b, w) in pl[l2 - 1]["parents"][p2])
                cache[(l2, p2)] = cell.solve_point(o2, k[0], lb[0], I)
            k, lb = mi.media(wl, pl[lv - 1]["points"][[i]], wl.n_level(lv))
            I = None
            if lv > 1:
                I = sum(w * cache[(a, b)]["Phi"].T for (a, b, w) in pl[lv - 1]["parents"][i])
            t0 = time.perf_counter()
            r = cell.solve_point(ops, k[0], lb[0], I)
            dt = time.perf_counter() - t0
            times.append(dt)
            t_used += dt
            cache[(lv, i)] = r
            if Eg_by_level is not None:
                errs.append(block_rel_err(Eg_by_level[lv - 1][i], r["E"], wl.n_cont, wl.dim))
            if t_used > budget_s:
                break
        per_point.append((npts, float(np.mean(times))))
    t_full = sum(n * t for n, t in per_point)
    total_rhs = sum(n for n, _ in per_point) * wl.n_rhs
    return {"value": total_rhs / t_full, "unit": "RHS/s", "cores": 1, "kind": "oracle",
            "sample": f"{per_level} points per level timed one by one (SciPy sparse LU + Schur "
                      f"+ FP64 refinement, one BLAS thread), extrapolated by level sizes "
                      f"{[n for n, _ in per_point]}",
            "seconds_per_point": [t for _, t in per_point]}, (max(errs) if errs else None)


def run_reference(args, rank, world):
    """The oracle arm: each step is the bounded oracle sample of the workload (two points per
    level, timed one by one on one host core, extrapolated to the whole workload)."""
    if rank != 0:
        return
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        env.pop(k, None)

    def leg():
        out = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-leg", "",
                              "--workload", args.workload],
                             capture_output=True, text=True, env=env, timeout=600)
        return json.loads(out.stdout.strip().splitlines()[-1])["cpu"]

    for _ in range(args.warmup):
        leg()
    legs = [leg() for _ in range(args.steps)]
    v = float(np.mean([c["value"] for c in legs]))
    wl = mi.workload(args.workload)
    rhs_per_step = sum(_level_sizes(wl)) * wl.n_rhs
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "RHS/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * rhs_per_step / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _config(wl, "fp64"),
            "cpu_baseline": {"value": v, "unit": "RHS/s", "cores": 1, "kind": "oracle",
                             "sample": legs[0]["sample"]},
            "e2e": {"value": v, "unit": "RHS/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _level_sizes(wl):
    from oracle import plan
    return [len(l["points"]) for l in plan.level_plan(wl)]


def _config(wl, precision):
    return {"workload": wl.name,
            "macropoints": "x".join([str(wl.macro_n)] * wl.dim),
            "levels": _level_sizes(wl), "rve_grids": [wl.n_level(k + 1) for k in range(wl.n_levels)],
            "rhs_per_point": wl.n_rhs, "contrast": wl.contrast, "precision": precision,
            "l2": "flushed before every timed step (512 MB write, untimed)"}


def macro_leg(s, wl, E_dev, stream):
    """Source densities (mch_macro_source, the Gaussian source of Sec. 5: weights 1/contrast
    and 1 for the two continua, alpha 40, centre of the unit domain) and the macroscopic solve
    (mch_macro_solve) from device coefficients; times of each, the CG record and the size."""
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


def plain_fp64_leg(wl, med_dev, flush, steps, stream):
    """The unbatched FP64 comparator: same workload and media, FP64 PCG, one macropoint per
    constrained-solve launch. Returns RHS/s, ms per step and the largest residual ratio."""
    import torch
    import paper_2503_01276_gb300 as mch
    s = mch.Solver.from_workload(wl, stream=stream.cuda_stream, precision="fp64",
                                 point_batch=1)
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mch", choices=["mch", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle baseline leg")
    ap.add_argument("--no-plain", action="store_true",
                    help="skip the unbatched per-macropoint FP64 comparator")
    ap.add_argument("--workload", default=WORKLOAD,
                    help="workload of mch_inputs (default: the benchmark workload)")
    ap.add_argument("--tiles", default=None,
                    help="comma-separated launch shapes per level instead of autotuning "
                         "(fixed launch counts, for profiling)")
    ap.add_argument("--cpu-leg", default=None, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.cpu_leg is not None:
        # oracle baseline in a single-threaded child process; GPU results in an .npz file
        Eg = None
        if args.cpu_leg:
            z = np.load(args.cpu_leg)
            Eg = [z[f"E{i}"] for i in range(len(z.files))]
        cb, err = cpu_baseline(mi.workload(args.workload, precision=args.precision), Eg)
        print(json.dumps({"cpu": cb, "err": err}), flush=True)
        return

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist
    import paper_2503_01276_gb300 as mch

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    wl = mi.workload(args.workload, precision=args.precision,
                     seed=mi.workload(args.workload).seed + rank)
    stream = torch.cuda.current_stream()
    s = mch.Solver.from_workload(wl, stream=stream.cuda_stream)
    s.set_timing(True)
    L = wl.n_levels
    med_host = []
    med_dev = []
    for lev in range(1, L + 1):
        pts = s.level_points(lev)
        k, lb = mi.media(wl, pts, s.n_elem(lev))
        kh = torch.from_numpy(k).pin_memory()
        lh = torch.from_numpy(lb).pin_memory()
        med_host.append((kh, lh))
        med_dev.append((kh.to(dev), lh.to(dev)))
    E_dev = [torch.zeros((s.num_points(l), s.R, s.R), dtype=torch.float64, device=dev)
             for l in range(1, L + 1)]
    E_host = [torch.zeros((s.num_points(l), s.R, s.R), dtype=torch.float64).pin_memory()
              for l in range(1, L + 1)]
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    rhs_per_step = sum(s.num_points(l) for l in range(1, L + 1)) * s.R

    # launch shapes of the level solves, chosen by the library's autotuner on this workload
    tiles = []
    if args.tiles:
        tiles = [int(v) for v in args.tiles.split(",")]
        for lev, v in enumerate(tiles, start=1):
            s.set_variant(lev, v)
    else:
        for lev in range(1, L + 1):
            v, ms = s.autotune_level(lev, *med_dev[lev - 1])
            tiles.append(v)

    def step(device_inputs=True):
        med = med_dev if device_inputs else med_host
        # constraint data of every level on the library's side stream, so that the later
        # levels' setup overlaps the level-1 solve
        for lev in range(1, L + 1):
            s.prepare_level(lev, *med[lev - 1])
        for lev in range(1, L + 1):
            k, lb = med[lev - 1]
            s.solve_level(lev, k, lb)
            s.effective_coeffs(lev, E_dev[lev - 1] if device_inputs else E_host[lev - 1])

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    gpu_index = local
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    pcg_ms = 0.0
    pcg_node_iters = 0
    pcg_launches = 0
    launches = 0
    relres = 0.0
    with ClockSampler(gpu_index) as clk:
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.zero_()
            evs[i][0].record(stream)
            step()
            evs[i][1].record(stream)
            for lev in range(1, L + 1):
                st = s.stats(lev)
                pcg_ms += st["pcg_ms"]
                pcg_node_iters += st["pcg_node_iters"]
                pcg_launches += st["pcg_launches"]
                launches += st["gpu_launches"]
                relres = max(relres, st["max_relres"])
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    t_total = max_over_ranks(float(np.sum(step_ms)) / 1e3, dist if world > 1 else None, dev)
    value = whole_job_rate(rhs_per_step, world, args.steps, t_total)

    # end to end through the public API with pinned host buffers
    e2e_steps = max(3, args.steps // 2)
    step(device_inputs=False)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    tt = 0.0
    for _ in range(e2e_steps):
        flush.zero_()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        step(device_inputs=False)
        torch.cuda.synchronize()
        tt += time.perf_counter() - t1
    tt = max_over_ranks(tt, dist if world > 1 else None, dev)
    h2d = sum(k.numel() * k.element_size() + lb.numel() * lb.element_size() for k, lb in med_host)
    d2h = sum(e.numel() * e.element_size() for e in E_host)
    e2e_value = whole_job_rate(rhs_per_step, world, e2e_steps, tt)

    # the macroscopic problem (Sec. 2, Eq. macro_eq) from the last step's coefficients, outside
    # the timed region: source densities of every level and the macro solve (CUDA events)
    try:
        macro_info = macro_leg(s, wl, E_dev, stream)
    except Exception as ex:  # an auxiliary record must not cost the benchmark line
        macro_info = {"error": f"{type(ex).__name__}: {ex}"[:300]}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    clocks = clk.summary()
    peaks = _peaks()
    sm_mhz = clocks.get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    fp32_peak = SMS * FP32_LANES * 2 * sm_mhz * 1e6 / 1e12
    pcg_flops = pcg_node_iters * FLOPS_PER_NODE_ITER
    achieved = pcg_flops / (pcg_ms / 1e3) / 1e12 if pcg_ms > 0 else None
    traffic, traffic_levels = ((_level_traffic() if args.precision == "mixed" and
                                wl.name == WORKLOAD and tiles == [0, 1, 1] else (None, None)))
    share = (pcg_ms / (t_total * 1e3)) if t_total > 0 else None
    if wl.dim == 2:
        roofline = {"bound": "alu", "kernel": "k_level2d (persistent level solve)",
                    "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                    "frac": (achieved / fp32_peak) if achieved else None, "traffic": traffic,
                    "traffic_per_launch_by_level": traffic_levels,
                    "peak_source": "152 SMs x 128 FP32 lanes x 2 flops x median sampled SM clock",
                    "flops_per_node_iteration": FLOPS_PER_NODE_ITER,
                    "kernel_share_of_step": share, "launches_timed": pcg_launches}
    else:
        # the 3D level kernel streams its vectors through HBM: bytes of the inner iterations
        bpn = BYTES3D_PER_NODE_ITER_UNIT + BYTES3D_PER_NODE_ITER_POINT / s.R
        gbs = pcg_node_iters * bpn / (pcg_ms / 1e3) / 1e9 if pcg_ms > 0 else None
        hbm = peaks.get("hbm_gbs")
        roofline = {"bound": "hbm", "kernel": "k_level3d (cooperative level solve)",
                    "achieved": gbs, "peak": hbm or 6800.0, "unit": "GB/s",
                    "frac": (gbs / (hbm or 6800.0)) if gbs else None, "traffic": None,
                    "peak_source": ("measured copy bandwidth" if hbm else
                                    "fallback 6.8 TB/s"),
                    "bytes_per_node_iteration": bpn,
                    "kernel_share_of_step": share, "launches_timed": pcg_launches}
    plain = None
    if not args.no_plain and wl.dim == 2:
        plain, E_plain = plain_fp64_leg(wl, med_dev, flush, 2, stream)
        plain["speedup_of_value"] = value / world / plain["value"]
        sys.path.insert(0, os.path.join(ROOT, "tests"))
        from util import block_rel_err
        plain["block_rel_diff_vs_batched"] = max(
            block_rel_err(a.cpu().numpy(), b.cpu().numpy(), wl.n_cont, wl.dim)
            for a, b in zip(E_dev, E_plain))
    cpu = None
    acc_err = None
    if not args.no_cpu:
        import tempfile
        Eg = [e.cpu().numpy() for e in E_dev]
        with tempfile.TemporaryDirectory() as td:
            fn = os.path.join(td, "eg.npz")
            np.savez(fn, **{f"E{i}": e for i, e in enumerate(Eg)})
            env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1",
                       MKL_NUM_THREADS="1")
            for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
                env.pop(k, None)
            out = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-leg", fn,
                                  "--precision", args.precision, "--workload", args.workload],
                                 capture_output=True, text=True, env=env, timeout=600)
            try:
                res = json.loads(out.stdout.strip().splitlines()[-1])
                cpu, acc_err = res["cpu"], res["err"]
            except Exception:
                cpu = {"error": out.stderr[-400:]}
    line = {"metric": METRIC, "value": value, "unit": "RHS/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(args.warmup, 3),
            "ms_per_step": float(np.mean(step_ms)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
            "config": dict(_config(wl, args.precision), rhs_per_step=rhs_per_step,
                           level_tiles=tiles),
            "roofline": roofline, "cpu_baseline": cpu, "plain_fp64_per_point": plain,
            "e2e": {"value": e2e_value, "unit": "RHS/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": launches, "clocks": clocks,
            "accuracy": {"max_relres": relres, "sampled_block_rel_err_vs_oracle": acc_err},
            "macro": macro_info}
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
