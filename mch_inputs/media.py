"""Synthetic high-contrast media on macropoint RVE grids.

A medium is a global function of position built from periods of side
eps = rve_len / P (P = the workload's medium_periods, by default its constraint
sub-block count). Every RVE starts on a period boundary, so an element of
an RVE grid with m = n / P elements per period sits at period-local
coordinate t = (i mod m + 1/2) / m along each axis (exact in binary for the
power-of-two m used here) inside global period K = K0 + i div m. All random
draws (channel offsets, inclusion log-conductivities) are keyed by the global
period index through a counter-based hash, so overlapping RVEs of different
macropoints, and the same macropoint at different resolutions, see the same
medium.

Families (continuum labels in parentheses):
  channel2d       horizontal channel of width eps/4 in rows [3/8+d, 5/8+d) of
                  each period, d in {-1/8, 0, +1/8} per period (label 0,
                  kappa = contrast); matrix elsewhere (label 1, kappa = 1);
                  both times 1 + 0.5 sin(2 pi x) sin(2 pi y).
  channel_incl2d  channel rows [1/8+d, 3/8+d) (label 0, kappa = contrast);
                  disc of radius 0.15 eps at (eps/2, 0.7 eps) (label 1,
                  kappa = 1e3 exp(0.5 Z), Z ~ N(0,1) per period); matrix
                  (label 2, kappa = 1).
  layered2d       periodic layers: channel rows [1/4, 1/2) of every period (label 0,
                  kappa = contrast), matrix elsewhere (label 1, kappa = 1); both
                  times the slowly varying g = 2 + sin(pi x) sin(pi y) of Sec. 4.
                  No random draw, and the layer edges fall on element edges of every
                  grid with at least 4 elements per period, so every level of a
                  hierarchy sees the same layers (only g is sampled per grid).
  channel3d       channel along x with square cross-section [3/8, 5/8)^2 in
                  (y, z) period coordinates (label 0, kappa = contrast);
                  matrix (label 1, kappa = 1); both times
                  1 + 0.5 sin(2 pi x) sin(2 pi y) sin(2 pi z).
"""
from __future__ import annotations

import numpy as np

from .configs import Workload

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def _splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser (Steele, Lea, Flood 2014) on a uint64 array."""
    with np.errstate(over="ignore"):
        z = (x + np.uint64(0x9E3779B97F4A7C15)) & _M64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
        return z ^ (z >> np.uint64(31))


def counter_uniform(seed: int, stream: int, kx, ky, kz=0) -> np.ndarray:
    """Uniform [0,1) draw keyed by (seed, stream, global period index)."""
    kx = np.asarray(kx, dtype=np.int64)
    ky = np.asarray(ky, dtype=np.int64)
    kz = np.asarray(kz, dtype=np.int64)
    off = np.int64(1 << 20)
    key = _splitmix64(np.full(np.broadcast(kx, ky, kz).shape,
                              np.uint64(seed * 1024 + stream), dtype=np.uint64))
    key = _splitmix64(key ^ (kx + off).astype(np.uint64))
    key = _splitmix64(key ^ ((ky + off).astype(np.uint64) << np.uint64(21)))
    key = _splitmix64(key ^ ((kz + off).astype(np.uint64) << np.uint64(42)))
    return (key >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def macro_points_xyz(wl: Workload, idx: np.ndarray) -> np.ndarray:
    """Physical centres of macropoints given integer macro indices [npts, d]."""
    return wl.origin + np.asarray(idx, dtype=np.float64) * wl.spacing


def _grids(wl: Workload, idx: np.ndarray, n: int):
    """Per point and element: global period index K and local coordinate t."""
    d = wl.dim
    P = wl.medium_periods or wl.periods
    if n % P:
        raise ValueError(f"RVE grid {n} is not a multiple of the period count {P}")
    m = n // P
    eps = wl.rve_len / P
    centres = macro_points_xyz(wl, idx)                       # [np, d]
    k0f = (centres - wl.rve_len / 2) / eps
    k0 = np.rint(k0f).astype(np.int64)
    if np.max(np.abs(k0f - k0)) > 1e-6:
        raise ValueError("RVE origins are not aligned with period boundaries")
    e = np.arange(n ** d)
    flat = [(e // (n ** a)) % n for a in range(d)]           # axis a index, x fastest
    K = np.stack([k0[:, a][:, None] + (flat[a] // m)[None, :] for a in range(d)])  # [d, np, ne]
    t = np.stack([np.broadcast_to(((flat[a] % m) + 0.5) / m, K.shape[1:]) for a in range(d)])
    x = (K + t) * eps
    return K, t, x


def media(wl: Workload, idx, n: int):
    """kappa [npts, n^d] float64 and labels [npts, n^d] uint8 for the RVEs of
    macropoints with integer macro indices ``idx`` [npts, d] on an n^d grid.
    Element order is lexicographic with x fastest."""
    idx = np.atleast_2d(np.asarray(idx, dtype=np.int64))
    if idx.shape[1] != wl.dim:
        raise ValueError("point indices must have one column per dimension")
    K, t, x = _grids(wl, idx, n)
    seed = wl.seed
    if wl.family == "channel2d":
        u = counter_uniform(seed, 1, K[0], K[1])
        dlt = (np.floor(3.0 * u) - 1.0) / 8.0
        lo = 3.0 / 8.0 + dlt
        hi = 5.0 / 8.0 + dlt
        chan = (t[1] >= lo) & (t[1] < hi)
        labels = np.where(chan, 0, 1).astype(np.uint8)
        g = 1.0 + 0.5 * np.sin(2 * np.pi * x[0]) * np.sin(2 * np.pi * x[1])
        kappa = np.where(chan, wl.contrast, 1.0) * g
    elif wl.family == "layered2d":
        chan = (t[1] >= 1.0 / 4.0) & (t[1] < 1.0 / 2.0)
        labels = np.where(chan, 0, 1).astype(np.uint8)
        g = 2.0 + np.sin(np.pi * x[0]) * np.sin(np.pi * x[1])
        kappa = np.where(chan, wl.contrast, 1.0) * g
    elif wl.family == "channel_incl2d":
        u = counter_uniform(seed, 1, K[0], K[1])
        dlt = (np.floor(3.0 * u) - 1.0) / 8.0
        chan = (t[1] >= 1.0 / 8.0 + dlt) & (t[1] < 3.0 / 8.0 + dlt)
        incl = (t[0] - 0.5) ** 2 + (t[1] - 0.7) ** 2 < 0.15 ** 2
        u1 = counter_uniform(seed, 2, K[0], K[1])
        u2 = counter_uniform(seed, 3, K[0], K[1])
        z = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)  # Box-Muller
        labels = np.where(chan, 0, np.where(incl, 1, 2)).astype(np.uint8)
        kappa = np.where(chan, wl.contrast, np.where(incl, 1e3 * np.exp(0.5 * z), 1.0))
    elif wl.family == "channel3d":
        if wl.dim != 3:
            raise ValueError("channel3d is a 3D medium")
        chan = ((t[1] >= 3.0 / 8.0) & (t[1] < 5.0 / 8.0) &
                (t[2] >= 3.0 / 8.0) & (t[2] < 5.0 / 8.0))
        labels = np.where(chan, 0, 1).astype(np.uint8)
        g = 1.0 + 0.5 * (np.sin(2 * np.pi * x[0]) * np.sin(2 * np.pi * x[1])
                         * np.sin(2 * np.pi * x[2]))
        kappa = np.where(chan, wl.contrast, 1.0) * g
    else:
        raise ValueError(f"unknown medium family {wl.family!r}")
    return np.ascontiguousarray(kappa, dtype=np.float64), np.ascontiguousarray(labels)
