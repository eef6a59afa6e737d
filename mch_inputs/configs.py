"""Workload descriptions for the hierarchical cell-problem solve.

Each workload fixes the macroscopic grid (``macro_n`` points per axis with
physical spacing ``spacing`` and first coordinate ``origin``), the nested
macrogrid strides T_1 ... T_L in macro-index units (the grid-refinement
hierarchy of Sec. 3.1), the FE resolution of the level-1 RVE grid
(``n_fine`` elements per side, coarsened by ``eta`` per level as in Sec. 3.2),
the number P of periods per RVE side (the constraint sub-blocks R_q), the
medium family, its contrast and seed.

The five full-size workloads describe: a 2D two-continuum channel medium on
4x4 points without hierarchy (n=32); the same family on 17x17 points with
three levels (RVE grids 128/64/32); a three-continuum 2D medium on 33x33
points with four levels (256/128/64/32); a 3D two-continuum medium on 9^3
points with three levels (64/32/16); and the 2D channel family at contrast
1e5 on 65x65 points with three levels, used for the adjoint.
"""
from __future__ import annotations

from dataclasses import dataclass, replace


@dataclass(frozen=True)
class Workload:
    name: str
    dim: int
    n_cont: int
    n_levels: int
    eta: int
    macro_n: int
    strides: tuple
    n_fine: int
    periods: int
    spacing: float
    origin: float
    rve_len: float
    family: str
    contrast: float
    seed: int = 1
    precision: str = "mixed"  # "fp64" | "mixed"
    interp: str = "multilinear"  # "multilinear" | "nearest1" (nearest point of S_1)
    overs: int = 0               # oversampling layers: R_p = central (P - 2 overs)^d periods
    medium_periods: int = 0      # medium periods per RVE side (0: the constraint sub-blocks P)

    @property
    def n_rhs(self) -> int:
        return self.n_cont * (1 + self.dim)

    def n_level(self, level: int) -> int:
        """Elements per RVE side at level ``level`` (1-based)."""
        return self.n_fine // (self.eta ** (level - 1))


WORKLOADS = {
    "channel2d_4x4_n32": Workload(
        name="channel2d_4x4_n32", dim=2, n_cont=2, n_levels=1, eta=2, macro_n=4,
        strides=(1,), n_fine=32, periods=4, spacing=0.25, origin=0.125,
        rve_len=0.25, family="channel2d", contrast=1e4, seed=1, precision="fp64"),
    "channel2d_17x17_L3": Workload(
        name="channel2d_17x17_L3", dim=2, n_cont=2, n_levels=3, eta=2, macro_n=17,
        strides=(8, 2, 1), n_fine=128, periods=4, spacing=1.0 / 16, origin=0.0,
        rve_len=1.0 / 16, family="channel2d", contrast=1e4, seed=2),
    "incl2d_33x33_L4": Workload(
        name="incl2d_33x33_L4", dim=2, n_cont=3, n_levels=4, eta=2, macro_n=33,
        strides=(8, 4, 2, 1), n_fine=256, periods=4, spacing=1.0 / 32, origin=0.0,
        rve_len=1.0 / 32, family="channel_incl2d", contrast=1e6, seed=3),
    "channel3d_9x9x9_L3": Workload(
        name="channel3d_9x9x9_L3", dim=3, n_cont=2, n_levels=3, eta=2, macro_n=9,
        strides=(8, 2, 1), n_fine=64, periods=4, spacing=1.0 / 8, origin=0.0,
        rve_len=1.0 / 8, family="channel3d", contrast=1e4, seed=4),
    "channel2d_65x65_L3_adj": Workload(
        name="channel2d_65x65_L3_adj", dim=2, n_cont=2, n_levels=3, eta=2, macro_n=65,
        strides=(4, 2, 1), n_fine=128, periods=4, spacing=1.0 / 64, origin=0.0,
        rve_len=1.0 / 64, family="channel2d", contrast=1e5, seed=5),
}


def workload(name: str, **overrides) -> Workload:
    wl = WORKLOADS[name]
    return replace(wl, **overrides) if overrides else wl


def small_workload(name: str, n_fine: int, macro_n: int | None = None,
                   strides: tuple | None = None, **overrides) -> Workload:
    """A reduced copy of a workload (smaller RVE grid and/or macrogrid) for
    tests the oracle finishes in seconds. The spacing and RVE length are kept
    consistent (rve_len = spacing) when the macrogrid changes."""
    wl = WORKLOADS[name]
    kw = dict(n_fine=n_fine)
    if macro_n is not None:
        kw["macro_n"] = macro_n
        if wl.origin == 0.0:
            sp = 1.0 / (macro_n - 1)
        else:
            sp = 1.0 / macro_n
            kw["origin"] = sp / 2
        kw["spacing"] = sp
        kw["rve_len"] = sp
    if strides is not None:
        kw["strides"] = tuple(strides)
        kw["n_levels"] = len(strides)
    kw.update(overrides)
    return replace(wl, **kw)
