"""ctypes binding of libmch.so (include/mch.h); argument marshalling only.

Every computation runs inside the library's sm_103a kernels. If the shared library
has not been built this module raises at import: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmch.so")

MCH_FP64, MCH_MIXED = 0, 1
STATUS = {0: "MCH_OK", 1: "MCH_ERR_ARG", 2: "MCH_ERR_CUDA", 3: "MCH_ERR_OOM", 4: "MCH_ERR_ORDER",
          5: "MCH_ERR_NOT_CONVERGED", 6: "MCH_ERR_BREAKDOWN", 7: "MCH_ERR_DEGENERATE",
          8: "MCH_ERR_UNSUPPORTED"}


class MchError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status
        self.name = STATUS.get(status, str(status))


class MchDesc(C.Structure):
    _fields_ = [("dim", C.c_int), ("n_cont", C.c_int), ("n_levels", C.c_int), ("eta", C.c_int),
                ("macro_n", C.c_int), ("level_stride", C.POINTER(C.c_int)), ("n_fine", C.c_int),
                ("periods", C.c_int), ("overs", C.c_int), ("rve_len", C.c_double),
                ("precision", C.c_int), ("rtol", C.c_double), ("inner_tol", C.c_double),
                ("max_iter", C.c_int), ("max_refine", C.c_int), ("keep_parents", C.c_int),
                ("interp", C.c_int), ("point_batch", C.c_int)]


class MchLevelStats(C.Structure):
    _fields_ = [("n_points", C.c_int), ("n_elem", C.c_int), ("sweeps", C.c_int),
                ("max_iters", C.c_int), ("total_iters", C.c_longlong), ("max_relres", C.c_double),
                ("n_dropped_rows", C.c_int), ("gpu_launches", C.c_int),
                ("h2d_bytes", C.c_longlong), ("d2h_bytes", C.c_longlong),
                ("setup_ms", C.c_double), ("interp_ms", C.c_double), ("pcg_ms", C.c_double),
                ("prep_ms", C.c_double), ("final_ms", C.c_double), ("pcg_launches", C.c_int),
                ("pcg_node_iters", C.c_longlong), ("pcg_node_applies", C.c_longlong)]


def load_library(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_2503_01276_gb300.build.build() "
                          "(there is no non-CUDA fallback)")
    lib = C.CDLL(path)
    P = C.c_void_p
    sig = {
        "mch_create": (C.c_int, [C.POINTER(MchDesc), P, C.POINTER(P)]),
        "mch_plan_level": (C.c_int, [C.POINTER(MchDesc), C.c_int, C.POINTER(C.c_int), P, P, P, P]),
        "mch_level_num_points": (C.c_int, [P, C.c_int]),
        "mch_set_level_variant": (C.c_int, [P, C.c_int, C.c_int]),
        "mch_prepare_level": (C.c_int, [P, C.c_int, P, P]),
        "mch_get_level_variant": (C.c_int, [P, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
        "mch_autotune_level": (C.c_int, [P, C.c_int, P, P, C.POINTER(C.c_int),
                                         C.POINTER(C.c_double)]),
        "mch_level_n_elem": (C.c_int, [P, C.c_int]),
        "mch_level_points": (C.c_int, [P, C.c_int, P]),
        "mch_level_parents": (C.c_int, [P, C.c_int, P, P, P]),
        "mch_solve_level": (C.c_int, [P, C.c_int, P, P]),
        "mch_solve_level_range": (C.c_int, [P, C.c_int, C.c_int, C.c_int, P, P]),
        "mch_set_cell_functions": (C.c_int, [P, C.c_int, C.c_int, C.c_int, P]),
        "mch_effective_coeffs": (C.c_int, [P, C.c_int, P, P, P]),
        "mch_cell_functions": (C.c_int, [P, C.c_int, P]),
        "mch_level_stats_get": (C.c_int, [P, C.c_int, C.POINTER(MchLevelStats)]),
        "mch_set_timing": (C.c_int, [P, C.c_int]),
        "mch_backward": (C.c_int, [P, P, P]),
        "mch_macro_source": (C.c_int, [P, C.c_int, P, P, C.c_double, P, C.c_double, P]),
        "mch_macro_solve": (C.c_int, [P, P, P, C.c_double, C.c_double, C.c_int, P,
                                      C.POINTER(C.c_int), C.POINTER(C.c_double)]),
        "mch_direct_noalloc": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_double, C.c_int,
                                         C.c_double, C.c_int, P, P, P, P]),
        "mch_destroy": (None, [P]),
        "mch_last_error": (C.c_char_p, [P]),
        "mch_status_name": (C.c_char_p, [C.c_int]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_LIB = load_library()


def _ptr(a) -> int:
    """Data pointer of a torch tensor or numpy array (host or device)."""
    if a is None:
        return 0
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors passed to the library must be contiguous")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays passed to the library must be C-contiguous")
        return a.ctypes.data
    raise TypeError(f"unsupported buffer type {type(a)}")


def make_desc(dim, n_cont, strides, eta, macro_n, n_fine, periods, rve_len, precision="mixed",
              rtol=0.0, inner_tol=0.0, max_iter=0, max_refine=0, keep_parents=1, overs=0,
              point_batch=0, interp="multilinear"):
    arr = (C.c_int * len(strides))(*[int(s) for s in strides])
    d = MchDesc(dim=dim, n_cont=n_cont, n_levels=len(strides), eta=eta, macro_n=macro_n,
                level_stride=C.cast(arr, C.POINTER(C.c_int)), n_fine=n_fine, periods=periods,
                overs=overs, rve_len=rve_len,
                precision=MCH_FP64 if precision == "fp64" else MCH_MIXED, rtol=rtol,
                inner_tol=inner_tol, max_iter=max_iter, max_refine=max_refine,
                keep_parents=keep_parents, point_batch=point_batch,
                interp={"multilinear": 0, "nearest1": 1}[interp] if isinstance(interp, str)
                else int(interp))
    d._strides_keepalive = arr
    return d


def desc_from_workload(wl, **kw) -> MchDesc:
    args = dict(dim=wl.dim, n_cont=wl.n_cont, strides=wl.strides, eta=wl.eta,
                macro_n=wl.macro_n, n_fine=wl.n_fine, periods=wl.periods, rve_len=wl.rve_len,
                precision=wl.precision, interp=getattr(wl, "interp", "multilinear"),
                overs=getattr(wl, "overs", 0))
    args.update(kw)
    return make_desc(**args)


def direct_noalloc(n_cont, n_elem, periods, rve_len, kappa, labels, E, precision="mixed",
                   rtol=0.0, stream=None) -> int:
    """Single-level effective coefficients through mch_direct_noalloc (no device allocation;
    kappa, labels and E must be device buffers). Returns the status code."""
    if stream is None:
        try:
            import torch
            stream = torch.cuda.current_stream().cuda_stream
        except Exception:
            stream = 0
    npts = int(kappa.shape[0])
    return _LIB.mch_direct_noalloc(n_cont, n_elem, periods, rve_len,
                                   MCH_FP64 if precision == "fp64" else MCH_MIXED, rtol, npts,
                                   _ptr(kappa), _ptr(labels), _ptr(E), C.c_void_p(stream))


def plan_level(desc: MchDesc, level: int):
    """Host-only level plan: (points [n, d], parent_level, parent_pos, weights [n, 2^d])."""
    npts = C.c_int(0)
    st = _LIB.mch_plan_level(C.byref(desc), level, C.byref(npts), None, None, None, None)
    if st:
        raise MchError(st, "mch_plan_level")
    n, d = npts.value, desc.dim
    idx = np.zeros((n, d), np.int32)
    pl = np.zeros((n, 2 ** d), np.int32)
    pp = np.zeros((n, 2 ** d), np.int32)
    w = np.zeros((n, 2 ** d), np.float64)
    st = _LIB.mch_plan_level(C.byref(desc), level, C.byref(npts), _ptr(idx), _ptr(pl), _ptr(pp),
                             _ptr(w))
    if st:
        raise MchError(st, "mch_plan_level")
    return idx, pl, pp, w


class Solver:
    """One handle of the library: a level plan plus device workspaces on the current GPU."""

    def __init__(self, desc: MchDesc, stream=None):
        self.desc = desc
        self.dim, self.n_cont = desc.dim, desc.n_cont
        self.R = desc.n_cont * (1 + desc.dim)
        self.n_levels = desc.n_levels
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream
            except Exception:
                stream = 0
        self._h = C.c_void_p()
        st = _LIB.mch_create(C.byref(desc), C.c_void_p(stream), C.byref(self._h))
        if st:
            raise MchError(st, "mch_create failed")

    @classmethod
    def from_workload(cls, wl, stream=None, **kw):
        return cls(desc_from_workload(wl, **kw), stream=stream)

    def _check(self, st, what):
        if st:
            raise MchError(st, f"{what}: {_LIB.mch_last_error(self._h).decode()}")

    def num_points(self, level: int) -> int:
        return _LIB.mch_level_num_points(self._h, level)

    def n_elem(self, level: int) -> int:
        return _LIB.mch_level_n_elem(self._h, level)

    def level_points(self, level: int) -> np.ndarray:
        out = np.zeros((self.num_points(level), self.dim), np.int32)
        self._check(_LIB.mch_level_points(self._h, level, _ptr(out)), "mch_level_points")
        return out

    def level_parents(self, level: int):
        n, s = self.num_points(level), 2 ** self.dim
        pl, pp, w = np.zeros((n, s), np.int32), np.zeros((n, s), np.int32), np.zeros((n, s))
        self._check(_LIB.mch_level_parents(self._h, level, _ptr(pl), _ptr(pp), _ptr(w)),
                    "mch_level_parents")
        return pl, pp, w

    def solve_level(self, level: int, kappa, labels, allow_not_converged: bool = False) -> int:
        st = _LIB.mch_solve_level(self._h, level, _ptr(kappa), _ptr(labels))
        if st == 5 and allow_not_converged:
            return st
        self._check(st, "mch_solve_level")
        return st

    def solve_level_range(self, level: int, p0: int, p1: int, kappa=None, labels=None,
                          allow_not_converged: bool = False) -> int:
        """Points [p0, p1) of a level (mch_solve_level_range); kappa and labels hold those
        points only."""
        st = _LIB.mch_solve_level_range(self._h, level, int(p0), int(p1), _ptr(kappa),
                                        _ptr(labels))
        if st == 5 and allow_not_converged:
            return st
        self._check(st, "mch_solve_level_range")
        return st

    def set_cell_functions(self, level: int, p0: int, p1: int, phi):
        """Imports the cell functions [p1 - p0][R][(n_fine + 1)^d] of points [p0, p1) of a
        level (mch_set_cell_functions)."""
        self._check(_LIB.mch_set_cell_functions(self._h, level, int(p0), int(p1), _ptr(phi)),
                    "mch_set_cell_functions")

    def prepare_level(self, level: int, kappa, labels):
        """Stages inputs and computes the constraint data of a level on the side stream
        (mch_prepare_level); a later solve_level with the same tensors reuses it."""
        self._check(_LIB.mch_prepare_level(self._h, level, _ptr(kappa), _ptr(labels)),
                    "mch_prepare_level")

    def set_variant(self, level: int, variant: int):
        """Launch shape of the level's 2D mixed-precision solve (0 = default)."""
        self._check(_LIB.mch_set_level_variant(self._h, level, variant), "mch_set_level_variant")

    def variant(self, level: int):
        """(current launch shape, number of shapes for the level's grid)."""
        v, c = C.c_int(), C.c_int()
        self._check(_LIB.mch_get_level_variant(self._h, level, C.byref(v), C.byref(c)),
                    "mch_get_level_variant")
        return v.value, c.value

    def autotune_level(self, level: int, kappa, labels):
        """Times every valid launch shape on this level, keeps the fastest and solves with it
        (mch_autotune_level). Returns (shape, level-solve ms)."""
        b, ms = C.c_int(), C.c_double()
        self._check(_LIB.mch_autotune_level(self._h, level, _ptr(kappa), _ptr(labels),
                                            C.byref(b), C.byref(ms)), "mch_autotune_level")
        return b.value, ms.value

    def effective_coeffs(self, level: int, E=None, iters=None, relres=None):
        if E is None:
            E = np.zeros((self.num_points(level), self.R, self.R))
        self._check(_LIB.mch_effective_coeffs(self._h, level, _ptr(E), _ptr(iters), _ptr(relres)),
                    "mch_effective_coeffs")
        return E

    def cell_functions(self, level: int, out=None):
        nf = self.desc.n_fine
        if out is None:
            out = np.zeros((self.num_points(level), self.R, (nf + 1) ** self.dim))
        self._check(_LIB.mch_cell_functions(self._h, level, _ptr(out)), "mch_cell_functions")
        return out

    def set_timing(self, enable: bool = True):
        self._check(_LIB.mch_set_timing(self._h, 1 if enable else 0), "mch_set_timing")

    def stats(self, level: int) -> dict:
        s = MchLevelStats()
        self._check(_LIB.mch_level_stats_get(self._h, level, C.byref(s)), "mch_level_stats_get")
        return {k: getattr(s, k) for k, _ in MchLevelStats._fields_}

    def backward(self, dL_dE, dL_dkappa):
        P = C.c_void_p
        a = (P * self.n_levels)(*[_ptr(t) for t in dL_dE])
        b = (P * self.n_levels)(*[_ptr(t) for t in dL_dkappa])
        self._check(_LIB.mch_backward(self._h, a, b), "mch_backward")

    def macro_source(self, level: int, weights, center, alpha: float, origin, spacing: float,
                     out=None):
        """Source densities fbar [points, N] of the macroscopic problem (mch_macro_source)."""
        w = np.ascontiguousarray(weights, dtype=np.float64)
        c = np.ascontiguousarray(center, dtype=np.float64)
        o = np.ascontiguousarray(origin, dtype=np.float64)
        if w.size != self.n_cont or c.size != self.dim or o.size != self.dim:
            raise ValueError("weights need N entries, center and origin d entries")
        if out is None:
            out = np.zeros((self.num_points(level), self.n_cont))
        self._check(_LIB.mch_macro_source(self._h, level, _ptr(w), _ptr(c), float(alpha),
                                          _ptr(o), float(spacing), _ptr(out)),
                    "mch_macro_source")
        return out

    def macro_solve(self, E, fbar, spacing: float, tol: float = 1e-12, max_iter: int = 0,
                    out=None):
        """Macroscopic solve (mch_macro_solve): E and fbar per level; returns
        (U [N, (macro_n + 1)^d], iterations, relative residual)."""
        P = C.c_void_p
        a = (P * self.n_levels)(*[_ptr(t) for t in E])
        b = (P * self.n_levels)(*[_ptr(t) for t in fbar])
        if out is None:
            out = np.zeros((self.n_cont, (self.desc.macro_n + 1) ** self.dim))
        it = C.c_int(0)
        rr = C.c_double(0.0)
        self._check(_LIB.mch_macro_solve(self._h, a, b, float(spacing), float(tol), int(max_iter),
                                         _ptr(out), C.byref(it), C.byref(rr)),
                    "mch_macro_solve")
        return out, it.value, rr.value

    def close(self):
        if self._h:
            _LIB.mch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
