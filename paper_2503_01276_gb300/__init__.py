"""GB300 (sm_103a) hierarchical multicontinuum homogenization: batched constrained cell
problems, interpolation-plus-correction hierarchy and effective coefficients.

The compute path is the C-ABI library ``libmch.so`` (include/mch.h); this package only
marshals arguments to it. The library is loaded on first use of any name below, and that
raises ImportError if it has not been built (``paper_2503_01276_gb300.build.build()``).
"""
_EXPORTS = ("MCH_FP64", "MCH_MIXED", "LIB_PATH", "MchDesc", "MchError", "Solver",
            "desc_from_workload", "direct_noalloc", "load_library", "make_desc", "plan_level")

__all__ = list(_EXPORTS) + ["homogenize", "HomogenizeFn"]


def __getattr__(name):
    if name in _EXPORTS:
        from . import _mch
        return getattr(_mch, name)
    if name in ("homogenize", "HomogenizeFn"):
        from . import autograd
        return getattr(autograd, name)
    raise AttributeError(name)
