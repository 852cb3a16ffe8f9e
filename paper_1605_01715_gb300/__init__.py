"""GB300 (sm_103a) kernel-independent FMM for Laplace boundary integrals.

The compute path is libkifmm.so (include/kifmm.h); this package is its ctypes
binding.  Build it with ``__graft_entry__.build()`` or ``python -m
paper_1605_01715_gb300.build``.
"""
from .capi import (  # noqa: F401
    KERNELS,
    PRECISIONS,
    KifmmError,
    Plan,
    Solver,
    Tree,
    exported_symbols,
    kifmm_peak_rate,
    kifmm_polarization_rhs,
    kifmm_quadrature_points,
    kifmm_up_skeleton,
    kifmm_version,
    lib,
)
