"""Oracle for the KIFMM boundary sums -- TEST INFRASTRUCTURE ONLY.

Plain, slow, obviously-correct CPU implementations of what the GPU library
computes, written from the paper:

* ``direct``       -- FP64 O(N^2) single-layer / double-layer / adjoint-double-layer
                      sums (Sec. II.A Eq. sum_fmm; Eq. kernel; Eq. kernel_pol) in C.
* ``quadrature``   -- one-point centroid rule with spherical or flat areas (Sec. III).
* ``bie``          -- the polarization operator A sigma (Eqs. Ax, Eb, pol_discret),
                      its right-hand side (Eq. rhs) and the demagnetizing phi_2
                      (Eq. fk_integral_discrete).
* ``gmres``        -- plain restarted GMRES (Saad & Schultz), matrix-free (Sec. III).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
may import this package.  It shares no code with ``paper_1605_01715_gb300``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "oracle.c")
_lock = threading.Lock()
_lib = None

KERNELS = {"sl": 0, "dl": 1, "adl": 2}
DELTA = 1e-5  # tolerance radius of Sec. III.A.1


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so with gcc + OpenMP."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp.%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            lib.oracle_direct.restype = ctypes.c_int
            lib.oracle_direct.argtypes = [
                ctypes.c_int,
                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                ctypes.c_void_p, ctypes.c_int64,
                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                ctypes.c_double, ctypes.c_void_p, ctypes.c_int]
            lib.oracle_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def _soa(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.ndim != 2 or a.shape[0] != 3:
        raise ValueError("expected a (3, n) structure-of-arrays array")
    if n is not None and a.shape[1] != n:
        raise ValueError("length mismatch")
    return a


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def direct(kernel: str, trg, src, q, src_nrm=None, trg_nrm=None, idx=None,
           delta: float = DELTA, nthreads: int = 0) -> np.ndarray:
    """FP64 direct sum f_i = sum_j K(r_i, r_j) q_j at targets ``idx`` (default all)."""
    lib = _load()
    trg = _soa(trg)
    src = _soa(src)
    nt, ns = trg.shape[1], src.shape[1]
    q = np.ascontiguousarray(q, dtype=np.float64)
    if q.shape != (ns,):
        raise ValueError("q must have one entry per source")
    sn = _soa(src_nrm, ns) if src_nrm is not None else None
    tn = _soa(trg_nrm, nt) if trg_nrm is not None else None
    if idx is not None:
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        if idx.size and (idx.min() < 0 or idx.max() >= nt):
            raise ValueError("target index out of range")
        nout = idx.size
    else:
        nout = nt
    out = np.empty(nout, dtype=np.float64)
    rc = lib.oracle_direct(KERNELS[kernel],
                           trg.ctypes.data, tn.ctypes.data if tn is not None else None, nt,
                           idx.ctypes.data if idx is not None else None,
                           nout if idx is not None else 0,
                           src.ctypes.data, sn.ctypes.data if sn is not None else None,
                           q.ctypes.data, ns, float(delta), out.ctypes.data, int(nthreads))
    if rc != 0:
        raise ValueError("oracle_direct: bad arguments for kernel %s" % kernel)
    return out


from . import quadrature, gmres, bie  # noqa: E402,F401
