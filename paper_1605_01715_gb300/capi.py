"""Thin ctypes binding of include/kifmm.h.

Every function here only marshals arguments: torch CUDA tensors become device
pointers, the current torch stream becomes the ``stream`` argument, and a non-zero
status raises ``KifmmError``.  All computation happens in libkifmm.so.  There is no
fallback: if the library is missing or no CUDA device is present, calls fail.

The functions keep the C names; ``Tree`` and ``Plan`` own the handles.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkifmm.so")

KERNELS = {"sl": 0, "dl": 1, "adl": 2, "field": 3}
PRECISIONS = {"fp64": 0, "mixed": 1, "cheb_fp64": 16}   # cheb_fp64: Chebyshev far field, FP64
LISTS = {"U": 0, "V": 1, "W": 2, "X": 3}
STATUS = {0: "OK", -1: "INVALID_ARG", -2: "OOM", -3: "CUDA", -4: "NOT_CONVERGED",
          -5: "TIMEOUT", -6: "BREAKDOWN", -7: "UNSUPPORTED"}

_lock = threading.Lock()
_lib = None


class KifmmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (STATUS.get(code, "?"), code, msg))
        self.code = code
        self.status = STATUS.get(code, "?")


class TreeStats(ctypes.Structure):
    _fields_ = [("n_src", ctypes.c_int64), ("n_trg", ctypes.c_int64),
                ("n_boxes", ctypes.c_int32), ("n_leaves", ctypes.c_int32),
                ("n_levels", ctypes.c_int32), ("max_leaf", ctypes.c_int32),
                ("n_u", ctypes.c_int64), ("n_v", ctypes.c_int64), ("n_w", ctypes.c_int64),
                ("n_x", ctypes.c_int64), ("p2p_pairs", ctypes.c_int64),
                ("root_center", ctypes.c_double * 3), ("root_half", ctypes.c_double),
                ("n_instances", ctypes.c_int32), ("forest_level", ctypes.c_int32)]


class PlanStats(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int32), ("p", ctypes.c_int32), ("q_points", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("pinv_cutoff", ctypes.c_double),
                ("device_bytes", ctypes.c_int64), ("m2l_pairs", ctypes.c_int64),
                ("u2u_pairs", ctypes.c_int64), ("l2l_pairs", ctypes.c_int64),
                ("s2u_leaves", ctypes.c_int64), ("x_pairs", ctypes.c_int64),
                ("launches_per_matvec", ctypes.c_int32), ("rank_up", ctypes.c_int32),
                ("rank_down", ctypes.c_int32), ("m2l_width", ctypes.c_int32),
                ("m2l_rows", ctypes.c_int32), ("near_units", ctypes.c_int32),
                ("near_split_leaves", ctypes.c_int32), ("near_overlap", ctypes.c_int32),
                ("s2u_points", ctypes.c_int32), ("m2l_chain_pairs", ctypes.c_int64),
                ("pinv_cutoff_up", ctypes.c_double), ("near_corr_ranges", ctypes.c_int64),
                ("near_pairs", ctypes.c_int64), ("near_axis_units", ctypes.c_int32),
                ("setup_ms", ctypes.c_double * 5), ("near_axis_pairs", ctypes.c_int64),
                ("near_zero_pairs", ctypes.c_int64)]


def _as_dict(st):
    out = {}
    for k, _ in st._fields_:
        v = getattr(st, k)
        out[k] = list(v) if isinstance(v, ctypes.Array) else v
    return out


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_SIGS = {
    "kifmm_last_error": ([], ctypes.c_char_p),
    "kifmm_version": ([], ctypes.c_char_p),
    "kifmm_quadrature_points": ([_P, _P, _I64, _P, _P, _P, _P], ctypes.c_int),
    "kifmm_tree_build": ([_P, _I64, _P, _I64, ctypes.c_int, _P, ctypes.POINTER(_P)], ctypes.c_int),
    "kifmm_forest_build": ([_P, _I64, _P, ctypes.c_int, ctypes.c_int, _P, ctypes.POINTER(_P)], ctypes.c_int),
    "kifmm_tree_get_stats": ([_P, ctypes.POINTER(TreeStats)], ctypes.c_int),
    "kifmm_tree_export": ([_P, _P, _P, _P, _P, _P, _P, _P], ctypes.c_int),
    "kifmm_tree_export_list": ([_P, ctypes.c_int, _P, _P], ctypes.c_int),
    "kifmm_tree_destroy": ([_P], ctypes.c_int),
    "kifmm_fmm_setup": ([_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, _P, _P, _P,
                         ctypes.POINTER(_P)], ctypes.c_int),
    "kifmm_fmm_matvec": ([_P, _P, _P, _P], ctypes.c_int),
    "kifmm_fmm_matvec_graph": ([_P, _P, _P, _P], ctypes.c_int),
    "kifmm_fmm_matvec_host": ([_P, _P, _P, ctypes.c_int, _P], ctypes.c_int),
    "kifmm_plan_get_stats": ([_P, ctypes.POINTER(PlanStats)], ctypes.c_int),
    "kifmm_up_skeleton": ([ctypes.c_int, ctypes.c_int, _P, _P, _P], ctypes.c_int),
    "kifmm_plan_profile": ([_P, ctypes.c_int, _P], ctypes.c_int),
    "kifmm_plan_check": ([_P], ctypes.c_int),
    "kifmm_plan_destroy": ([_P], ctypes.c_int),
    "kifmm_polarization_rhs": ([_P, _P, ctypes.c_double, _P, _I64, _P, _P], ctypes.c_int),
    "kifmm_solver_create": ([_P, _P, _P, ctypes.c_double, _P, _P, _P, ctypes.c_double, ctypes.c_int,
                             ctypes.c_int, ctypes.POINTER(_P)], ctypes.c_int),
    "kifmm_solver_launch": ([_P, _P], ctypes.c_int),
    "kifmm_solver_finish": ([_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                             ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "kifmm_solver_destroy": ([_P], ctypes.c_int),
    "kifmm_solver_instances": ([_P, ctypes.c_int, _P, _P, _P], ctypes.c_int),
    "kifmm_bie_solve": ([_P, _P, _P, ctypes.c_double, _P, _P, _P, ctypes.c_double, ctypes.c_int,
                         ctypes.c_int, _P, _P, _P], ctypes.c_int),
    "kifmm_bie_apply": ([_P, _P, _P, ctypes.c_double, _P, _P, _P, _P], ctypes.c_int),
    "kifmm_demag_phi2": ([_P, _P, _P, _P, _P, _P], ctypes.c_int),
    "kifmm_demag_phi2_noalloc": ([_P, _P, _P, _P, _P, _P], ctypes.c_int),
    "kifmm_polarization_rhs_free": ([_P, _P, _P, ctypes.c_double, _P, _P, _P, _P, _P, _P], ctypes.c_int),
    "kifmm_polarization_field": ([_P, _P, _P, _P, _P, _P, _P, _P], ctypes.c_int),
    "kifmm_polarization_force": ([_P, _P, _P, _P, _P, ctypes.c_double, _P, _P, ctypes.c_int, _P, _P], ctypes.c_int),
    "kifmm_peak_rate": ([ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                         ctypes.POINTER(ctypes.c_double), _P], ctypes.c_int),
}


def lib():
    """Load libkifmm.so (built by ``__graft_entry__.build()``); raise if absent."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError("libkifmm.so not built: run `python -c 'import __graft_entry__ as g; "
                                  "g.build()'` (no CPU fallback exists)")
            L = ctypes.CDLL(LIB_PATH)
            for name, (args, res) in _SIGS.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def _check(rc):
    if rc != 0:
        raise KifmmError(rc, lib().kifmm_last_error().decode())


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _dev(t, n=None, name="tensor"):
    if t is None:
        return None
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("%s must be a contiguous float64 CUDA tensor" % name)
    if n is not None and t.numel() != n:
        raise ValueError("%s must have %d elements, has %d" % (name, n, t.numel()))
    return ctypes.c_void_p(t.data_ptr())


def _host(t, n, name="tensor"):
    if not (isinstance(t, torch.Tensor) and t.device.type == "cpu" and t.dtype == torch.float64
            and t.is_contiguous()):
        raise TypeError("%s must be a contiguous float64 CPU tensor" % name)
    if t.numel() != n:
        raise ValueError("%s must have %d elements, has %d" % (name, n, t.numel()))
    return ctypes.c_void_p(t.data_ptr())


def kifmm_version() -> str:
    return lib().kifmm_version().decode()


def kifmm_quadrature_points(tri, sph, stream=None):
    """tri (T,3,3) and sph (T,4) float64 CUDA -> xyz (3,T), w (T,), nrm (3,T)."""
    n = tri.shape[0]
    xyz = torch.empty((3, n), dtype=torch.float64, device=tri.device)
    w = torch.empty(n, dtype=torch.float64, device=tri.device)
    nrm = torch.empty((3, n), dtype=torch.float64, device=tri.device)
    _check(lib().kifmm_quadrature_points(_dev(tri, 9 * n, "tri"), _dev(sph, 4 * n, "sph"), n,
                                         _dev(xyz), _dev(w), _dev(nrm), _stream(stream)))
    return xyz, w, nrm


class Tree:
    """Owns a kifmm_tree handle (kifmm_tree_build / kifmm_forest_build /
    kifmm_tree_destroy).  ``instances``: offsets (n_inst + 1 ints, 0 ... n) of
    independent instances stored back to back in ``src_xyz`` -- a forest, where each
    instance is its own sources and targets (``trg_xyz`` must then be None)."""

    def __init__(self, src_xyz, trg_xyz=None, max_leaf=64, stream=None, instances=None):
        h = ctypes.c_void_p()
        ns = src_xyz.shape[-1]
        if instances is not None:
            if trg_xyz is not None:
                raise ValueError("a forest's targets are its sources")
            off = np.ascontiguousarray(instances, dtype=np.int64)
            _check(lib().kifmm_forest_build(_dev(src_xyz, 3 * ns, "src_xyz"), ns, off.ctypes.data,
                                            int(off.size - 1), int(max_leaf), _stream(stream),
                                            ctypes.byref(h)))
        else:
            nt = trg_xyz.shape[-1] if trg_xyz is not None else 0
            _check(lib().kifmm_tree_build(_dev(src_xyz, 3 * ns, "src_xyz"), ns,
                                          _dev(trg_xyz, 3 * nt, "trg_xyz"), nt, int(max_leaf),
                                          _stream(stream), ctypes.byref(h)))
        self.handle = h
        self._lib = lib()

    def stats(self):
        st = TreeStats()
        _check(lib().kifmm_tree_get_stats(self.handle, ctypes.byref(st)))
        return _as_dict(st)

    def export(self):
        import numpy as np
        st = self.stats()
        nb = st["n_boxes"]
        lvl = np.empty(nb, np.int32)
        coord = np.empty(3 * nb, np.int32)
        parent = np.empty(nb, np.int32)
        leaf = np.empty(nb, np.int32)
        rng = np.empty(4 * nb, np.int64)
        sperm = np.empty(st["n_src"], np.int64)
        tperm = np.empty(st["n_trg"], np.int64)
        _check(lib().kifmm_tree_export(self.handle, lvl.ctypes.data, coord.ctypes.data, parent.ctypes.data,
                                       leaf.ctypes.data, rng.ctypes.data, sperm.ctypes.data,
                                       tperm.ctypes.data))
        return dict(level=lvl, coord=coord.reshape(nb, 3), parent=parent, leaf=leaf.astype(bool),
                    range=rng.reshape(nb, 4), src_perm=sperm, trg_perm=tperm)

    def list(self, which):
        import numpy as np
        nb = self.stats()["n_boxes"]
        off = np.empty(nb + 1, np.int64)
        _check(lib().kifmm_tree_export_list(self.handle, LISTS[which], off.ctypes.data, None))
        idx = np.empty(max(1, int(off[-1])), np.int32)
        _check(lib().kifmm_tree_export_list(self.handle, LISTS[which], None, idx.ctypes.data))
        return off, idx[: int(off[-1])]

    def close(self):
        if getattr(self, "handle", None):
            self._lib.kifmm_tree_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Plan:
    """Owns a kifmm_plan handle (kifmm_fmm_setup / kifmm_plan_destroy)."""

    def __init__(self, tree: Tree, kernel="sl", p=6, precision="fp64", pinv_cutoff=0.0,
                 src_nrm=None, trg_nrm=None, stream=None):
        h = ctypes.c_void_p()
        st = tree.stats()
        _check(lib().kifmm_fmm_setup(tree.handle, KERNELS[kernel], int(p), PRECISIONS[precision],
                                     float(pinv_cutoff),
                                     _dev(src_nrm, 3 * st["n_src"], "src_nrm") if kernel == "dl" else None,
                                     _dev(trg_nrm, 3 * st["n_trg"], "trg_nrm") if kernel == "adl" else None,
                                     _stream(stream), ctypes.byref(h)))
        self.handle = h
        self.tree = tree  # keep the tree alive
        self.n_src = st["n_src"]
        self.n_trg = st["n_trg"]
        self.kernel = kernel
        self.n_out = self.n_trg * (3 if kernel == "field" else 1)   # the field: x, y, z blocks
        self._lib = lib()

    def matvec(self, q, out=None, stream=None):
        if out is None:
            out = torch.empty(self.n_out, dtype=torch.float64, device=q.device)
        _check(lib().kifmm_fmm_matvec(self.handle, _dev(q, self.n_src, "q"), _dev(out, self.n_out, "out"),
                                      _stream(stream)))
        return out

    def matvec_graph(self, q, out, stream=None):
        """kifmm_fmm_matvec_graph: replay a captured matvec reading ``q`` and writing
        ``out`` by address (both must stay allocated; refill ``q`` in place)."""
        _check(lib().kifmm_fmm_matvec_graph(self.handle, _dev(q, self.n_src, "q"),
                                            _dev(out, self.n_out, "out"), _stream(stream)))
        return out

    def matvec_host(self, q, out, graph=True, stream=None):
        """kifmm_fmm_matvec_host: ``q`` and ``out`` are CPU float64 tensors.  Pinned
        ones are read and written in place by the first and last kernels (asynchronous:
        synchronize the stream before reading ``out``), pageable ones staged.  ``graph``
        replays a matvec captured for this pair."""
        _check(lib().kifmm_fmm_matvec_host(self.handle, _host(q, self.n_src, "q"), _host(out, self.n_out, "out"),
                                           1 if graph else 0, _stream(stream)))
        return out

    def check(self):
        """kifmm_plan_check: raise KifmmError(TIMEOUT) if a bounded device wait gave up."""
        _check(lib().kifmm_plan_check(self.handle))

    def stats(self):
        st = PlanStats()
        _check(lib().kifmm_plan_get_stats(self.handle, ctypes.byref(st)))
        return _as_dict(st)

    def profile(self, enable=True, serial=False):
        """kifmm_plan_profile: the per-phase means since the last call, then recording
        on or off; ``serial`` runs the near field after the far field (its own time)."""
        ph = (ctypes.c_double * 9)()
        _check(lib().kifmm_plan_profile(self.handle, (2 if serial else 1) if enable else 0, ph))
        names = ["gather", "s2u", "u2u", "x", "m2l", "l2l", "d2t", "p2p", "total"]
        return dict(zip(names, list(ph)))

    def bie_apply(self, area, eps_in, eps_out, curv, x, y=None, stream=None):
        n = self.n_trg
        if y is None:
            y = torch.empty(n, dtype=torch.float64, device=x.device)
        _check(lib().kifmm_bie_apply(self.handle, _dev(area, n, "area"), _dev(eps_in, n, "eps_in"),
                                     float(eps_out), _dev(curv, n, "curv"), _dev(x, n, "x"), _dev(y, n, "y"),
                                     _stream(stream)))
        return y

    def bie_solve(self, area, eps_in, eps_out, curv, b, x=None, tol=1e-6, restart=50, max_iter=1000,
                  stream=None, raise_on_failure=True):
        n = self.n_trg
        if x is None:
            x = torch.zeros(n, dtype=torch.float64, device=b.device)
        it = ctypes.c_int(0)
        rr = ctypes.c_double(0)
        rc = lib().kifmm_bie_solve(self.handle, _dev(area, n, "area"), _dev(eps_in, n, "eps_in"),
                                   float(eps_out), _dev(curv, n, "curv"), _dev(b, n, "b"), _dev(x, n, "x"),
                                   float(tol), int(restart), int(max_iter), ctypes.byref(it), ctypes.byref(rr),
                                   _stream(stream))
        if rc != 0 and raise_on_failure:
            _check(rc)
        return x, it.value, rr.value, rc

    def polarization_rhs_free(self, area, eps_in, eps_out, curv, nrm, sigma_f, e0, b=None, stream=None):
        """kifmm_polarization_rhs_free (ADL plan): b with free surface charge sigma_f."""
        n = self.n_trg
        if b is None:
            b = torch.empty(n, dtype=torch.float64, device=area.device)
        e = (ctypes.c_double * 3)(*[float(v) for v in e0])
        _check(lib().kifmm_polarization_rhs_free(self.handle, _dev(area, n, "area"), _dev(eps_in, n, "eps_in"),
                                                 float(eps_out), _dev(curv, n, "curv"), _dev(nrm, 3 * n, "nrm"),
                                                 _dev(sigma_f, n, "sigma_f"), e, _dev(b, n, "b"), _stream(stream)))
        return b

    def polarization_field(self, area, curv, nrm, sigma, e0=(0.0, 0.0, 0.0), E=None, stream=None):
        """kifmm_polarization_field (FIELD plan): E^j at the elements, (3, n)."""
        n = self.n_trg
        if E is None:
            E = torch.empty((3, n), dtype=torch.float64, device=area.device)
        e = (ctypes.c_double * 3)(*[float(v) for v in e0])
        _check(lib().kifmm_polarization_field(self.handle, _dev(area, n, "area"), _dev(curv, n, "curv"),
                                              _dev(nrm, 3 * n, "nrm"), _dev(sigma, n, "sigma"), e,
                                              _dev(E, 3 * n, "E"), _stream(stream)))
        return E

    def polarization_force(self, area, curv, nrm, sigma, eps_out, body, n_body, e0=(0.0, 0.0, 0.0), F=None,
                           stream=None):
        """kifmm_polarization_force (FIELD plan): the force on each body, (n_body, 3)."""
        n = self.n_trg
        if not (isinstance(body, torch.Tensor) and body.is_cuda and body.dtype == torch.int32
                and body.is_contiguous() and body.numel() == n):
            raise TypeError("body must be a contiguous int32 CUDA tensor of n elements")
        if F is None:
            F = torch.empty((int(n_body), 3), dtype=torch.float64, device=area.device)
        e = (ctypes.c_double * 3)(*[float(v) for v in e0])
        _check(lib().kifmm_polarization_force(self.handle, _dev(area, n, "area"), _dev(curv, n, "curv"),
                                              _dev(nrm, 3 * n, "nrm"), _dev(sigma, n, "sigma"), float(eps_out), e,
                                              ctypes.c_void_p(body.data_ptr()), int(n_body),
                                              _dev(F, 3 * int(n_body), "F"), _stream(stream)))
        return F

    def demag_phi2(self, phi1, w, omega, out=None, stream=None):
        n = self.n_trg
        if out is None:
            out = torch.empty(n, dtype=torch.float64, device=phi1.device)
        _check(lib().kifmm_demag_phi2(self.handle, _dev(phi1, n, "phi1"), _dev(w, n, "w"),
                                      _dev(omega, n, "omega"), _dev(out, n, "out"), _stream(stream)))
        return out

    def demag_phi2_noalloc(self, phi1, w, omega, out, stream=None):
        """kifmm_demag_phi2_noalloc: `out` must be preallocated; nothing is allocated."""
        n = self.n_trg
        _check(lib().kifmm_demag_phi2_noalloc(self.handle, _dev(phi1, n, "phi1"), _dev(w, n, "w"),
                                              _dev(omega, n, "omega"), _dev(out, n, "out"), _stream(stream)))
        return out

    def close(self):
        if getattr(self, "handle", None):
            self._lib.kifmm_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def kifmm_up_skeleton(p, k):
    """Skeleton of the upward check surface of order p (host only, no GPU): returns
    (idx, E, k_tol) -- k check-point indices (int32), the Q x k interpolation matrix
    (float64) with u(c_i) = sum_m E[i, m] u(c_idx[m]), and the pivot count above 1e-9
    (include/kifmm.h, kifmm_up_skeleton)."""
    import numpy as np
    Q = 6 * (p - 1) ** 2 + 2
    idx = np.zeros(max(k, 0), dtype=np.int32)
    E = np.zeros((Q, max(k, 0)), dtype=np.float64)
    kt = ctypes.c_int32(0)
    _check(lib().kifmm_up_skeleton(int(p), int(k), idx.ctypes.data_as(_P), E.ctypes.data_as(_P),
                                   ctypes.byref(kt)))
    return idx, E, kt.value


PEAK_UNITS = {"fp32_fma": 0, "fp32x2_fma": 1, "rsqrt": 2, "fp64_fma": 3}


def kifmm_peak_rate(unit, reps=3, stream=None):
    """kifmm_peak_rate: (rate, ms) of one microbenchmark unit on the current device --
    flops/s for the FMA units, reciprocal square roots/s for "rsqrt"."""
    rate, ms = ctypes.c_double(0), ctypes.c_double(0)
    _check(lib().kifmm_peak_rate(PEAK_UNITS[unit], int(reps), ctypes.byref(rate), ctypes.byref(ms),
                                 _stream(stream)))
    return rate.value, ms.value


def kifmm_polarization_rhs(nrm, eps_in, eps_out, e0, out=None, stream=None):
    n = eps_in.numel()
    if out is None:
        out = torch.empty(n, dtype=torch.float64, device=eps_in.device)
    e = (ctypes.c_double * 3)(*[float(v) for v in e0])
    _check(lib().kifmm_polarization_rhs(_dev(nrm, 3 * n, "nrm"), _dev(eps_in, n, "eps_in"), float(eps_out), e, n,
                                        _dev(out, n, "b"), _stream(stream)))
    return out


class Solver:
    """A resumable polarization GMRES solve (kifmm_solver_*): ``launch`` enqueues the
    next step on a stream, ``finish`` waits for it and advances.  The tensors passed in
    are kept alive by the object; ``x`` is updated in place."""

    def __init__(self, plan, area, eps_in, eps_out, curv, b, x=None, tol=1e-6, restart=50, max_iter=1000):
        n = plan.n_trg
        if x is None:
            x = torch.zeros(n, dtype=torch.float64, device=b.device)
        self._keep = (plan, area, eps_in, curv, b, x)
        self.x = x
        h = ctypes.c_void_p()
        _check(lib().kifmm_solver_create(plan.handle, _dev(area, n, "area"), _dev(eps_in, n, "eps_in"),
                                         float(eps_out), _dev(curv, n, "curv"), _dev(b, n, "b"),
                                         _dev(x, n, "x"), float(tol), int(restart), int(max_iter),
                                         ctypes.byref(h)))
        self.handle = h
        self._lib = lib()
        self.n_inst = plan.tree.stats()["n_instances"]
        self.done, self.iters, self.rel_res, self.status = False, 0, float("inf"), 0

    def instances(self):
        """Per-instance (iters, rel_res, status) arrays (kifmm_solver_instances)."""
        it = np.zeros(self.n_inst, np.int32)
        rr = np.zeros(self.n_inst, np.float64)
        stt = np.zeros(self.n_inst, np.int32)
        _check(lib().kifmm_solver_instances(self.handle, self.n_inst, it.ctypes.data, rr.ctypes.data,
                                            stt.ctypes.data))
        return it, rr, stt

    def launch(self, stream=None):
        _check(lib().kifmm_solver_launch(self.handle, _stream(stream)))

    def finish(self):
        d, it, rr = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_double(0)
        rc = lib().kifmm_solver_finish(self.handle, ctypes.byref(d), ctypes.byref(it), ctypes.byref(rr))
        if rc not in (0, -4, -6):                  # OK, NOT_CONVERGED, BREAKDOWN end a solve
            _check(rc)
        self.done, self.iters, self.rel_res, self.status = bool(d.value), it.value, rr.value, rc
        return self.done

    def close(self):
        if getattr(self, "handle", None):
            self._lib.kifmm_solver_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
