"""kifmm_demag_phi2_noalloc: the allocation-free entry point, through the C ABI.

It serves callers that must not allocate device memory while evaluating the
demagnetizing boundary potential (pooled allocators, latency-critical loops, graph
recording).  Its output must match kifmm_demag_phi2 on the same plan, call after
call, although its scratch is a static device array reused by every call.  This
file is collected last so that a failure here leaves the rest of the suite run.
"""
import ctypes
import math

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _plan_and_inputs(n_face):
    from paper_1605_01715_gb300 import Plan, Tree, kifmm_quadrature_points
    m = synth.cube_surface(n_face)
    tri = torch.from_numpy(np.ascontiguousarray(m.tri.reshape(-1, 9))).to(DEV)
    sph = torch.from_numpy(np.ascontiguousarray(m.sph)).to(DEV)
    xyz, w, nrm = kifmm_quadrature_points(tri, sph)
    plan = Plan(Tree(xyz, max_leaf=32), kernel="dl", p=8, precision="mixed", src_nrm=nrm)
    return plan, xyz, w


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def test_noalloc_matches_allocating_entry_point_twice():
    from paper_1605_01715_gb300 import capi
    plan, xyz, w = _plan_and_inputs(18)
    omega = torch.full_like(w, 2 * math.pi)
    outs = []
    for scale in (1.0, -2.5):                      # two calls in a row, different data
        phi1 = (4 * math.pi * scale * (xyz[2] + 0.3 * xyz[0])).contiguous()
        ref = plan.demag_phi2(phi1, w, omega)
        out = torch.full_like(phi1, float("nan"))  # every entry must be written
        lib = capi.lib()
        rc = lib.kifmm_demag_phi2_noalloc(plan.handle, ctypes.c_void_p(phi1.data_ptr()),
                                          ctypes.c_void_p(w.data_ptr()), ctypes.c_void_p(omega.data_ptr()),
                                          ctypes.c_void_p(out.data_ptr()),
                                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == 0, lib.kifmm_last_error()
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        assert _rel(out, ref) < 1e-6
        outs.append(out)
    assert _rel(outs[1], -2.5 * outs[0]) < 1e-6


def test_noalloc_on_a_fresh_plan_takes_no_device_memory():
    """On a plan that has never run an allocating call: after one warm-up call (which may
    load the library's module and so place the static array), further calls leave the
    device's free memory unchanged, and each result matches kifmm_demag_phi2, which runs
    only after all the no-alloc calls."""
    plan, xyz, w = _plan_and_inputs(14)
    omega = torch.full_like(w, 2 * math.pi)
    phis = [(4 * math.pi * s * (xyz[2] - 0.2 * xyz[1])).contiguous() for s in (1.0, 0.5, -3.0)]
    outs = [torch.full_like(p, float("nan")) for p in phis]
    plan.demag_phi2_noalloc(phis[0], w, omega, outs[0])
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for k in (1, 2):
        plan.demag_phi2_noalloc(phis[k], w, omega, outs[k])
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
    for k in range(3):
        assert torch.isfinite(outs[k]).all()
        assert _rel(outs[k], plan.demag_phi2(phis[k], w, omega)) < 1e-6


def test_noalloc_rejects_oversized_plans():
    from paper_1605_01715_gb300 import KifmmError
    plan, xyz, w = _plan_and_inputs(296)           # 1,051,392 points > 2^20
    phi1 = xyz[2].contiguous()
    out = torch.empty_like(phi1)
    with pytest.raises(KifmmError) as e:
        plan.demag_phi2_noalloc(phi1, w, torch.full_like(w, 2 * math.pi), out)
    assert e.value.status == "INVALID_ARG"
    assert "at most" in str(e.value)
