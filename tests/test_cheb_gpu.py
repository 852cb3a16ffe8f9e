"""The Chebyshev-interpolation far field (KIFMM_ENGINE_CHEB, the paper's own FMM: Sec. I
and Sec. III.A.1, Eq. p2m) against the oracle.

Both engines approximate the same discrete sum (Sec. II.A, Eq. sum_fmm), so the oracle
is the same.  The tolerances are the interpolation's truncation error at each order n
(nodes per dimension): it must fall by at least half from n to n + 2 and stay below a
bound at n = 8 that follows from the measured decay (about 6x per two orders for the
single layer, 4-5x for the double layers, whose far field interpolates a derivative).
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import bie as obie
from oracle.quadrature import quadrature_points

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"

# error bound at n = 8, per kernel
BOUND8 = {"sl": 3e-7, "dl": 3e-5, "adl": 3e-5, "field": 3e-6}


def gpu_points(m):
    from paper_1605_01715_gb300 import kifmm_quadrature_points
    tri = torch.from_numpy(np.ascontiguousarray(m.tri.reshape(-1, 9))).to(DEV)
    sph = torch.from_numpy(np.ascontiguousarray(m.sph)).to(DEV)
    return kifmm_quadrature_points(tri, sph)


@pytest.mark.parametrize("geom", ["sphere", "pack"])
@pytest.mark.parametrize("kernel", ["sl", "dl", "adl", "field"])
def test_cheb_converges_to_the_oracle(geom, kernel):
    from paper_1605_01715_gb300 import Plan, Tree
    m = synth.geodesic_sphere(16) if geom == "sphere" else \
        synth.pack_mesh(*synth.sphere_pack(4, 0.5, 1.5, 8.0, 0.05, 1), 10)
    h = quadrature_points(m.tri, m.sph)
    xyz, w, nrm = gpu_points(m)
    sig = synth.uniform_density(m.n, 21)
    if kernel == "field":
        ref = obie.field(h[0], h[0], sig * h[1]).ravel()
    else:
        ref = oracle.direct(kernel, h[0], h[0], sig * h[1], src_nrm=h[2] if kernel == "dl" else None,
                            trg_nrm=h[2] if kernel == "adl" else None)
    tree = Tree(xyz, max_leaf=40)
    q = torch.from_numpy(sig).to(DEV) * w
    errs = {}
    for n in (4, 6, 8):
        plan = Plan(tree, kernel=kernel, p=n, precision="cheb_fp64", src_nrm=nrm, trg_nrm=nrm)
        st = plan.stats()
        assert st["q_points"] == n ** 3
        out = plan.matvec(q).cpu().numpy()
        errs[n] = float(np.linalg.norm(out - ref) / np.linalg.norm(ref))
    print("%s %s Chebyshev rel-L2 by order: %s" % (geom, kernel, errs))
    assert errs[6] < 0.5 * errs[4] and errs[8] < 0.5 * errs[6]
    assert errs[8] < BOUND8[kernel]


def test_cheb_rejects_large_orders_and_mixed_precision():
    import ctypes

    from paper_1605_01715_gb300 import KifmmError, Plan, Tree, capi
    tree = Tree(torch.rand((3, 100), dtype=torch.float64, device=DEV), max_leaf=16)
    with pytest.raises(KifmmError) as e:
        Plan(tree, kernel="sl", p=9, precision="cheb_fp64")
    assert e.value.status == "INVALID_ARG"
    h = ctypes.c_void_p()
    rc = capi.lib().kifmm_fmm_setup(tree.handle, 0, 6, capi.PRECISIONS["mixed"] | 16, 0.0, None, None, None,
                                    ctypes.byref(h))
    assert rc == -1 and not h.value
