"""GPU KIFMM through the C ABI at the stored oracle fixture (tests/golden/): the
sums at every 9th centroid of a 720-point sphere, FP64 form at p = 12 and the mixed
form (p = 10; the adjoint double layer at p = 11), against the values the oracle
wrote."""
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

sys.path.insert(0, os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden"))

import make_golden  # noqa: E402
import synth  # noqa: E402


@pytest.mark.parametrize("prec,p,tol", [("fp64", 12, 1e-7), ("mixed", 10, 1e-6)])
def test_fmm_at_golden_points(prec, p, tol):
    from paper_1605_01715_gb300 import Plan, Tree, kifmm_quadrature_points
    data = np.loadtxt(make_golden.PATH)
    idx = data[:, 0].astype(np.int64)
    m = synth.geodesic_sphere(6)
    tri = torch.from_numpy(np.ascontiguousarray(m.tri.reshape(-1, 9))).to("cuda:0")
    sph = torch.from_numpy(np.ascontiguousarray(m.sph)).to("cuda:0")
    xyz, w, nrm = kifmm_quadrature_points(tri, sph)
    q = torch.from_numpy(synth.uniform_density(m.n, 6)).to("cuda:0") * w
    tree = Tree(xyz, max_leaf=32)
    for col, k in ((1, "sl"), (2, "dl"), (3, "adl")):
        pk = p + 1 if (prec == "mixed" and k == "adl") else p
        plan = Plan(tree, kernel=k, p=pk, precision=prec, src_nrm=nrm, trg_nrm=nrm)
        out = plan.matvec(q).cpu().numpy()[idx]
        plan.check()
        ref = data[:, col]
        err = np.linalg.norm(out - ref) / np.linalg.norm(ref)
        assert err < tol, (k, prec, err)
