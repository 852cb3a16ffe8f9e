"""Resumable GMRES and the continuous-batching serving loop on the GPU."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _polar_case(seed=7):
    from paper_1605_01715_gb300 import kifmm_quadrature_points
    c, r = synth.sphere_pack(3, 0.5, 1.0, 4.0, 0.05, seed)
    m = synth.pack_mesh(c, r, 8)
    tri = torch.from_numpy(np.ascontiguousarray(m.tri.reshape(-1, 9))).to(DEV)
    sph = torch.from_numpy(np.ascontiguousarray(m.sph)).to(DEV)
    xyz, w, nrm = kifmm_quadrature_points(tri, sph)
    eps = torch.from_numpy(np.array([3.0, 8.0, 15.0])[m.body]).to(DEV)
    curv = torch.from_numpy(1.0 / m.sph[:, 3]).to(DEV)
    return m, xyz, w, nrm, eps, curv


def test_stepwise_solver_equals_blocking_solve():
    """kifmm_solver_* runs the same GMRES as kifmm_bie_solve: same iteration count,
    same iterate to rounding, same true residual."""
    from paper_1605_01715_gb300 import Plan, Solver, Tree, kifmm_polarization_rhs
    m, xyz, w, nrm, eps, curv = _polar_case()
    tree = Tree(xyz, max_leaf=32)
    plan = Plan(tree, kernel="adl", p=8, precision="fp64", trg_nrm=nrm)
    b = kifmm_polarization_rhs(nrm, eps, 1.0, (0.0, 0.0, 1.0))
    x_ref, it_ref, rr_ref, rc = plan.bie_solve(w, eps, 1.0, curv, b, tol=1e-8, restart=10, max_iter=200)
    assert rc == 0 and rr_ref < 2e-8
    sv = Solver(plan, w, eps, 1.0, curv, b, tol=1e-8, restart=10, max_iter=200)
    steps = 0
    while True:
        sv.launch()
        steps += 1
        if sv.finish():
            break
    assert sv.status == 0 and sv.iters == it_ref
    # norm of b, one restart per cycle (one more if a restart finds convergence), the
    # Arnoldi steps, the final residual
    cycles = (it_ref + 9) // 10
    assert steps in (it_ref + 2 + cycles, it_ref + 3 + cycles)
    assert abs(sv.rel_res - rr_ref) < 1e-10
    assert float(torch.linalg.norm(sv.x - x_ref) / torch.linalg.norm(x_ref)) < 1e-10


def test_serving_loop_matches_direct_calls():
    """Every request of a small mixed stream completes; polarization answers agree with
    kifmm_bie_solve on the same plan settings, demag answers with kifmm_demag_phi2."""
    import math

    from paper_1605_01715_gb300 import Plan, Tree, kifmm_polarization_rhs, kifmm_quadrature_points
    from paper_1605_01715_gb300.serve import Request, Server
    reqs = [Request(rid=i, **d) for i, d in enumerate(synth.serve_requests(6, 200.0, 11, lo=2000, hi=9000))]
    assert {r.kind for r in reqs} == {"polar", "demag"}
    server = Server(mem_budget=8 << 30, p=8, precision="mixed", max_live=4)
    recs, tot = server.run(reqs, keep_results=True)
    assert len(recs) == len(reqs) and tot["peak_live"] >= 2
    for rec in recs:
        r = reqs[rec["rid"]]
        tri = torch.from_numpy(np.ascontiguousarray(r.tri.reshape(-1, 9))).to(DEV)
        sph = torch.from_numpy(np.ascontiguousarray(r.sph)).to(DEV)
        xyz, w, nrm = kifmm_quadrature_points(tri, sph)
        tree = Tree(xyz, max_leaf=64)
        if r.kind == "polar":
            assert rec["status"] == 0 and rec["rel_res"] < 2e-6
            plan = Plan(tree, kernel="adl", p=8, precision="mixed", trg_nrm=nrm)
            eps = torch.from_numpy(r.eps_in).to(DEV)
            curv = torch.from_numpy(r.curv).to(DEV)
            b = kifmm_polarization_rhs(nrm, eps, r.eps_out, r.e0)
            x, _, _, rc = plan.bie_solve(w, eps, r.eps_out, curv, b, tol=1e-6, restart=50, max_iter=500)
            assert rc == 0
            assert float(torch.linalg.norm(rec["result"] - x) / torch.linalg.norm(x)) < 2e-5
        else:
            plan = Plan(tree, kernel="dl", p=8, precision="mixed", src_nrm=nrm)
            phi1 = 4 * math.pi * xyz[2]
            ref = plan.demag_phi2(phi1, w, torch.full_like(w, 2 * math.pi))
            assert float(torch.linalg.norm(rec["result"] - ref) / torch.linalg.norm(ref)) < 1e-5
        assert rec["latency"] >= 0 and rec["completed"] >= rec["admitted"] >= rec["arrival"] - 1e-9
