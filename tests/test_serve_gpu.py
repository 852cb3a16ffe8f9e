"""Resumable GMRES, per-instance GMRES on forests, and the batching server on the GPU."""
import math

import numpy as np
import pytest

import synth
from oracle import bie as obie
from oracle.quadrature import quadrature_points

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"
P_ADL = 11            # the mixed form's ADL matvec meets rel-L2 1e-6 from p = 11
P_DL = 10


def t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _polar_mesh(seed, ns, contrast, f=8):
    c, r = synth.sphere_pack(ns, 0.5, 1.0, 4.0, 0.05, seed)
    m = synth.pack_mesh(c, r, f)
    eps = np.asarray(contrast, dtype=np.float64)[m.body % len(contrast)]
    return m, eps, 1.0 / m.sph[:, 3]


def _polar_case(seed=7):
    from paper_1605_01715_gb300 import kifmm_quadrature_points
    m, eps, curv = _polar_mesh(seed, 3, [3.0, 8.0, 15.0])
    xyz, w, nrm = kifmm_quadrature_points(t(m.tri.reshape(-1, 9)), t(m.sph))
    return m, xyz, w, nrm, t(eps), t(curv)


def oracle_residual(m, eps, curv, x, eps_out=1.0, e0=(0.0, 0.0, 1.0)):
    """||b - A x|| / ||b|| under the oracle's operator (Eqs. Ax, pol_discret)."""
    hx, hw, hn = quadrature_points(m.tri, m.sph)
    A = obie.polarization_operator(hx, hn, hw, eps, eps_out, curv)
    b = obie.polarization_rhs_uniform_field(hn, eps, eps_out, e0)
    return float(np.linalg.norm(b - A(x)) / np.linalg.norm(b))


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


# Three polarization instances of different contrast: their GMRES iteration counts differ.
FOREST = [(11, 2, [2.0]), (12, 3, [4.0, 9.0, 6.0]), (13, 2, [20.0, 14.0])]


def _forest():
    from paper_1605_01715_gb300 import kifmm_quadrature_points
    cases = [_polar_mesh(seed, ns, con) for seed, ns, con in FOREST]
    off = np.concatenate([[0], np.cumsum([c[0].n for c in cases])]).astype(np.int64)
    tri = np.concatenate([c[0].tri.reshape(-1, 9) for c in cases])
    sph = np.concatenate([c[0].sph for c in cases])
    xyz, w, nrm = kifmm_quadrature_points(t(tri), t(sph))
    eps = np.concatenate([c[1] for c in cases])
    curv = np.concatenate([c[2] for c in cases])
    return cases, off, xyz, w, nrm, eps, curv


def test_forest_gmres_solves_each_instance_on_its_own():
    """On a forest every instance runs its own GMRES while sharing each matvec: each
    instance's iteration count is that of its own solve on its own tree (within 2:
    the two trees' operators differ at the 1e-7 level), its residual under the
    oracle's operator meets the matvec accuracy plus the tolerance (1e-6 + 1e-7), and
    the contrasts give different counts."""
    from paper_1605_01715_gb300 import Plan, Solver, Tree, kifmm_polarization_rhs, kifmm_quadrature_points
    cases, off, xyz, w, nrm, eps, curv = _forest()
    tol = 1e-7
    tree = Tree(xyz, max_leaf=32, instances=off)
    assert tree.stats()["n_instances"] == len(cases)
    plan = Plan(tree, kernel="adl", p=P_ADL, precision="mixed", trg_nrm=nrm)
    b = kifmm_polarization_rhs(nrm, t(eps), 1.0, (0.0, 0.0, 1.0))
    sv = Solver(plan, w, t(eps), 1.0, t(curv), b, tol=tol, restart=50, max_iter=300)
    while True:
        sv.launch()
        if sv.finish():
            break
    assert sv.status == 0
    its, rrs, sts = sv.instances()
    assert (sts == 0).all() and (rrs > 0).all() and (rrs < 2 * tol).all()
    assert sv.iters == its.max()
    x = sv.x.cpu().numpy()
    for i, (m, e, c) in enumerate(cases):
        xs, ws, ns = kifmm_quadrature_points(t(m.tri.reshape(-1, 9)), t(m.sph))
        p1 = Plan(Tree(xs, max_leaf=32), kernel="adl", p=P_ADL, precision="mixed", trg_nrm=ns)
        b1 = kifmm_polarization_rhs(ns, t(e), 1.0, (0.0, 0.0, 1.0))
        x1, it1, rr1, rc1 = p1.bie_solve(ws, t(e), 1.0, t(c), b1, tol=tol, restart=50, max_iter=300)
        assert rc1 == 0
        xi = x[off[i]:off[i + 1]]
        res = oracle_residual(m, e, c, xi)
        d = float(np.linalg.norm(xi - x1.cpu().numpy()) / np.linalg.norm(xi))
        print("instance %d: n %d, forest %d its, alone %d its, oracle residual %.2e, |x - x_alone|/|x| %.2e"
              % (i, m.n, its[i], it1, res, d))
        assert abs(int(its[i]) - it1) <= 2
        assert res < 1.1e-6
    assert len(set(its.tolist())) > 1
    # the blocking solve on the forest runs the same per-instance GMRES (the mixed
    # matvec's FP32 atomics add in run-dependent order, so the iterates agree to the
    # solve's tolerance, not bit for bit)
    x2, it2, rr2, rc2 = plan.bie_solve(w, t(eps), 1.0, t(curv), b, tol=tol, restart=50, max_iter=300)
    assert rc2 == 0 and it2 == sv.iters
    assert float(torch.linalg.norm(x2 - sv.x) / torch.linalg.norm(sv.x)) < 10 * tol


def test_forest_gmres_statuses_are_per_instance():
    """Edge cases of the per-instance GMRES: an instance with b = 0 ends at x = 0
    exactly, whatever x0 was, with status OK; with max_iter between the instances'
    iteration counts the fast instances converge (OK) and the slow one does not
    (NOT_CONVERGED, which is also the solve's status)."""
    from paper_1605_01715_gb300 import Plan, Solver, Tree, kifmm_polarization_rhs
    cases, off, xyz, w, nrm, eps, curv = _forest()
    tree = Tree(xyz, max_leaf=32, instances=off)
    plan = Plan(tree, kernel="adl", p=8, precision="fp64", trg_nrm=nrm)
    b = kifmm_polarization_rhs(nrm, t(eps), 1.0, (0.0, 0.0, 1.0))
    b[off[1]:off[2]] = 0.0
    x0 = torch.ones_like(b)
    sv = Solver(plan, w, t(eps), 1.0, t(curv), b, x=x0, tol=1e-8, restart=50, max_iter=300)
    while not (sv.launch() or sv.finish()):
        pass
    its, rrs, sts = sv.instances()
    assert sv.status == 0 and (sts == 0).all()
    assert float(sv.x[off[1]:off[2]].abs().max()) == 0.0 and rrs[1] == 0.0
    assert rrs[0] < 2e-8 and rrs[2] < 2e-8
    # max_iter between the counts of the two nonzero instances
    b = kifmm_polarization_rhs(nrm, t(eps), 1.0, (0.0, 0.0, 1.0))
    sv = Solver(plan, w, t(eps), 1.0, t(curv), b, tol=1e-8, restart=50, max_iter=300)
    while not (sv.launch() or sv.finish()):
        pass
    full, _, _ = sv.instances()
    lo, hi = int(full.min()), int(full.max())
    assert hi > lo
    sv = Solver(plan, w, t(eps), 1.0, t(curv), b, tol=1e-8, restart=50, max_iter=(lo + hi) // 2)
    while not (sv.launch() or sv.finish()):
        pass
    its, rrs, sts = sv.instances()
    print("iterations alone %s; with max_iter %d: statuses %s" % (full.tolist(), (lo + hi) // 2, sts.tolist()))
    for i in range(len(cases)):
        if full[i] <= (lo + hi) // 2:
            assert sts[i] == 0 and rrs[i] < 2e-8
        else:
            assert sts[i] == -4
    assert sv.status == -4


def test_serving_batches_match_the_oracle():
    """A burst of mixed requests: the server admits them in batches (forests), and
    every answer meets the stated tolerance against the oracle, in the batch and
    alone.
    - demag: phi2 against the oracle's direct phi2 (Eq. fk_integral_discrete) at
      rel-L2 <= 1e-6, served and alone, and served against alone within 2e-6;
    - polarization: residual under the oracle's operator <= tol + 1e-6 (the GMRES
      tolerance 1e-6 plus the matvec's accuracy), served and alone.  The solutions
      themselves differ by at most cond(A) times that residual."""
    from paper_1605_01715_gb300.serve import Request, Server, _Batch
    reqs = [Request(rid=i, **d) for i, d in enumerate(synth.serve_requests(8, 2000.0, 11, lo=1500, hi=5000))]
    assert {r.kind for r in reqs} == {"polar", "demag"}
    server = Server(mem_budget=16 << 30, precision="mixed", tol=1e-6)
    recs, tot = server.run(reqs, keep_results=True)
    print("batches %d, peak batch %d, set-up %.3f s, makespan %.3f s"
          % (tot["batches"], tot["peak_batch"], tot["setup_s"], tot["makespan_s"]))
    assert len(recs) == len(reqs) and tot["peak_batch"] >= 2
    for rec in recs:
        r = reqs[rec["rid"]]
        hx, hw, hn = quadrature_points(r.tri, r.sph)
        alone = _Batch([r], torch.device(DEV), server.p[r.kind], server.max_leaf, "mixed", 1e-6, 50, 500)
        while not (alone.launch() or alone.finish()):
            pass
        xa = alone.result.cpu().numpy()
        alone.close()
        xm = rec["result"].cpu().numpy()
        if r.kind == "polar":
            assert rec["status"] == 0 and 0 < rec["rel_res"] < 1.1e-6
            res_m = oracle_residual(_mesh(r), r.eps_in, r.curv, xm)
            res_a = oracle_residual(_mesh(r), r.eps_in, r.curv, xa)
            d = float(np.linalg.norm(xm - xa) / np.linalg.norm(xa))
            print("polar n=%d batch %d: %d its, residual %.2e, oracle residual %.2e (alone %.2e), "
                  "|x - x_alone|/|x| %.2e" % (r.n, rec["batch"], rec["iters"], rec["rel_res"], res_m, res_a, d))
            assert res_m < 2e-6 and res_a < 2e-6
        else:
            phi1 = 4 * math.pi * (np.asarray(r.magnetization)[:, None] * hx).sum(0)
            ref = obie.demag_phi2(hx, hn, hw, phi1, np.full(r.n, 2 * math.pi))
            em = float(np.linalg.norm(xm - ref) / np.linalg.norm(ref))
            ea = float(np.linalg.norm(xa - ref) / np.linalg.norm(ref))
            d = float(np.linalg.norm(xm - xa) / np.linalg.norm(xa))
            print("demag n=%d batch %d: rel-L2 vs oracle %.2e (alone %.2e), served vs alone %.2e"
                  % (r.n, rec["batch"], em, ea, d))
            assert em < 1e-6 and ea < 1e-6 and d < 2e-6
        assert rec["latency"] >= 0 and rec["completed"] >= rec["admitted"] >= rec["arrival"] - 1e-9
    server.close()


def _mesh(r):
    return synth.Mesh(r.tri, r.sph, np.zeros(r.n, dtype=np.int32))
