"""Forests of independent instances (kifmm_forest_build) on the GPU.

Each instance is its own sources and targets; the forest's matvec must equal, per
instance, the FP64 oracle run on that instance alone, and no interaction list may
join two instances."""
import numpy as np
import pytest

import oracle
import synth
from oracle.quadrature import quadrature_points

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def one_triangle():
    tri = np.array([[[0.0, 0.0, 0.0], [0.1, 0.0, 0.0], [0.0, 0.1, 0.0]]])
    return synth.Mesh(tri, np.zeros((1, 4)), np.zeros(1, dtype=np.int32))


def instances():
    """Uneven instances: spheres, a cube, a small adaptive pack, a single point."""
    return [
        synth.geodesic_sphere(6, center=(5.0, 0.0, 0.0), radius=2.0),        # 720
        synth.cube_surface(5, side=3.0),                                      # 300
        synth.pack_mesh(*synth.sphere_pack(3, 0.5, 1.0, 4.0, 0.05, 2), 4),    # 960
        one_triangle(),                                                       # 1
        synth.geodesic_sphere(10, center=(-1.0, 2.0, 0.5), radius=0.3),      # 2,000
    ]


_cache = {}


def forest_case():
    if "c" in _cache:
        return _cache["c"]
    ms = instances()
    off = np.concatenate([[0], np.cumsum([m.n for m in ms])]).astype(np.int64)
    tri = np.concatenate([m.tri for m in ms])
    sph = np.concatenate([m.sph for m in ms])
    from paper_1605_01715_gb300 import kifmm_quadrature_points
    g = kifmm_quadrature_points(torch.from_numpy(np.ascontiguousarray(tri.reshape(-1, 9))).to(DEV),
                                torch.from_numpy(np.ascontiguousarray(sph)).to(DEV))
    sig = synth.uniform_density(int(off[-1]), 33)
    refs = {k: [] for k in ("sl", "dl", "adl")}
    for i, m in enumerate(ms):
        xyz, w, nrm = quadrature_points(m.tri, m.sph)
        q = sig[off[i]:off[i + 1]] * w
        for k in refs:
            refs[k].append(oracle.direct(k, xyz, xyz, q, src_nrm=nrm if k == "dl" else None,
                                         trg_nrm=nrm if k == "adl" else None))
    refs = {k: np.concatenate(v) for k, v in refs.items()}
    _cache["c"] = (off, g, sig, refs)
    return _cache["c"]


def test_forest_lists_stay_inside_instances():
    from paper_1605_01715_gb300 import Tree
    off, (xyz, w, nrm), _, _ = forest_case()
    tree = Tree(xyz, max_leaf=16, instances=off)
    st = tree.stats()
    assert st["n_instances"] == len(off) - 1 and st["forest_level"] == 1
    ex = tree.export()
    inst_of_sorted = np.searchsorted(off, ex["src_perm"], side="right") - 1
    lvl, rng = ex["level"], ex["range"]
    owner = np.full(len(lvl), -1)
    for b in range(len(lvl)):
        ids = inst_of_sorted[rng[b, 0]:rng[b, 1]]
        if lvl[b] >= st["forest_level"] and ids.size:
            assert ids.min() == ids.max(), "a box below the forest level mixes instances"
            owner[b] = ids[0]
    for which in ("U", "V", "W", "X"):
        o, idx = tree.list(which)
        for b in range(len(lvl)):
            srcs = idx[o[b]:o[b + 1]]
            if srcs.size:
                assert lvl[b] >= st["forest_level"]
                assert np.all(owner[srcs] == owner[b]), ("list %s joins instances" % which)


@pytest.mark.parametrize("kernel,prec,p,tol", [("sl", "mixed", 10, 1e-6), ("dl", "mixed", 10, 1e-6),
                                               ("adl", "mixed", 11, 1e-6), ("sl", "fp64", 12, 1e-8),
                                               ("dl", "fp64", 12, 1e-7), ("adl", "fp64", 12, 1e-7)])
def test_forest_matches_oracle_per_instance(kernel, prec, p, tol):
    from paper_1605_01715_gb300 import Plan, Tree
    off, (xyz, w, nrm), sig, refs = forest_case()
    tree = Tree(xyz, max_leaf=24, instances=off)
    plan = Plan(tree, kernel=kernel, p=p, precision=prec, src_nrm=nrm, trg_nrm=nrm)
    out = plan.matvec(torch.from_numpy(sig).to(DEV) * w).cpu().numpy()
    plan.check()
    ref = refs[kernel]
    assert out[off[3]] == 0.0                          # the single-point instance sees nothing
    for i in range(len(off) - 1):
        a, b = off[i], off[i + 1]
        if b - a > 1:
            err = np.linalg.norm(out[a:b] - ref[a:b]) / np.linalg.norm(ref[a:b])
            assert err < tol, (kernel, prec, i, err)


def test_single_instance_forest_matches_oracle():
    from paper_1605_01715_gb300 import Plan, Tree
    m = synth.geodesic_sphere(12)
    xyz, w, nrm = quadrature_points(m.tri, m.sph)
    sig = synth.uniform_density(m.n, 5)
    ref = oracle.direct("dl", xyz, xyz, sig * w, src_nrm=nrm)
    d = [torch.from_numpy(np.ascontiguousarray(a)).to(DEV) for a in (xyz, w, nrm)]
    tree = Tree(d[0], max_leaf=32, instances=[0, m.n])
    assert tree.stats()["forest_level"] == 0
    plan = Plan(tree, kernel="dl", p=10, precision="mixed", src_nrm=d[2], trg_nrm=d[2])
    out = plan.matvec(torch.from_numpy(sig).to(DEV) * d[1]).cpu().numpy()
    assert np.linalg.norm(out - ref) / np.linalg.norm(ref) < 1e-6


def test_graph_matvec_matches_direct_launches():
    """A captured matvec replays the launch sequence: the plain call's result (to the
    rounding-order spread of the FP32 atomics), re-reads q after it is refilled in
    place, and recaptures for new buffers; all against the oracle too."""
    from paper_1605_01715_gb300 import Plan, Tree
    off, (xyz, w, nrm), sig, refs = forest_case()
    tree = Tree(xyz, max_leaf=24, instances=off)
    plan = Plan(tree, kernel="sl", p=10, precision="mixed")
    q = torch.from_numpy(sig).to(DEV) * w
    ref = plan.matvec(q).clone()

    def rel(a, b):
        return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))

    oref = torch.from_numpy(refs["sl"]).to(DEV)
    out = torch.full_like(ref, float("nan"))
    plan.matvec_graph(q, out)
    torch.cuda.synchronize()
    assert rel(out, ref) < 1e-6 and rel(out, oref) < 1e-6
    q.mul_(-2.0)                                      # same buffer, new values
    plan.matvec_graph(q, out)
    torch.cuda.synchronize()
    assert rel(out, -2.0 * ref) < 1e-6 and rel(out, -2.0 * oref) < 1e-6
    out2 = torch.empty_like(ref)
    plan.matvec_graph(q, out2)                        # other buffers: captured again
    torch.cuda.synchronize()
    assert rel(out2, out) < 1e-6
    plan.check()


@pytest.mark.parametrize("kernel", ["sl", "dl", "adl"])
def test_autotune_picks_an_order_that_meets_the_target(kernel):
    """The autotuner's order, chosen without the oracle (against the FP64 form at
    p = 12), meets its target against the oracle, for every kernel: the double layers
    need higher orders than the single layer on the curved instances (ADL: p = 11)."""
    from paper_1605_01715_gb300 import Plan, Tree
    from paper_1605_01715_gb300.autotune import autotune
    off, (xyz, w, nrm), sig, refs = forest_case()
    q = torch.from_numpy(sig).to(DEV) * w
    r = autotune(xyz, q, kernel, off, nrm=nrm, target=1e-6, leaf_sizes=(16, 32), stride=1, reps=2)
    print("%s: p %d, leaf %d, estimated errors %s" % (kernel, r["p"], r["max_leaf"], r["errors"]))
    assert r["p"] in (4, 6, 8, 10, 11, 12) and r["max_leaf"] in (16, 32)
    assert r["est_err"] <= 0.7e-6 and set(r["times_ms"]) == {16, 32}
    tree = Tree(xyz, max_leaf=r["max_leaf"], instances=off)
    out = Plan(tree, kernel=kernel, p=r["p"], precision="mixed", src_nrm=nrm, trg_nrm=nrm).matvec(q).cpu().numpy()
    ref = refs[kernel]
    assert np.linalg.norm(out - ref) / np.linalg.norm(ref) < 1e-6
