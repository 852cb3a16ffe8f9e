"""Octree and interaction lists built on the GPU vs their geometric definitions.

The lists of the adaptive KIFMM (Ying, Biros & Zorin 2004) are recomputed here by
brute force over all boxes from the exported tree, and every (target leaf, source
leaf) pair must be covered by exactly one interaction (near or far).
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DEPTH = 20


def _geom(t):
    lvl = t["level"].astype(np.int64)
    sh = DEPTH - lvl
    lo = t["coord"].astype(np.int64) << sh[:, None]
    hi = (t["coord"].astype(np.int64) + 1) << sh[:, None]
    return lvl, lo, hi


def _adj(lo, hi, a, b):
    return bool(np.all(lo[a] <= hi[b]) and np.all(lo[b] <= hi[a]))


def _contains(lo, hi, outer, inner):
    return bool(np.all(lo[outer] <= lo[inner]) and np.all(hi[inner] <= hi[outer]))


def brute_lists(t):
    lvl, lo, hi = _geom(t)
    nb = lvl.size
    leaf = t["leaf"]
    rng = t["range"]
    has_s = rng[:, 1] > rng[:, 0]
    has_t = rng[:, 3] > rng[:, 2]
    par = np.where(t["parent"] >= 0, t["parent"], 0)
    nlev = int(lvl.max()) + 1
    anc_at = np.zeros((nlev, nb), np.int64)      # anc_at[l][b]: ancestor of b at level min(l, lvl[b])
    for l in range(nlev):
        a = np.arange(nb)
        for _ in range(nlev):
            a = np.where(lvl[a] > l, par[a], a)
        anc_at[l] = a

    def adj_vec(ia, b):
        return np.all(lo[ia] <= hi[b], axis=-1) & np.all(lo[b] <= hi[ia], axis=-1)

    def adj_pair(ia, ib):
        return np.all(lo[ia] <= hi[ib], axis=-1) & np.all(lo[ib] <= hi[ia], axis=-1)

    allA = np.arange(nb)
    U, V, W, X = ([set() for _ in range(nb)] for _ in range(4))
    for B in range(nb):
        if not has_t[B]:
            continue
        adj = adj_vec(allA, B)
        if leaf[B]:
            U[B] = set(np.nonzero(leaf & has_s & adj)[0].tolist())
            m = has_s & (lvl > lvl[B]) & ~adj & adj_vec(par, B) & adj_vec(anc_at[lvl[B]], B)
            W[B] = set(np.nonzero(m)[0].tolist())
        if lvl[B] >= 2:
            m = has_s & (lvl == lvl[B]) & ~adj & adj_vec(par, par[B])
            V[B] = set(np.nonzero(m)[0].tolist())
        if lvl[B] >= 1:
            ancB = anc_at[np.minimum(lvl, nlev - 1), B]          # B's ancestor at each A's level
            m = leaf & has_s & (lvl < lvl[B]) & ~adj & adj_vec(allA, par[B]) & adj_pair(allA, ancB)
            X[B] = set(np.nonzero(m)[0].tolist())
    return U, V, W, X


def _lists(tree):
    out = {}
    for k in "UVWX":
        off, idx = tree.list(k)
        out[k] = [set(idx[off[b]:off[b + 1]].tolist()) for b in range(off.size - 1)]
        # no duplicates within a list
        assert sum(len(s) for s in out[k]) == idx.size
    return out


def _check_tree(xyz_s, xyz_t, tree, max_leaf):
    t = tree.export()
    st = tree.stats()
    lvl, lo, hi = _geom(t)
    rng = t["range"]
    nb = lvl.size
    ns, nt = st["n_src"], st["n_trg"]
    # permutations are permutations
    assert np.array_equal(np.sort(t["src_perm"]), np.arange(ns))
    assert np.array_equal(np.sort(t["trg_perm"]), np.arange(nt))
    # leaves partition sources and targets; non-leaves obey the capacity rule
    for col, n in ((0, ns), (2, nt)):
        cover = np.zeros(n, np.int64)
        for b in np.nonzero(t["leaf"])[0]:
            cover[rng[b, col]:rng[b, col + 1]] += 1
        assert np.all(cover == 1)
    for b in range(nb):
        cnt = max(rng[b, 1] - rng[b, 0], rng[b, 3] - rng[b, 2])
        if not t["leaf"][b]:
            assert cnt > max_leaf
        elif lvl[b] < DEPTH:
            assert cnt <= max_leaf
        if b > 0:
            p = t["parent"][b]
            assert lvl[p] == lvl[b] - 1 and _contains(lo, hi, p, b)
            assert rng[p, 0] <= rng[b, 0] <= rng[b, 1] <= rng[p, 1]
    # sorted points lie in their leaves
    c = np.array(st["root_center"])
    h = st["root_half"]
    for xyz, perm, col in ((xyz_s, t["src_perm"], 0), (xyz_t, t["trg_perm"], 2)):
        P = xyz[:, perm]
        cell = np.floor((P - (c - h)[:, None]) / (2 * h) * (1 << DEPTH)).astype(np.int64)
        for b in np.nonzero(t["leaf"])[0]:
            seg = cell[:, rng[b, col]:rng[b, col + 1]]
            assert np.all(seg >= lo[b][:, None] - 1) and np.all(seg <= hi[b][:, None])
    # lists equal their definitions
    got = _lists(tree)
    U, V, W, X = brute_lists(t)
    for k, ref in zip("UVWX", (U, V, W, X)):
        for b in range(nb):
            assert got[k][b] == ref[b], (k, b, sorted(got[k][b] ^ ref[b]))
    # every (target leaf, source leaf) pair interacts exactly once
    leaves = np.nonzero(t["leaf"])[0]
    src_leaves = np.array([a for a in leaves if rng[a, 1] > rng[a, 0]])
    # contains[D, k]: box D is src_leaves[k] or one of its ancestors
    contains = np.all(lo[:, None, :] <= lo[None, src_leaves, :], axis=2) & \
        np.all(hi[None, src_leaves, :] <= hi[:, None, :], axis=2)
    pos = {int(a): k for k, a in enumerate(src_leaves)}
    for B in leaves:
        if rng[B, 3] <= rng[B, 2]:
            continue
        n = np.zeros(src_leaves.size, np.int64)
        for A in got["U"][B]:
            n[pos[A]] += 1
        for D in got["W"][B]:
            n += contains[D]
        Bp = B
        while Bp >= 0:
            for D in got["V"][Bp]:
                n += contains[D]
            for A in got["X"][Bp]:
                n[pos[A]] += 1
            Bp = t["parent"][Bp]
        assert np.all(n == 1), (B, src_leaves[n != 1], n[n != 1])
    return st


def _points(kind, seed):
    rng = np.random.default_rng(seed)
    if kind == "sphere":
        from oracle.quadrature import quadrature_points
        m = synth.geodesic_sphere(9)
        return quadrature_points(m.tri, m.sph)[0]
    if kind == "pack":
        from oracle.quadrature import quadrature_points
        c, r = synth.sphere_pack(3, 0.3, 1.2, 5.0, 0.05, seed)
        m = synth.pack_mesh(c, r, 6)
        return quadrature_points(m.tri, m.sph)[0]
    if kind == "cluster":  # strongly non-uniform: forces W and X lists
        a = rng.normal(scale=0.02, size=(3, 900)) + 0.3
        b = rng.uniform(-1, 1, size=(3, 700))
        return np.concatenate([a, b], axis=1)
    raise ValueError(kind)


@pytest.mark.parametrize("kind,max_leaf", [("sphere", 16), ("pack", 24), ("cluster", 20), ("cluster", 1)])
def test_lists_match_definitions(kind, max_leaf):
    from paper_1605_01715_gb300 import Tree
    xyz = _points(kind, 5)
    tree = Tree(torch.from_numpy(xyz).cuda(), max_leaf=max_leaf)
    st = _check_tree(xyz, xyz, tree, max_leaf)
    if kind == "cluster" and max_leaf > 1:
        assert st["n_w"] > 0 and st["n_x"] > 0


def test_target_source_model_lists():
    """Separate targets and sources in one tree (Sec. III.A.1, target-source model)."""
    from paper_1605_01715_gb300 import Tree
    rng = np.random.default_rng(3)
    src = _points("cluster", 6)
    trg = rng.uniform(-0.5, 1.0, size=(3, 800))
    tree = Tree(torch.from_numpy(src).cuda(), torch.from_numpy(trg).cuda(), max_leaf=24)
    _check_tree(src, trg, tree, 24)


def test_degenerate_trees():
    from paper_1605_01715_gb300 import Tree
    # one point
    one = np.array([[0.5], [0.25], [-1.0]])
    st = Tree(torch.from_numpy(one).cuda(), max_leaf=8).stats()
    assert st["n_boxes"] == 1 and st["n_leaves"] == 1
    # coincident points cannot be separated: the tree stops at the maximum depth
    same = np.ones((3, 50))
    tr = Tree(torch.from_numpy(same).cuda(), max_leaf=8)
    st = tr.stats()
    assert st["n_levels"] == DEPTH + 1
    t = tr.export()
    assert t["leaf"][-1] and t["range"][-1, 1] - t["range"][-1, 0] == 50
