"""Choice of expansion order p and leaf capacity for a batch of instances.

Host logic over the public API only (no oracle, no CPU arithmetic of the method):

* order: the smallest p among ``orders`` whose mixed-precision matvec agrees with
  an FP64 matvec at p = ``p_ref`` to ``safety * target`` (relative L2) on the tuning
  subset -- the FP64 form at p = 12 is two orders of magnitude more accurate than
  the mixed target, so the difference estimates the mixed form's own error;
* leaf capacity (the octree-height knob that balances near-field P2P against the
  far field, Sec. III.A.1 and IV.A): the capacity among ``leaf_sizes`` with the
  shortest captured-graph matvec at the chosen p.

Both are measured on a subset of the instances (every ``stride``-th) so tuning costs a
fraction of one full setup; the time per point transfers because the instances are
evaluated independently.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from .capi import Plan, Tree


def subset(instances, stride):
    """Instance indices taken for tuning and their offsets in the subset."""
    off = np.asarray(instances, dtype=np.int64)
    pick = np.arange(0, off.size - 1, max(1, int(stride)))
    sizes = off[pick + 1] - off[pick]
    return pick, np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)


def gather_subset(t, instances, pick):
    """Columns (last axis) of a device tensor belonging to the picked instances."""
    off = np.asarray(instances, dtype=np.int64)
    idx = np.concatenate([np.arange(off[i], off[i + 1]) for i in pick])
    return t[..., torch.from_numpy(idx).to(t.device)].contiguous()


def _time_graph(plan, q, out, reps):
    plan.matvec_graph(q, out)                      # capture + warm
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        plan.matvec_graph(q, out)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def autotune(xyz, q, kernel, instances, nrm=None, target=1e-6, safety=0.7,
             orders=(4, 6, 8, 10, 11, 12), leaf_sizes=(32, 48, 64, 96, 128, 192, 256), p_ref=12,
             ref_leaf=64, stride=8, reps=5, log=None):
    """Returns dict(p, max_leaf, est_err, errors, times_ms, tune_s) for the batch.

    xyz (3, n) and q (n,) are device FP64 tensors over all instances (q = density
    times weight), nrm (3, n) the normals (DL / ADL), instances the n_inst + 1 offsets.
    """
    t0 = time.perf_counter()
    pick, off = subset(instances, stride)
    sx = gather_subset(xyz, instances, pick)
    sq = gather_subset(q, instances, pick)
    sn = gather_subset(nrm, instances, pick) if nrm is not None else None

    tree = Tree(sx, max_leaf=ref_leaf, instances=off)
    ref = Plan(tree, kernel=kernel, p=p_ref, precision="fp64", src_nrm=sn, trg_nrm=sn).matvec(sq)
    ref_norm = float(torch.linalg.norm(ref))
    errors, p_best = {}, None
    for p in sorted(orders):
        out = Plan(tree, kernel=kernel, p=p, precision="mixed", src_nrm=sn, trg_nrm=sn).matvec(sq)
        errors[p] = float(torch.linalg.norm(out - ref)) / ref_norm
        if log:
            log("autotune: p=%d est. rel-L2 %.2e" % (p, errors[p]))
        if errors[p] <= safety * target:
            p_best = p
            break
    if p_best is None:                             # none meets the target: the most accurate
        p_best = min(errors, key=errors.get)
    del tree

    times = {}
    out = torch.empty_like(sq)
    for s in leaf_sizes:
        tr = Tree(sx, max_leaf=s, instances=off)
        pl = Plan(tr, kernel=kernel, p=p_best, precision="mixed", src_nrm=sn, trg_nrm=sn)
        times[s] = _time_graph(pl, sq, out, reps)
        if log:
            log("autotune: leaf %d: %.3f ms" % (s, times[s]))
        del pl, tr
    leaf = min(times, key=times.get)
    return dict(p=p_best, max_leaf=leaf, est_err=errors[p_best], errors=errors, times_ms=times,
                subset_points=int(off[-1]), subset_instances=int(pick.size),
                tune_s=time.perf_counter() - t0)
