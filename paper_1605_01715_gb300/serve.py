"""Serving loop: a stream of solve requests on one GPU, batched into shared launches.

Host scheduler over the C ABI (no arithmetic of the method here).  Requests arrive on
a wall clock; each is

* ``polar`` -- a dielectric polarization solve (Sec. II.C): GMRES on the ADL operator,
  one matvec per step; or
* ``demag`` -- the demagnetizing boundary potential phi2 of the Fredkin-Koehler split
  (Sec. II.B, Eq. fk_integral_discrete), one DL matvec.

Batches.  At every admission point the waiting requests of one kind (and, for
polarization, one exterior permittivity and applied field) are admitted together, as
far as the device-memory budget and the batch limits allow, into one forest
(``kifmm_forest_build``): one tree, one plan and -- for polarization -- one solver
whose instances each run their own GMRES while sharing every matvec.  Every FMM phase
of a step is then one launch for the whole batch.  A request that arrives while a
batch runs waits for the next admission point and joins a new batch; batches run
concurrently, each on its own CUDA stream: every round launches the next step of
every live batch before it waits on any.  A batch's set-up (tree, plan, evaluation
rows) runs on one of two worker threads while the live batches keep stepping: the
set-up is host work (work lists, tiles) and FP64 device work (the evaluation rows),
and two set-ups overlap one's host part with the other's device part.  A batch releases
its requests when its last instance has finished.  Latency = completion - arrival
(queueing, set-up and solve).  The operator tables are built once, at server start,
and kept by one small anchor plan per kind.

Orders.  The adjoint double layer of the polarization operator runs at p = 11 and the
double layer of the demag potential at p = 10: the lowest orders at which the mixed
form's matvec meets rel-L2 1e-6 on curved surfaces.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from .capi import Plan, Solver, Tree, kifmm_polarization_rhs, kifmm_quadrature_points

PI4 = 4.0 * math.pi
DEFAULT_P = {"polar": 11, "demag": 10}


@dataclass
class Request:
    rid: int
    arrival: float                 # seconds after the start of the run
    kind: str                      # "polar" or "demag"
    tri: np.ndarray                # (T, 3, 3) triangle vertices
    sph: np.ndarray                # (T, 4) sphere centre + radius (0 = flat facet)
    eps_in: np.ndarray | None = None   # polar: per-triangle interior permittivity
    curv: np.ndarray | None = None     # polar: per-triangle mean curvature
    eps_out: float = 1.0
    e0: tuple = (0.0, 0.0, 1.0)
    magnetization: tuple = (0.0, 0.0, 1.0)
    n: int = field(init=False)

    def __post_init__(self):
        self.n = int(self.tri.shape[0])

    def key(self):
        """Requests with equal keys can share a batch."""
        if self.kind == "polar":
            return ("polar", float(self.eps_out), tuple(float(v) for v in self.e0))
        return ("demag",)


def device_bytes(n, p, restart=50, kind="polar"):
    """Upper estimate of a request's resident device memory: per-point D2T rows,
    tree and vectors, per-box check potentials, the plan's operator tables and, for
    polarization, the Krylov basis."""
    Q = 6 * (p - 1) ** 2 + 2
    Qp = (Q + 15) // 16 * 16
    per_pt = 4 * Qp + 400 + (8 * (restart + 1) + 64 if kind == "polar" else 0)
    boxes = max(64, n // 16)
    tables = (343 + 16) * Qp * Qp * 4 * 2       # FP32 build + FP16 hi/lo during set-up
    return n * per_pt + boxes * Qp * 16 + tables


class _Batch:
    """Admitted requests of one key: their forest (or tree, for one request), plan,
    solver or demag inputs, and their stream."""

    def __init__(self, reqs, dev, p, max_leaf, precision, tol, restart, max_iter):
        t0 = time.perf_counter()
        self.reqs = reqs
        self.kind = reqs[0].kind
        sizes = [r.n for r in reqs]
        self.off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        tri = np.concatenate([r.tri.reshape(-1, 9) for r in reqs])
        sph = np.concatenate([r.sph for r in reqs])
        self.stream = torch.cuda.Stream(device=dev)
        with torch.cuda.stream(self.stream):
            tri_d = torch.from_numpy(np.ascontiguousarray(tri)).to(dev)
            sph_d = torch.from_numpy(np.ascontiguousarray(sph)).to(dev)
            xyz, w, nrm = kifmm_quadrature_points(tri_d, sph_d, stream=self.stream)
            self.stream.synchronize()
            if len(reqs) == 1:
                self.tree = Tree(xyz, max_leaf=max_leaf, stream=self.stream)
            else:
                self.tree = Tree(xyz, max_leaf=max_leaf, stream=self.stream, instances=self.off)
            if self.kind == "polar":
                r0 = reqs[0]
                self.plan = Plan(self.tree, kernel="adl", p=p, precision=precision, src_nrm=nrm, trg_nrm=nrm,
                                 stream=self.stream)
                eps = torch.from_numpy(np.concatenate([r.eps_in for r in reqs])).to(dev)
                curv = torch.from_numpy(np.concatenate([r.curv for r in reqs])).to(dev)
                b = kifmm_polarization_rhs(nrm, eps, r0.eps_out, r0.e0, stream=self.stream)
                self.stream.synchronize()
                self.solver = Solver(self.plan, w, eps, r0.eps_out, curv, b, tol=tol, restart=restart,
                                     max_iter=max_iter)
                self.result = self.solver.x
            else:
                self.plan = Plan(self.tree, kernel="dl", p=p, precision=precision, src_nrm=nrm, trg_nrm=nrm,
                                 stream=self.stream)
                # phi1 = 4 pi M.r per request: the Fredkin-Koehler interior potential of uniform M
                M = torch.from_numpy(np.repeat(np.array([r.magnetization for r in reqs], np.float64).T,
                                               sizes, axis=1)).to(dev)
                self.phi1 = PI4 * (M * xyz).sum(0)
                self.w = w
                self.omega = torch.full_like(w, 2.0 * math.pi)   # face centroids: Omega = 2 pi
                self.result = torch.empty_like(w)
                self.solver = None
        self.stream.synchronize()
        self.setup_s = time.perf_counter() - t0
        self.done = False

    def launch(self):
        if self.solver is not None:
            self.solver.launch(self.stream)
        else:
            self.plan.demag_phi2(self.phi1, self.w, self.omega, out=self.result, stream=self.stream)

    def finish(self):
        if self.solver is not None:
            self.done = self.solver.finish()
        else:
            self.stream.synchronize()
            self.done = True
        return self.done

    def outcome(self, i):
        """(iters, rel_res, status) of request i of the batch."""
        if self.solver is None:
            return 1, None, 0
        it, rr, st = self.solver.instances()
        return int(it[i]), float(rr[i]), int(st[i])

    def close(self):
        if self.solver is not None:
            self.solver.close()
        self.plan.close()
        self.tree.close()


class Server:
    """Batching server for polarization solves and demag evaluations.

    ``start()`` (called by ``run`` if needed) builds one small anchor plan per kind:
    the operator tables depend only on the kernel, order, precision and cutoffs, and a
    live plan of the same key keeps them resident, so batches never rebuild them.
    Batches are set up on a worker thread (the library's calls release the GIL), so
    the scheduler keeps stepping the live batches meanwhile."""

    def __init__(self, mem_budget=64 << 30, p=None, max_leaf=96, precision="mixed", tol=1e-6, restart=50,
                 max_iter=500, max_live=64, max_batch=64, max_batch_points=4 << 20, setup_workers=2,
                 device="cuda:0"):
        self.mem_budget = int(mem_budget)
        self.setup_workers = max(1, int(setup_workers))
        self.p = dict(DEFAULT_P)
        if isinstance(p, dict):
            self.p.update(p)
        elif p is not None:
            self.p = {"polar": int(p), "demag": int(p)}
        self.max_leaf, self.precision = max_leaf, precision
        self.tol, self.restart, self.max_iter = tol, restart, max_iter
        self.max_live, self.max_batch, self.max_batch_points = max_live, max_batch, max_batch_points
        self.dev = torch.device(device)
        self._anchors = None
        self.start_s = None

    def start(self):
        """Build the anchor plans (once); returns the seconds it took."""
        if self._anchors is not None:
            return 0.0
        t0 = time.perf_counter()
        # the 8 corners of a small cube with their diagonal normals: one leaf
        c = np.array([[x, y, z] for x in (-1.0, 1.0) for y in (-1.0, 1.0) for z in (-1.0, 1.0)]).T
        xyz = torch.from_numpy(np.ascontiguousarray(0.1 * c)).to(self.dev)
        nrm = torch.from_numpy(np.ascontiguousarray(c / math.sqrt(3.0))).to(self.dev)
        tree = Tree(xyz, max_leaf=self.max_leaf)
        plans = [Plan(tree, kernel=k, p=self.p[kind], precision=self.precision, src_nrm=nrm, trg_nrm=nrm)
                 for kind, k in (("polar", "adl"), ("demag", "dl"))]
        torch.cuda.synchronize(self.dev)
        self._anchors = (tree, plans)
        self.start_s = time.perf_counter() - t0
        return self.start_s

    def close(self):
        if self._anchors is not None:
            tree, plans = self._anchors
            for pl in plans:
                pl.close()
            tree.close()
            self._anchors = None

    def _need(self, r):
        return device_bytes(r.n, self.p[r.kind], self.restart, r.kind)

    def _take_batch(self, waiting, mem_free, first_fits):
        """Requests of the head's key, in arrival order, while the memory budget and the
        batch limits allow (the head always, if nothing else is live)."""
        key = waiting[0].key()
        group, need, pts = [], 0, 0
        for r in waiting:
            if r.key() != key:
                continue
            nr = self._need(r)
            if group and (len(group) >= self.max_batch or pts + r.n > self.max_batch_points):
                break
            if need + nr > mem_free and not (first_fits and not group):
                break
            group.append(r)
            need += nr
            pts += r.n
        return group, need

    def _new_batch(self, group):
        return _Batch(group, self.dev, self.p[group[0].kind], self.max_leaf, self.precision, self.tol,
                      self.restart, self.max_iter)

    def run(self, requests, keep_results=False):
        """Serve ``requests`` (sorted by arrival) in real time; returns per-request
        records (rid, kind, n, arrival, admitted, completed, latency, iters, rel_res,
        status, batch, setup_s) and run totals."""
        from concurrent.futures import FIRST_COMPLETED, ThreadPoolExecutor, wait

        self.start()
        reqs = sorted(requests, key=lambda r: r.arrival)
        i_next, waiting, live, pending, mem_used, out = 0, [], [], [], 0, []
        peak_live = peak_batch = rounds = n_batches = 0
        setup_total = 0.0
        pool = ThreadPoolExecutor(max_workers=self.setup_workers)
        t0 = time.perf_counter()
        try:
            while i_next < len(reqs) or waiting or live or pending:
                now = time.perf_counter() - t0
                while i_next < len(reqs) and reqs[i_next].arrival <= now:
                    waiting.append(reqs[i_next])
                    i_next += 1
                # admission: a batch of the head's key, first come first served, within
                # the budget, whenever a set-up worker is free (requests that arrive
                # while the workers are busy gather into the next batch)
                if waiting and len(pending) < self.setup_workers and len(live) + len(pending) < self.max_live:
                    group, need = self._take_batch(waiting, self.mem_budget - mem_used, not (live or pending))
                    if group:
                        ids = {id(r) for r in group}
                        waiting = [r for r in waiting if id(r) not in ids]
                        pending.append((pool.submit(self._new_batch, group), time.perf_counter() - t0, need))
                        mem_used += need
                        n_batches += 1
                        peak_batch = max(peak_batch, len(group))
                # batches whose set-up has finished join the live set
                still_pending = []
                for fut, t_adm, need in pending:
                    if fut.done():
                        bt = fut.result()
                        bt.admitted, bt.need = t_adm, need
                        setup_total += bt.setup_s
                        live.append(bt)
                    else:
                        still_pending.append((fut, t_adm, need))
                pending = still_pending
                if not live:
                    if pending:                  # wait (briefly) for a set-up to finish
                        wait([f for f, _, _ in pending], timeout=0.05, return_when=FIRST_COMPLETED)
                    elif i_next < len(reqs):
                        time.sleep(max(0.0, reqs[i_next].arrival - (time.perf_counter() - t0)))
                    continue
                peak_live = max(peak_live, len(live))
                # one round: every live batch's next step on its own stream, then the waits
                for bt in live:
                    bt.launch()
                rounds += 1
                still = []
                for bt in live:
                    if bt.finish():
                        t_done = time.perf_counter() - t0
                        for i, r in enumerate(bt.reqs):
                            iters, rel_res, status = bt.outcome(i)
                            rec = dict(rid=r.rid, kind=r.kind, n=r.n, arrival=r.arrival, admitted=bt.admitted,
                                       completed=t_done, latency=t_done - r.arrival, iters=iters, rel_res=rel_res,
                                       status=status, batch=len(bt.reqs), setup_s=bt.setup_s)
                            if keep_results:
                                rec["result"] = bt.result[int(bt.off[i]):int(bt.off[i + 1])].clone()
                            out.append(rec)
                        mem_used -= bt.need
                        bt.close()
                    else:
                        still.append(bt)
                live = still
        finally:
            pool.shutdown(wait=True)
        span = time.perf_counter() - t0
        return out, dict(makespan_s=span, rounds=rounds, peak_live=peak_live, batches=n_batches,
                         peak_batch=peak_batch, setup_s=setup_total, start_s=self.start_s)


def serial_baseline(requests, p=None, max_leaf=96, precision="fp64", tol=1e-6, restart=50, max_iter=500,
                    device="cuda:0"):
    """The same requests one at a time -- set up, solved (or evaluated) to the end and
    released before the next starts, the plain FP64 form by default, with the operator
    tables built once beforehand as for the server; returns each request's service
    time in seconds."""
    srv = Server(p=p, max_leaf=max_leaf, precision=precision, tol=tol, restart=restart, max_iter=max_iter,
                 device=device)
    srv.start()
    times = []
    try:
        for r in requests:
            t0 = time.perf_counter()
            bt = srv._new_batch([r])
            done = False
            while not done:
                bt.launch()
                done = bt.finish()
            bt.close()
            times.append(time.perf_counter() - t0)
    finally:
        srv.close()
    return times


def percentiles(lat):
    a = np.asarray(lat, dtype=float)
    return float(np.percentile(a, 50)), float(np.percentile(a, 99))
