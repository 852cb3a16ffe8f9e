"""Serving loop: a stream of solve requests on one GPU with continuous batching.

Host scheduler over the C ABI (no arithmetic of the method here).  Requests arrive on
a wall clock; each is

* ``polar`` -- a dielectric polarization solve (Sec. II.C): GMRES on the ADL operator
  (``kifmm_solver_*``), one matvec per step; or
* ``demag`` -- the demagnetizing boundary potential phi2 of the Fredkin-Koehler split
  (Sec. II.B, Eq. fk_integral_discrete), one DL matvec.

A request is admitted when the device-memory estimate of its tree, plan and Krylov
basis fits the budget; its tree, plan and solver state then stay on the device until
it completes.  Every round launches the next step of every live request, each on its
own CUDA stream, and only then waits for them, so the matvecs of all live solves
overlap on the GPU; completed requests leave and waiting ones are admitted between
rounds.  Latency = completion - arrival (queueing, set-up and solve).
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from .capi import Plan, Solver, Tree, kifmm_polarization_rhs, kifmm_quadrature_points

PI4 = 4.0 * math.pi


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


class _Live:
    """One admitted request: its device data, plan and step state."""

    def __init__(self, req, dev, p, max_leaf, precision, tol, restart, max_iter):
        self.req = req
        tri = torch.from_numpy(np.ascontiguousarray(req.tri.reshape(-1, 9))).to(dev)
        sph = torch.from_numpy(np.ascontiguousarray(req.sph)).to(dev)
        xyz, w, nrm = kifmm_quadrature_points(tri, sph)
        self.stream = torch.cuda.Stream(device=dev)
        self.tree = Tree(xyz, max_leaf=max_leaf)
        if req.kind == "polar":
            self.plan = Plan(self.tree, kernel="adl", p=p, precision=precision, src_nrm=nrm, trg_nrm=nrm)
            eps = torch.from_numpy(np.ascontiguousarray(req.eps_in)).to(dev)
            curv = torch.from_numpy(np.ascontiguousarray(req.curv)).to(dev)
            b = kifmm_polarization_rhs(nrm, eps, req.eps_out, req.e0)
            self.solver = Solver(self.plan, w, eps, req.eps_out, curv, b, tol=tol, restart=restart,
                                 max_iter=max_iter)
            self.result = self.solver.x
        else:
            self.plan = Plan(self.tree, kernel="dl", p=p, precision=precision, src_nrm=nrm, trg_nrm=nrm)
            M = req.magnetization
            # phi1 = 4 pi M.r: the Fredkin-Koehler interior potential of uniform M
            self.phi1 = PI4 * (M[0] * xyz[0] + M[1] * xyz[1] + M[2] * xyz[2])
            self.w = w
            self.omega = torch.full_like(w, 2.0 * math.pi)   # face centroids: Omega = 2 pi
            self.result = torch.empty_like(w)
            self.solver = None
        torch.cuda.synchronize()
        self.done = False
        self.iters = 0
        self.rel_res = None
        self.status = 0

    def launch(self):
        if self.solver is not None:
            self.solver.launch(self.stream)
        else:
            self.plan.demag_phi2(self.phi1, self.w, self.omega, out=self.result, stream=self.stream)

    def finish(self):
        if self.solver is not None:
            self.done = self.solver.finish()
            self.iters, self.rel_res, self.status = self.solver.iters, self.solver.rel_res, self.solver.status
        else:
            self.stream.synchronize()
            self.done = True
        return self.done

    def close(self):
        if self.solver is not None:
            self.solver.close()
        self.plan.close()
        self.tree.close()


class Server:
    """Continuous-batching server for polarization solves and demag evaluations."""

    def __init__(self, mem_budget=64 << 30, p=10, max_leaf=64, precision="mixed", tol=1e-6, restart=50,
                 max_iter=500, max_live=256, device="cuda:0"):
        self.mem_budget = int(mem_budget)
        self.p, self.max_leaf, self.precision = p, max_leaf, precision
        self.tol, self.restart, self.max_iter = tol, restart, max_iter
        self.max_live = max_live
        self.dev = torch.device(device)

    def run(self, requests, keep_results=False):
        """Serve ``requests`` (sorted by arrival) in real time; returns per-request
        records (rid, kind, n, arrival, admitted, completed, latency, iters, rel_res,
        status) and run totals."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        i_next, waiting, live, mem_used, out = 0, [], [], 0, []
        peak_live = 0
        rounds = 0
        t0 = time.perf_counter()
        while i_next < len(reqs) or waiting or live:
            now = time.perf_counter() - t0
            while i_next < len(reqs) and reqs[i_next].arrival <= now:
                waiting.append(reqs[i_next])
                i_next += 1
            # admission: first come, first served, within the memory budget
            while waiting and len(live) < self.max_live:
                r = waiting[0]
                need = device_bytes(r.n, self.p, self.restart, r.kind)
                if live and mem_used + need > self.mem_budget:
                    break
                waiting.pop(0)
                t_adm = time.perf_counter() - t0
                lv = _Live(r, self.dev, self.p, self.max_leaf, self.precision, self.tol, self.restart,
                           self.max_iter)
                lv.admitted, lv.need = t_adm, need
                mem_used += need
                live.append(lv)
            if not live:
                if i_next < len(reqs):
                    time.sleep(max(0.0, reqs[i_next].arrival - (time.perf_counter() - t0)))
                continue
            peak_live = max(peak_live, len(live))
            # one round: every live request's next step on its own stream, then the waits
            for lv in live:
                lv.launch()
            rounds += 1
            still = []
            for lv in live:
                if lv.finish():
                    t_done = time.perf_counter() - t0
                    rec = dict(rid=lv.req.rid, kind=lv.req.kind, n=lv.req.n, arrival=lv.req.arrival,
                               admitted=lv.admitted, completed=t_done, latency=t_done - lv.req.arrival,
                               iters=lv.iters, rel_res=lv.rel_res, status=lv.status)
                    if keep_results:
                        rec["result"] = lv.result.clone()
                    out.append(rec)
                    mem_used -= lv.need
                    lv.close()
                else:
                    still.append(lv)
            live = still
        span = time.perf_counter() - t0
        return out, dict(makespan_s=span, rounds=rounds, peak_live=peak_live)


def serial_baseline(requests, p=10, max_leaf=64, precision="fp64", tol=1e-6, restart=50, max_iter=500,
                    device="cuda:0"):
    """The same requests one at a time -- set up, solved (or evaluated) to the end and
    released before the next starts, the plain FP64 form by default; returns each
    request's service time in seconds."""
    dev = torch.device(device)
    times = []
    for r in requests:
        t0 = time.perf_counter()
        lv = _Live(r, dev, p, max_leaf, precision, tol, restart, max_iter)
        done = False
        while not done:
            lv.launch()
            done = lv.finish()
        lv.close()
        times.append(time.perf_counter() - t0)
    return times


def percentiles(lat):
    a = np.asarray(lat, dtype=float)
    return float(np.percentile(a, 50)), float(np.percentile(a, 99))
