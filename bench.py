"""KIFMM matvec throughput (targets/s) on GB300 -- one JSON line on stdout.

Default workload: the magnetostatic demag double-layer matvec on the unit cube,
n = 296 squares per face (1,051,392 surface triangles, one quadrature point each),
density n.M with M = z-hat, targets = sources, mixed precision.

A step is one kifmm_fmm_matvec over the whole point set (gather, S2U, U2U, X, M2L,
L2L, D2T, P2P).  Tree and operators are built once before timing (the geometry is
fixed across the matvecs of an iterative solve).  `value` is device-timed with
CUDA events on the launching stream, inputs resident in HBM; `e2e` calls the C ABI
with host buffers every step (kifmm_fmm_matvec_host): q is read from pinned host
memory and the result written back to it by the matvec's first and last kernels.
The working set (D2T rows, check potentials, operators: > 1 GB) is far larger than
the 129 MB L2, so no explicit flush is done between steps.

--impl reference times the FP64 CPU oracle (direct sum) on the host cores on a
bounded sample of targets per step.  Under torchrun each rank runs an independent
replica (weak scaling); rank 0 reports.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

WORKLOAD = "demag_cube_1m"
METRIC = "KIFMM matvec targets/s at rel-err<=1e-6 vs FP64 oracle"


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """SM clock / throttle-reason samples taken while the timed region runs.

    One `nvidia-smi -lms 50` loop runs for the whole window; each line it prints is
    stamped on arrival and kept if it arrived between enter and exit."""

    QUERY = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0, interval_ms=20):
        self.index = index
        self.interval_ms = interval_ms
        self.samples = []
        self._lines = []
        self._proc = None
        self._t = None
        self._t0 = self._t1 = None

    def _reader(self):
        for ln in self._proc.stdout:
            self._lines.append((time.monotonic(), ln))

    def __enter__(self):
        try:
            self._proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY, "--format=csv,noheader,nounits",
                 "-lms", str(self.interval_ms)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._reader, daemon=True)
            self._t.start()
            t_wait = time.monotonic() + 5.0           # the loop is printing before the window opens
            while not self._lines and time.monotonic() < t_wait and self._proc.poll() is None:
                time.sleep(0.01)
        except Exception:
            self._proc = None
        self._t0 = time.monotonic()
        return self

    def __exit__(self, *a):
        self._t1 = time.monotonic()
        if self._proc is not None:
            time.sleep(self.interval_ms * 1e-3)       # the sample due at the window's end
            self._proc.terminate()
            try:
                self._proc.wait(timeout=5)
            except Exception:
                self._proc.kill()
            if self._t:
                self._t.join(timeout=5)
        for t, ln in self._lines:
            if self._t0 <= t <= self._t1 + self.interval_ms * 1e-3:
                f = [x.strip() for x in ln.strip().split(",")]
                if len(f) >= 7:
                    self.samples.append(f)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if s[3 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def make_inputs(name, device):
    """Points, weights, normals on the device (GPU quadrature) and the density."""
    import torch

    from paper_1605_01715_gb300 import kifmm_quadrature_points
    wl = synth.workload(name)
    m = wl["mesh"]
    tri = torch.from_numpy(np.ascontiguousarray(m.tri.reshape(-1, 9))).to(device)
    sph = torch.from_numpy(np.ascontiguousarray(m.sph)).to(device)
    xyz, w, nrm = kifmm_quadrature_points(tri, sph)
    if wl["kernel"] == "dl":
        M = wl["magnetization"]
        sigma = nrm[0] * M[0] + nrm[1] * M[1] + nrm[2] * M[2]
    else:
        sigma = torch.from_numpy(wl.get("density", synth.uniform_density(m.n, 1000))).to(device)
    q = (sigma * w).contiguous()
    return wl, m, xyz, w, nrm, q


def oracle_sample(wl, m, q_host, n_sample, seed=12345):
    """Time the FP64 oracle on a seeded sample of targets (the CPU baseline).  In a
    forest of instances a target sums over its own instance's sources only."""
    import oracle
    from oracle.quadrature import quadrature_points
    xyz, w, nrm = quadrature_points(m.tri, m.sph)
    idx = np.sort(np.random.default_rng(seed).choice(m.n, size=min(n_sample, m.n), replace=False))
    kern = wl["kernel"]
    off = wl.get("instances")
    if off is None:
        off = np.array([0, m.n], dtype=np.int64)
    which = np.searchsorted(off, idx, side="right") - 1
    ref = np.empty(idx.size)
    t0 = time.perf_counter()
    for i in np.unique(which):
        a, b = int(off[i]), int(off[i + 1])
        sel = which == i
        sl = slice(a, b)
        ref[sel] = oracle.direct(kern, xyz[:, sl], xyz[:, sl], q_host[sl],
                                 src_nrm=nrm[:, sl] if kern == "dl" else None,
                                 trg_nrm=nrm[:, sl] if kern == "adl" else None, idx=idx[sel] - a)
    dt = time.perf_counter() - t0
    return idx, ref, dt, oracle.max_threads()


REF_BUDGET_S = 120.0     # wall time the reference arm aims for


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    wl = synth.workload(args.workload)
    m = wl["mesh"]
    from oracle.quadrature import quadrature_points
    xyz, w, nrm = quadrature_points(m.tri, m.sph)
    if wl["kernel"] == "dl":
        M = wl["magnetization"]
        q = (nrm[0] * M[0] + nrm[1] * M[1] + nrm[2] * M[2]) * w
    else:
        q = wl.get("density", synth.uniform_density(m.n, 1000)) * w
    # per-target time of the oracle; the sample per step is sized after the first warm-up
    # step so the whole run stays within about two minutes whatever --steps is
    nstep = args.warmup + args.steps
    sample, per_target = args.ref_sample, []
    for s in range(nstep):
        _, _, dt, cores = oracle_sample(wl, m, q, sample, seed=100 + s)
        if s >= args.warmup:
            per_target.append(dt / sample)
        if s == 0:
            sample = int(max(32, min(sample, sample * REF_BUDGET_S / (dt * nstep))))
    value = 1.0 / float(np.mean(per_target))
    per_step = sample / value
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "targets/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "n_targets": m.n,
                                            "sample_targets_per_step": sample},
            "cpu_baseline": {"value": value, "unit": "targets/s", "cores": cores, "kind": "oracle",
                             "sample": "%d seeded targets x all %d sources%s per step"
                                       % (sample, m.n, " of their instance" if "instances" in wl else "")},
            "e2e": {"value": value, "unit": "targets/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_kifmm(args):
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    from paper_1605_01715_gb300 import Plan, Tree
    peaks = None if args.lean else measure_peaks(local)
    wl, m, xyz, w, nrm, q = make_inputs(args.workload, device)
    inst = wl.get("instances")
    p = args.p or wl["p"]
    max_leaf = args.max_leaf or wl["max_leaf"]
    tune = None
    if inst is not None and not args.no_autotune and not (args.p and args.max_leaf):
        from paper_1605_01715_gb300.autotune import autotune
        tune = autotune(xyz, q, wl["kernel"], inst, nrm=nrm if wl["kernel"] != "sl" else None,
                        log=lambda msg: print(msg, file=sys.stderr, flush=True))
        p, max_leaf = args.p or tune["p"], args.max_leaf or tune["max_leaf"]
    t0 = time.perf_counter()
    tree = Tree(xyz, max_leaf=max_leaf, instances=inst)
    torch.cuda.synchronize()
    t_tree = time.perf_counter() - t0
    t0 = time.perf_counter()
    cut = args.pinv_cutoff if args.pinv_cutoff > 0 else wl.get("pinv_cutoff", 0.0)
    plan = Plan(tree, kernel=wl["kernel"], p=p, precision=args.precision, src_nrm=nrm, trg_nrm=nrm,
                pinv_cutoff=cut if args.precision != "fp64" else 0.0)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    n = m.n
    out = torch.empty(n, dtype=torch.float64, device=device)
    stream = torch.cuda.current_stream()
    # every timed matvec replays the captured graph (kifmm_fmm_matvec_graph: one launch
    # on the host; the phase breakdown comes from direct launches after the timed region)
    # unless --no-graph, which launches each matvec's kernels directly
    use_graph = inst is not None or not args.no_graph
    matvec = plan.matvec_graph if use_graph else plan.matvec

    for _ in range(args.warmup):
        matvec(q, out)
    torch.cuda.synchronize()

    # device-timed region
    plan.profile(not use_graph)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            matvec(q, out)
        ev1.record(stream)
        torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    phases = plan.profile(False)
    if use_graph:                                  # phase breakdown from direct launches
        plan.profile(True)
        for _ in range(min(args.steps, 10)):
            plan.matvec(q, out)
        torch.cuda.synchronize()
        phases = plan.profile(False)
    ms = ev0.elapsed_time(ev1) / args.steps
    ms_t = torch.tensor([ms], device=device)
    if ws > 1:
        torch.distributed.all_reduce(ms_t, op=torch.distributed.ReduceOp.MAX)
    ms = float(ms_t.item())
    value = n * ws / (ms * 1e-3)

    if args.lean:                                  # the timed matvecs only (profiling runs)
        print(json.dumps({"metric": METRIC, "value": n * ws / (ms * 1e-3), "unit": "targets/s", "n_gpus": ws,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                          "config": {"workload": args.workload, "lean": True}}), flush=True)
        return 0
    # end to end through the C ABI with host buffers (kifmm_fmm_matvec_host): q and f in
    # pinned host memory, read and written in input order by the matvec's first and last
    # kernels every step (over NVLink-C2C on the Grace host), graph-replayed like the
    # device-timed steps unless --no-graph
    q_host = q.cpu().pin_memory()
    out_host = torch.empty(n, dtype=torch.float64).pin_memory()
    for _ in range(2):
        plan.matvec_host(q_host, out_host, graph=use_graph)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        plan.matvec_host(q_host, out_host, graph=use_graph)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_e2e = e0.elapsed_time(e1) / args.steps
    ms_e = torch.tensor([ms_e2e], device=device)
    if ws > 1:
        torch.distributed.all_reduce(ms_e, op=torch.distributed.ReduceOp.MAX)
    ms_e2e = float(ms_e.item())

    st = plan.stats()
    tst = tree.stats()
    line = {"metric": METRIC, "value": value, "unit": "targets/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32",
            "data": "synthetic",
            "config": {"workload": args.workload, "n_targets": n, "kernel": wl["kernel"], "p": p,
                       "q_points": st["q_points"], "max_leaf": max_leaf, "precision": args.precision,
                       "pinv_cutoff": st["pinv_cutoff"], "pinv_cutoff_up": st["pinv_cutoff_up"], "parallelism": "replica" if ws > 1 else "single",
                       "l2": "no flush: per-step working set %.2f GB > 129 MB L2" % (st["device_bytes"] / 1e9),
                       "tree": {k: tst[k] for k in ("n_boxes", "n_leaves", "n_levels", "n_v", "n_w", "n_x",
                                                     "p2p_pairs")},
                       "tree_build_ms": t_tree * 1e3, "setup_ms": t_setup * 1e3,
                       "instances": 1 if inst is None else int(len(inst) - 1), "graph": bool(use_graph)},
            "phases_ms": phases,
            "e2e": {"value": n * ws / (ms_e2e * 1e-3), "unit": "targets/s", "h2d_bytes_per_step": 8 * n,
                    "d2h_bytes_per_step": 8 * n},
            "gpu_launches": st["launches_per_matvec"] * args.steps,
            "clocks": clk.summary()}
    if tune is not None:
        line["config"]["autotune"] = {k: tune[k] for k in ("p", "max_leaf", "est_err", "subset_points",
                                                           "subset_instances", "tune_s")}
        line["config"]["autotune"]["errors"] = {str(k): v for k, v in tune["errors"].items()}
        line["config"]["autotune"]["times_ms"] = {str(k): v for k, v in tune["times_ms"].items()}
    serial = serial_phases(plan, q, out)
    line["phases_serial_ms"] = serial
    line["roofline"], line["rooflines"] = rooflines(serial, st, tst, args, wl["kernel"], peaks)
    line["peaks_measured"] = peaks
    if line["clocks"].get("sm_mhz"):
        line["clocks"]["ms_x_mhz"] = ms * line["clocks"]["sm_mhz"]
    line["clocks_long"] = long_clock_window(plan, q, out, local, use_graph)

    idx = ref = None
    if rank == 0 and not args.no_cpu_baseline:
        idx, ref, dt, cores = oracle_sample(wl, m, q.cpu().numpy(), args.cpu_sample)
        plan.matvec(q, out)
        got = out.cpu().numpy()[idx]
        line["cpu_baseline"] = {"value": idx.size / dt, "unit": "targets/s", "cores": cores, "kind": "oracle",
                                "sample": "%d seeded targets x all %d sources of their instance (FP64 direct sum)"
                      % (idx.size, n)}
        line["rel_err_sampled"] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    if rank == 0 and args.fp64_plain and inst is None:
        line["fp64_plain"] = fp64_plain(wl, tree, xyz, nrm, q, p, idx, ref, ms, peaks)
    del plan
    if args.solves > 0:
        line["solve"] = solve_latency(args, device)
    if rank == 0 and args.field_check and inst is None:
        line["demag_sphere_interior"] = demag_interior_field(device)
    if rank == 0 and ws == 1 and args.extras and inst is None:
        line["batched"] = batched_summary(device)
        line["serving"] = serving_summary(args)
    if ws > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_serve(args):
    """Serving stream (Poisson arrivals, mixed polarization solves and demag
    evaluations, 2k-500k unknowns): p50/p99 latency and throughput of the batching
    server (requests admitted together share a forest and its launches) at each
    arrival rate, against serial FP64 solves of the same requests.  One JSON line;
    value = throughput at the highest rate."""
    import torch

    from paper_1605_01715_gb300.serve import Request, Server, percentiles, serial_baseline
    device = torch.device("cuda", 0)
    torch.cuda.set_device(device)
    rates = [float(x) for x in args.serve_rates.split(",")]
    sweep = []
    n_req = args.serve_requests
    with ClockSampler(0) as clk:
        for k, rate in enumerate(rates):
            reqs = [Request(rid=i, **d) for i, d in enumerate(synth.serve_requests(n_req, rate, 5000 + k))]
            server = Server(mem_budget=args.serve_mem_gb * (1 << 30), p=args.serve_p, precision=args.precision,
                            max_batch=args.serve_max_batch, max_batch_points=args.serve_max_batch_points,
                            setup_workers=args.serve_setup_workers)
            recs, tot = server.run(reqs)
            server.close()
            lat = [r["latency"] for r in recs]
            p50, p99 = percentiles(lat)
            polar = [r for r in recs if r["kind"] == "polar"]
            unknowns = sum(r["n"] for r in recs)
            sweep.append({"rate_req_s": rate, "requests": len(recs), "p50_ms": p50 * 1e3, "p99_ms": p99 * 1e3,
                          "throughput_req_s": len(recs) / tot["makespan_s"],
                          "unknowns_per_s": unknowns / tot["makespan_s"], "makespan_s": tot["makespan_s"],
                          "peak_live": tot["peak_live"], "rounds": tot["rounds"], "batches": tot["batches"],
                          "peak_batch": tot["peak_batch"], "setup_s": tot["setup_s"],
                          "server_start_s": tot["start_s"],
                          "polar_max_true_rel_residual": max((r["rel_res"] for r in polar), default=None),
                          "polar_failed": sum(1 for r in polar if r["status"] != 0)})
            print("serve rate %g: p50 %.1f ms p99 %.1f ms, %.1f req/s" % (rate, p50 * 1e3, p99 * 1e3,
                                                                    sweep[-1]["throughput_req_s"]),
                  file=sys.stderr, flush=True)
    serial = None
    if args.serve_serial > 0:
        base_reqs = [Request(rid=i, **d) for i, d in enumerate(synth.serve_requests(args.serve_serial, 1.0, 5999))]
        st = serial_baseline(base_reqs, p=args.serve_p, precision="fp64")
        serial = {"requests": len(st), "precision": "fp64", "mean_service_ms": float(np.mean(st)) * 1e3,
                  "throughput_req_s": len(st) / float(np.sum(st)),
                  "unknowns_per_s": sum(r.n for r in base_reqs) / float(np.sum(st))}
    top = sweep[-1]
    line = {"metric": "serving throughput (solve requests/s) with p50/p99 latency", "value": top["throughput_req_s"],
            "unit": "requests/s", "n_gpus": 1, "steps": n_req, "warmup": 0,
            "ms_per_step": 1e3 / max(top["throughput_req_s"], 1e-9), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32", "data": "synthetic",
            "config": {"workload": "serve_stream", "sizes": "log-uniform 2k-500k",
                       "p": args.serve_p if args.serve_p else {"polar": 11, "demag": 10},
                       "max_batch": args.serve_max_batch, "max_batch_points": args.serve_max_batch_points,
                       "setup_workers": args.serve_setup_workers,
                       "precision": args.precision, "mem_budget_gb": args.serve_mem_gb,
                       "kinds": "half polarization GMRES(50) tol 1e-6, half demag phi2"},
            "serve": sweep, "serial_fp64": serial, "clocks": clk.summary(),
            "gpu_launches": None}
    print(json.dumps(line), flush=True)
    return 0


def long_clock_window(plan, q, out, index, use_graph, seconds=1.0):
    """SM clocks while matvecs repeat for about a second right after the timed region
    (the timed region itself may be shorter than a few sampling intervals)."""
    import torch
    mv = plan.matvec_graph if use_graph else plan.matvec
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    mv(q, out)
    torch.cuda.synchronize()
    e0.record()
    mv(q, out)
    e1.record()
    torch.cuda.synchronize()
    reps = max(10, int(seconds / max(e0.elapsed_time(e1) * 1e-3, 1e-5)))
    with ClockSampler(index) as clk:
        e0.record()
        for _ in range(reps):
            mv(q, out)
        e1.record()
        torch.cuda.synchronize()
    c = clk.summary()
    c["matvecs"] = reps
    c["ms_per_matvec"] = e0.elapsed_time(e1) / reps
    return c


def fp64_plain(wl, tree, xyz, nrm, q, p, idx, ref, ms_mixed, peaks, steps=3):
    """The plain form: the same matvec with every step in FP64 (KIFMM_PREC_FP64) at the
    same order, timed with CUDA events, with its error on the same oracle sample."""
    import torch

    from paper_1605_01715_gb300 import Plan
    t0 = time.perf_counter()
    plan = Plan(tree, kernel=wl["kernel"], p=p, precision="fp64", src_nrm=nrm, trg_nrm=nrm)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    out = torch.empty_like(q)
    plan.matvec(q, out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        plan.matvec(q, out)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    res = {"precision": "fp64", "p": p, "ms_per_matvec": ms, "targets_per_s": q.numel() / (ms * 1e-3),
           "setup_ms": t_setup * 1e3, "mixed_speedup": ms / ms_mixed, "steps": steps}
    if idx is not None:
        got = out.cpu().numpy()[idx]
        res["rel_err_sampled"] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    return res


def batched_summary(device, steps=20, n_sample=2048):
    """The batched-instance workload (batch_256: 256 sphere-pack instances, 10.9M
    points, SL) as one forest, at the order and leaf size the autotuner picks for it
    (p = 8, leaf 64; `--workload batch_256` reruns the tuning): graph-replayed matvecs
    and their sampled error against the per-instance oracle."""
    import torch

    from paper_1605_01715_gb300 import Plan, Tree
    wl, m, xyz, w, nrm, q = make_inputs("batch_256", device)
    t0 = time.perf_counter()
    tree = Tree(xyz, max_leaf=64, instances=wl["instances"])
    plan = Plan(tree, kernel="sl", p=8, precision="mixed")
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    out = torch.empty_like(q)
    plan.matvec(q, out)                              # one direct matvec: its launch count
    launches = plan.stats()["launches_per_matvec"]
    for _ in range(3):
        plan.matvec_graph(q, out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        plan.matvec_graph(q, out)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    idx, ref, _, _ = oracle_sample(wl, m, q.cpu().numpy(), n_sample)
    got = out.cpu().numpy()[idx]
    st = plan.stats()
    res = {"workload": "batch_256", "instances": int(len(wl["instances"]) - 1), "n_targets": m.n, "kernel": "sl",
           "p": 8, "max_leaf": 64, "precision": "mixed", "ms_per_matvec": ms, "targets_per_s": m.n / (ms * 1e-3),
           "setup_ms": t_setup * 1e3, "m2l_pairs": st["m2l_pairs"], "gpu_launches": launches * steps,
           "rel_err_sampled": float(np.linalg.norm(got - ref) / np.linalg.norm(ref)), "sampled_targets": int(idx.size)}
    plan.close()
    tree.close()
    return res


def serving_summary(args, rate=100.0, n_req=32, n_serial=4):
    """One point of the serving sweep (`--serve` runs the whole sweep): Poisson
    arrivals at 100 requests/s of polarization and demag requests of 2k-500k unknowns,
    served mixed with batching, against the same kind of requests served one at a
    time in the plain FP64 form."""
    from paper_1605_01715_gb300.serve import Request, Server, percentiles, serial_baseline
    reqs = [Request(rid=i, **d) for i, d in enumerate(synth.serve_requests(n_req, rate, 5001))]
    server = Server(mem_budget=96 << 30, precision="mixed")
    recs, tot = server.run(reqs)
    server.close()
    p50, p99 = percentiles([r["latency"] for r in recs])
    polar = [r for r in recs if r["kind"] == "polar"]
    base = [Request(rid=i, **d) for i, d in enumerate(synth.serve_requests(n_serial, 1.0, 5999))]
    st = serial_baseline(base, precision="fp64")
    return {"workload": "serve_stream", "rate_req_s": rate, "requests": len(recs),
            "throughput_req_s": len(recs) / tot["makespan_s"],
            "unknowns_per_s": sum(r["n"] for r in recs) / tot["makespan_s"], "p50_ms": p50 * 1e3, "p99_ms": p99 * 1e3,
            "batches": tot["batches"], "peak_batch": tot["peak_batch"], "server_start_s": tot["start_s"],
            "polar_max_true_rel_residual": max((r["rel_res"] for r in polar), default=None),
            "polar_failed": sum(1 for r in polar if r["status"] != 0),
            "serial_fp64": {"requests": len(st), "throughput_req_s": len(st) / float(np.sum(st)),
                            "mean_service_ms": float(np.mean(st)) * 1e3}}


def demag_interior_field(device, n_trg=4096):
    """The demagnetizing field inside the uniformly magnetized 1M-point sphere (M = z):
    H_z = (1/4pi) sum_j (n_j . M) w_j z.(r - r_j)/|r - r_j|^3 at seeded interior points,
    an adjoint-double-layer matvec with target normal z (Sec. IV.A's check; -1/3 exactly
    for the continuous sphere).  Mixed form at p = 11, against the oracle at every
    target and against -1/3."""
    import torch

    import oracle
    from oracle.quadrature import quadrature_points
    from paper_1605_01715_gb300 import Plan, Tree
    wl = synth.workload("demag_sphere_1m")
    m = wl["mesh"]
    _, _, xyz, w, nrm, q = make_inputs("demag_sphere_1m", device)
    rng = np.random.default_rng(2024)
    v = rng.normal(size=(3, n_trg))
    trg = v / np.linalg.norm(v, axis=0) * 0.8 * rng.uniform(0, 1, n_trg) ** (1 / 3)
    zhat = np.zeros((3, n_trg))
    zhat[2] = 1.0
    t0 = time.perf_counter()
    tree = Tree(xyz, torch.from_numpy(trg).to(device), max_leaf=wl["max_leaf"])
    plan = Plan(tree, kernel="adl", p=11, precision="mixed", trg_nrm=torch.from_numpy(zhat).to(device))
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    out = plan.matvec(q)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(5):
        plan.matvec(q, out)
    e1.record()
    torch.cuda.synchronize()
    Hz = out.cpu().numpy() / (4 * math.pi)
    hx, hw, hn = quadrature_points(m.tri, m.sph)
    t1 = time.perf_counter()
    ref = oracle.direct("adl", trg, hx, hn[2] * hw, trg_nrm=zhat) / (4 * math.pi)
    t_or = time.perf_counter() - t1
    return {"workload": "demag_sphere_1m", "n_sources": m.n, "interior_targets": n_trg, "p": 11,
            "precision": "mixed", "Hz_mean": float(Hz.mean()), "Hz_max_dev_from_minus_third":
            float(np.abs(Hz + 1.0 / 3.0).max()), "rel_err_vs_oracle": float(np.linalg.norm(Hz - ref) /
                                                                            np.linalg.norm(ref)),
            "oracle_max_dev_from_minus_third": float(np.abs(ref + 1.0 / 3.0).max()),
            "ms_per_matvec": e0.elapsed_time(e1) / 5, "setup_ms": t_setup * 1e3, "oracle_s": t_or}


# GMRES stopping tolerance of the timed solves: the configuration's relative residual
# 1e-6, less the mixed matvec's own error (about 2e-7 on the 64-sphere pack at p = 11), so
# that the residual under the exact operator -- what the oracle measures -- is within 1e-6
SOLVE_TOL = 7e-7


def solve_latency(args, device, precision=None, p=None):
    """p50/p99 wall time of full GMRES polarization solves (64-sphere pack, mixed matvec,
    FP64 Krylov) with the plan, tree and Krylov basis resident between solves."""
    import torch

    from paper_1605_01715_gb300 import Plan, Tree, kifmm_polarization_rhs
    wl, m, xyz, w, nrm, _ = make_inputs("polar_64", device)
    n = m.n
    eps = torch.from_numpy(wl["contrast"][m.body] * wl["eps_out"]).to(device)
    curv = torch.from_numpy(1.0 / m.sph[:, 3]).to(device)
    t0 = time.perf_counter()
    tree = Tree(xyz, max_leaf=wl["max_leaf"])
    precision = precision or args.precision
    p = p or wl["p"]
    plan = Plan(tree, kernel="adl", p=p, precision=precision, trg_nrm=nrm)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    b = kifmm_polarization_rhs(nrm, eps, wl["eps_out"], wl["e0"])
    x = torch.zeros(n, dtype=torch.float64, device=device)
    times, iters, rres = [], [], []
    for k in range(args.solves + 1):          # the first solve warms up
        x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, it, rr, rc = plan.bie_solve(w, eps, wl["eps_out"], curv, b, x=x, tol=SOLVE_TOL, restart=50, max_iter=500)
        torch.cuda.synchronize()
        if k:
            times.append((time.perf_counter() - t0) * 1e3)
            iters.append(it)
            rres.append(rr)
    plan.check()
    ts = np.array(times)
    res = {"workload": "polar_64", "precision": precision, "p": p, "n_unknowns": n, "tol": SOLVE_TOL, "restart": 50,
           "solves": len(times),
           "p50_ms": float(np.percentile(ts, 50)), "p99_ms": float(np.percentile(ts, 99)),
           "iterations": int(np.median(iters)), "true_rel_residual": float(max(rres)),
           "setup_ms": t_setup * 1e3, "ms_per_iteration": float(np.median(ts) / max(1, np.median(iters)))}
    if not args.no_cpu_baseline:
        res.update(solve_oracle_checks(wl, m, plan, x, b, eps, curv, w, device))
    return res


def solve_oracle_checks(wl, m, plan, x, b, eps, curv, w, device, n_sample=2048):
    """Against the FP64 oracle on a seeded sample of rows: the plan's matvec (a random
    density) and the residual of the GPU solution x, b - A x with A the oracle's
    polarization operator (Eqs. Ax, pol_discret) -- both relative on the sample."""
    import torch

    import oracle
    from oracle.quadrature import quadrature_points
    hx, hw, hn = quadrature_points(m.tri, m.sph)
    idx = np.sort(np.random.default_rng(77).choice(m.n, n_sample, replace=False))
    sig = synth.uniform_density(m.n, 31)
    mv = plan.matvec(torch.from_numpy(sig).to(device) * w).cpu().numpy()[idx]
    ref = oracle.direct("adl", hx, hx, sig * hw, trg_nrm=hn, idx=idx)
    xh, bh = x.cpu().numpy(), b.cpu().numpy()
    adl = oracle.direct("adl", hx, hx, xh * hw, trg_nrm=hn, idx=idx)
    e = eps.cpu().numpy()[idx]
    c = curv.cpu().numpy()[idx] * np.sqrt(math.pi * hw[idx])
    ebar, deps = 0.5 * (e + wl["eps_out"]), wl["eps_out"] - e
    Ax = ebar * xh[idx] + deps * (adl + c * xh[idx]) / (4 * math.pi)
    return {"matvec_rel_err_sampled": float(np.linalg.norm(mv - ref) / np.linalg.norm(ref)),
            "oracle_residual_sampled": float(np.linalg.norm(bh[idx] - Ax) / np.linalg.norm(bh[idx])),
            "oracle_sample_rows": n_sample}


def measure_peaks(index):
    """FP32 FMA (scalar and packed), rsqrt and FP64 FMA rates of this GPU, from the
    library's own microbenchmark kernels (kifmm_peak_rate), with the SM clock sampled
    while they run; also scaled to the maximum SM clock."""
    from paper_1605_01715_gb300 import kifmm_peak_rate
    rates = {}
    with ClockSampler(index) as clk:
        for unit in ("fp32_fma", "fp32x2_fma", "rsqrt", "fp64_fma"):
            rates[unit] = kifmm_peak_rate(unit, reps=3)[0]
    c = clk.summary()
    out = {"fp32_tflops": rates["fp32_fma"] / 1e12, "fp32x2_tflops": rates["fp32x2_fma"] / 1e12,
           "rsqrt_per_s": rates["rsqrt"], "fp64_tflops": rates["fp64_fma"] / 1e12,
           "sm_mhz": c["sm_mhz"], "sm_max_mhz": c["sm_max_mhz"], "clock_reasons": c["reasons"],
           "how": "kifmm_peak_rate: one instruction kind on 8 independent chains per thread, every SM, "
                  "~10 ms launches, best of 3 (CUDA events)"}
    if c["sm_mhz"] and c["sm_max_mhz"]:
        f = c["sm_max_mhz"] / c["sm_mhz"]
        out["at_max_clock"] = {"fp32_tflops": out["fp32_tflops"] * f, "rsqrt_per_s": out["rsqrt_per_s"] * f,
                               "fp64_tflops": out["fp64_tflops"] * f}
    return out


# FP32 flops per near-field pair as the kernels evaluate it (an FMA counts 2; the rsqrt
# is counted separately against the MUFU rate): single layer d (3), r^2 (5), q/r FMA (2);
# double layers also 1/r^3 (2), the exact hi products (6) and the lo cross terms (12),
# their sum (1) and the product with q (ADL, 1); field 1/r^3 q (3) and three FMAs (6)
P2P_FLOPS = {"sl": 10, "dl": 31, "adl": 32, "field": 17}


def serial_phases(plan, q, out, reps=10):
    """Per-phase device times with the near field run after the far field (each phase
    with the whole GPU), from the plan's CUDA-event profile."""
    import torch
    plan.profile(True, serial=True)
    for _ in range(reps):
        plan.matvec(q, out)
    torch.cuda.synchronize()
    return plan.profile(False)


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def _kernel_sha():
    import hashlib
    path = os.path.join(ROOT, "paper_1605_01715_gb300", "csrc", "pair_tc.cuh")
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:16]


def _m2l_traffic(pairs, ku, kd):
    """DRAM bytes per M2L launch: the operator tables (343 offsets x Kd x Ku, FP16 hi
    and lo, read once) plus the per-pair bytes of the committed ncu record, if that
    record is for this kernel source."""
    path = os.path.join(ROOT, "profiles", "m2l_tc_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except Exception:
        return None
    if rec.get("kernel_sha") != _kernel_sha():
        return None
    return rec["dram_bytes_per_pair"] * pairs + 343 * kd * ku * 2 * 2


def rooflines(phases, st, tst, args, kernel, peaks):
    """Rooflines of the three kernel families from their own (serialized) event times:
    the tensor-core translations (M2L dominant), the near field (FP32 ALU and MUFU), D2T
    (HBM).  Returns (dominant, all)."""
    pk, src = _peaks()
    Q = st["q_points"]
    mixed = args.precision != "fp64"
    out = {}
    # M2L
    t = phases["m2l"] * 1e-3
    pairs = st["m2l_pairs"]
    ru, rd = (st["rank_up"], st["rank_down"]) if mixed else (Q, Q)
    flops = 2.0 * rd * ru * pairs
    if mixed:                                       # two-term FP16 on tcgen05: 3 MMAs per product
        peak = pk["bf16_tflops"] / 3.0
        out["m2l"] = {"kernel": "k_m2l_tc (tcgen05, two-term FP16)", "bound": "tensor",
                      "peak_source": "%s bf16/fp16 dense burst %.0f / 3 (hi*hi + hi*lo + lo*hi)"
                                     % (src, pk["bf16_tflops"])}
    else:
        peak = peaks["fp64_tflops"]
        out["m2l"] = {"kernel": "k_m2l_gemm<double>", "bound": "alu",
                      "peak_source": "measured FP64 FMA rate (kifmm_peak_rate)"}
    out["m2l"].update({"achieved": flops / t / 1e12 if t > 0 else None, "peak": peak, "unit": "TFLOP/s",
                       "frac": flops / t / 1e12 / peak if t > 0 else None,
                       "traffic": _m2l_traffic(pairs, (ru + 15) // 16 * 16, (rd + 15) // 16 * 16) if mixed else None,
                       "ms": phases["m2l"],
                       "work": "2*R*W flops x %d pairs, R=%d, W=%d" % (pairs, rd, ru)})
    # near field
    t = phases["p2p"] * 1e-3
    npairs = st["near_pairs"] if mixed and st.get("near_pairs") else tst["p2p_pairs"]
    if mixed:
        fpp = P2P_FLOPS[kernel]
        peak = peaks["fp32_tflops"]
        kinds = "<%d>" % {"sl": 0, "dl": 1, "adl": 2, "field": 3}[kernel]
        if st.get("near_axis_pairs"):
            kinds += " + <4> (axis-aligned dipoles)"
        out["p2p"] = {"kernel": "k_p2p_warp%s (FP32x2)" % kinds,
                      "bound": "alu", "achieved": fpp * npairs / t / 1e12, "peak": peak, "unit": "TFLOP/s",
                      "frac": fpp * npairs / t / 1e12 / peak, "traffic": None, "ms": phases["p2p"],
                      "pairs": npairs, "axis_pairs": st.get("near_axis_pairs", 0), "flops_per_pair": fpp,
                      "pairs_per_s": npairs / t,
                      "mufu_frac": npairs / t / peaks["rsqrt_per_s"],
                      "peak_source": "measured FP32 FMA rate (kifmm_peak_rate) at %.0f MHz" % (peaks["sm_mhz"] or 0)}
    else:
        out["p2p"] = {"kernel": "k_p2p<double>", "bound": "alu", "ms": phases["p2p"], "pairs": npairs,
                      "achieved": 20.0 * npairs / t / 1e12, "peak": peaks["fp64_tflops"], "unit": "TFLOP/s",
                      "frac": 20.0 * npairs / t / 1e12 / peaks["fp64_tflops"], "traffic": None,
                      "peak_source": "measured FP64 FMA rate (kifmm_peak_rate)"}
    # D2T: rows (Kd FP32, or Qp FP64) streamed once per target and component
    t = phases["d2t"] * 1e-3
    K = (rd + 15) // 16 * 16 if mixed else (Q + 15) // 16 * 16
    nbytes = (4 if mixed else 8) * (K + 1) * tst["n_trg"] * (3 if kernel == "field" else 1)
    out["d2t"] = {"kernel": "k_d2t", "bound": "hbm", "achieved": nbytes / t / 1e9, "peak": pk["hbm_gbs"],
                  "unit": "GB/s", "frac": nbytes / t / 1e9 / pk["hbm_gbs"], "traffic": None, "ms": phases["d2t"],
                  "peak_source": src, "work": "%d B of rows + 4 B result per target" % ((4 if mixed else 8) * K)}
    dom = max(("m2l", "p2p", "d2t"), key=lambda k: out[k]["ms"])
    return dict(out[dom]), out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="kifmm", choices=["kifmm", "reference"])
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(synth.WORKLOADS))
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--p", type=int, default=0)
    ap.add_argument("--pinv-cutoff", type=float, default=0.0,
                    help="pseudo-inverse truncation (0: the workload's, else the library default)")
    ap.add_argument("--max-leaf", type=int, default=0)
    ap.add_argument("--cpu-sample", type=int, default=8192)
    ap.add_argument("--ref-sample", type=int, default=2048)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="batch workloads: take p / leaf from the workload")
    ap.add_argument("--graph", action="store_true", help="(the default) time captured-graph matvecs")
    ap.add_argument("--no-graph", action="store_true",
                    help="single instance: launch each matvec's kernels directly (batches always replay a graph)")
    ap.add_argument("--serve", action="store_true", help="serving-stream sweep instead of the matvec bench")
    ap.add_argument("--serve-rates", default="10,100,1000")
    ap.add_argument("--serve-requests", type=int, default=48)
    ap.add_argument("--serve-serial", type=int, default=8)
    ap.add_argument("--serve-p", type=int, default=None,
                    help="one order for both kinds (default: ADL p = 11, DL p = 10)")
    ap.add_argument("--serve-max-batch", type=int, default=64, help="requests per batch (1: no shared launches)")
    ap.add_argument("--serve-max-batch-points", type=int, default=4 << 20, help="unknowns per batch")
    ap.add_argument("--serve-setup-workers", type=int, default=2, help="threads setting batches up")
    ap.add_argument("--serve-mem-gb", type=float, default=96.0)
    ap.add_argument("--solves", type=int, default=5, help="timed polarization solves (0: skip)")
    ap.add_argument("--no-fp64-plain", dest="fp64_plain", action="store_false",
                    help="skip timing the FP64 plain form of the same matvec")
    ap.add_argument("--no-field-check", dest="field_check", action="store_false",
                    help="skip the interior demagnetizing field of the 1M sphere")
    ap.add_argument("--no-extras", dest="extras", action="store_false",
                    help="skip the batched-instance and serving summaries of the default run")
    ap.add_argument("--lean", action="store_true",
                    help="set-up, warm-up and the timed matvecs only, then a short line (for profiler runs)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.serve:
        return run_serve(args)
    return run_kifmm(args)


if __name__ == "__main__":
    sys.exit(main())
