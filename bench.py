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

    def __init__(self, index=0, interval_ms=50):
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
    plan = Plan(tree, kernel=wl["kernel"], p=p, precision=args.precision, src_nrm=nrm, trg_nrm=nrm)
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
                       "pinv_cutoff": st["pinv_cutoff"], "parallelism": "replica" if ws > 1 else "single",
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
    line["roofline"] = roofline(phases, st, tst, args)

    if args.solves > 0:
        line["solve"] = solve_latency(args, device)
        if args.precision == "mixed":
            # the configuration whose ADL matvec meets 1e-6 against the oracle (compensated
            # near field, p = 11; the plain mixed matvec above is at 3e-6 on this pack)
            line["solve_1e6"] = solve_latency(args, device, precision="mixed_cn", p=11)
    if rank == 0 and not args.no_cpu_baseline:
        idx, ref, dt, cores = oracle_sample(wl, m, q.cpu().numpy(), args.cpu_sample)
        got = out.cpu().numpy()[idx]
        line["cpu_baseline"] = {"value": idx.size / dt, "unit": "targets/s", "cores": cores, "kind": "oracle",
                                "sample": "%d seeded targets x all %d sources of their instance (FP64 direct sum)"
                      % (idx.size, n)}
        line["rel_err_sampled"] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    if ws > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_serve(args):
    """Serving stream (Poisson arrivals, mixed polarization solves and demag
    evaluations, 2k-500k unknowns): p50/p99 latency and throughput of the
    continuous-batching server at each arrival rate, against serial FP64 solves of
    the same requests.  One JSON line; value = throughput at the highest rate."""
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
            server = Server(mem_budget=args.serve_mem_gb * (1 << 30), p=args.serve_p, precision=args.precision)
            recs, tot = server.run(reqs)
            lat = [r["latency"] for r in recs]
            p50, p99 = percentiles(lat)
            polar = [r for r in recs if r["kind"] == "polar"]
            unknowns = sum(r["n"] for r in recs)
            sweep.append({"rate_req_s": rate, "requests": len(recs), "p50_ms": p50 * 1e3, "p99_ms": p99 * 1e3,
                          "throughput_req_s": len(recs) / tot["makespan_s"],
                          "unknowns_per_s": unknowns / tot["makespan_s"], "makespan_s": tot["makespan_s"],
                          "peak_live": tot["peak_live"], "rounds": tot["rounds"],
                          "polar_max_true_rel_residual": max((r["rel_res"] for r in polar), default=None),
                          "polar_failed": sum(1 for r in polar if r["status"] != 0)})
            print("serve rate %g: p50 %.1f ms p99 %.1f ms, %.1f req/s" % (rate, p50 * 1e3, p99 * 1e3,
                                                                    sweep[-1]["throughput_req_s"]),
                  file=sys.stderr, flush=True)
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
            "config": {"workload": "serve_stream", "sizes": "log-uniform 2k-500k", "p": args.serve_p,
                       "precision": args.precision, "mem_budget_gb": args.serve_mem_gb,
                       "kinds": "half polarization GMRES(50) tol 1e-6, half demag phi2"},
            "serve": sweep, "serial_fp64": serial, "clocks": clk.summary(),
            "gpu_launches": None}
    print(json.dumps(line), flush=True)
    return 0


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
        _, it, rr, rc = plan.bie_solve(w, eps, wl["eps_out"], curv, b, x=x, tol=1e-6, restart=50, max_iter=500)
        torch.cuda.synchronize()
        if k:
            times.append((time.perf_counter() - t0) * 1e3)
            iters.append(it)
            rres.append(rr)
    plan.check()
    ts = np.array(times)
    return {"workload": "polar_64", "precision": precision, "p": p, "n_unknowns": n, "tol": 1e-6, "restart": 50,
            "solves": len(times),
            "p50_ms": float(np.percentile(ts, 50)), "p99_ms": float(np.percentile(ts, 99)),
            "iterations": int(np.median(iters)), "true_rel_residual": float(max(rres)),
            "setup_ms": t_setup * 1e3, "ms_per_iteration": float(np.median(ts) / max(1, np.median(iters)))}


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


def _m2l_traffic(pairs):
    """DRAM bytes per M2L launch from the committed ncu record, if it is for this kernel source."""
    path = os.path.join(ROOT, "profiles", "m2l_tc_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except Exception:
        return None
    if rec.get("kernel_sha") != _kernel_sha():
        return None
    return rec["dram_bytes_per_pair"] * pairs + rec["dram_bytes_fixed"]


def roofline(phases, st, tst, args):
    """Roofline of the dominant kernel from algorithmic work per launch and live event times."""
    pk, src = _peaks()
    sm_max = pk.get("sm_max_mhz", 2070.0) * 1e6
    fp32_peak = 152 * 128 * 2 * sm_max / 1e12       # TFLOP/s, CUDA-core FMA at max SM clock
    fp64_peak = 1.25                                 # TFLOP/s nominal
    Q = st["q_points"]
    # an overlapped near field's phase spans the far field it runs beside, not its own
    # duration, so it does not compete for the dominant kernel (its launch-list share
    # is below M2L's)
    items = {k: v for k, v in phases.items() if k != "total" and not (k == "p2p" and st.get("near_overlap"))}
    dom = max(items, key=items.get)
    t = items[dom] * 1e-3
    mixed = args.precision != "fp64"
    if dom in ("m2l", "u2u", "l2l"):
        pairs = {"m2l": st["m2l_pairs"], "u2u": st["u2u_pairs"], "l2l": st["l2l_pairs"]}[dom]
        # algorithmic: one R x W operator per pair; R = W = Q in FP64; mixed, every
        # translation acts between projections onto the pseudo-inverses' ranges (up
        # basis: rank_up values, down basis: rank_down)
        ru, rd = (st["rank_up"], st["rank_down"]) if mixed else (Q, Q)
        R, W = {"m2l": (rd, ru), "u2u": (ru, ru), "l2l": (rd, rd)}[dom]
        flops = 2.0 * R * W * pairs
        if mixed:                                   # two-term FP16 on tcgen05: 3 MMAs per product
            peak = pk["bf16_tflops"] / 3.0
            out = {"kernel": "k_%s_tc (tcgen05, two-term FP16)" % dom, "bound": "tensor",
                   "peak_source": "%s bf16/fp16 dense burst %.0f / 3 (hi*hi + hi*lo + lo*hi)"
                                  % (src, pk["bf16_tflops"])}
        else:
            peak = fp64_peak
            out = {"kernel": "k_%s_gemm<double>" % dom, "bound": "alu", "peak_source": "FP64 nominal"}
        out.update({"achieved": flops / t / 1e12, "peak": peak, "unit": "TFLOP/s",
                    "frac": flops / t / 1e12 / peak,
                    "traffic": _m2l_traffic(pairs) if (mixed and dom == "m2l") else None,
                    "work": "2*R*W flops x %d pairs, R=%d, W=%d" % (pairs, R, W)})
        return out
    if dom == "p2p":
        flops = 20.0 * tst["p2p_pairs"]            # ~20 FP32 ops per pair (FMA counted as 2)
        peak = fp32_peak if mixed else fp64_peak
        return {"kernel": "k_p2p", "bound": "alu", "achieved": flops / t / 1e12, "peak": peak,
                "unit": "TFLOP/s", "frac": flops / t / 1e12 / peak, "traffic": None,
                "peak_source": "152 SM x 128 FP32 lanes x 2 x %.0f MHz" % (sm_max / 1e6)}
    if dom == "d2t":
        nbytes = (4 if mixed else 8) * (st["q_points"] + 8) * tst["n_src"]
        return {"kernel": "k_d2t", "bound": "hbm", "achieved": nbytes / t / 1e9, "peak": pk["hbm_gbs"],
                "unit": "GB/s", "frac": nbytes / t / 1e9 / pk["hbm_gbs"], "traffic": None, "peak_source": src}
    return {"kernel": dom, "bound": "alu", "achieved": None, "peak": None, "unit": None, "frac": None,
            "traffic": None}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="kifmm", choices=["kifmm", "reference"])
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(synth.WORKLOADS))
    ap.add_argument("--precision", default="mixed", choices=["mixed", "mixed_cn", "fp64"],
                    help="mixed_cn: mixed with the compensated DL/ADL near field")
    ap.add_argument("--p", type=int, default=0)
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
    ap.add_argument("--serve-p", type=int, default=10)
    ap.add_argument("--serve-mem-gb", type=float, default=96.0)
    ap.add_argument("--solves", type=int, default=5, help="timed polarization solves (0: skip)")
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
