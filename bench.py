#!/usr/bin/env python
"""Benchmark of the FP64 free-mesh transform hot path on GB300.

One step = one pass of the whole hot path on one synthetic problem whose
inputs are already resident in HBM: oct_build (tau, Morton codes, sort,
gather, root), fit_level / refine for every level, then evaluate at the
targets.  Workload (default): 1e6 points (half uniform, half in 8 Gaussian
clusters), 3-D Franke values, p = 8 (165 monomials), max depth 7, min 128
points, tol 1e-8 relative, 1e7 uniform targets.

Printed (rank 0, one JSON line): value = fitted points/s (the fit phase of
the step, CUDA events on the launching stream), evals_per_s, the roofline of
the dominant kernel (tile_qr, FP64 pipe), an end-to-end figure through host
buffers, the CPU oracle baseline, clocks sampled during the timed region, and
the kernel launch count.

Multi-GPU: the path does not shard one problem; every rank fits its own
replica (weak scaling) and value sums the ranks' points over the slowest
rank's time.  --impl reference times the FP64 CPU oracle instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fitted pts/s & evals/s, mixed vs FP64 at stated err; p50/p99 req latency"
UNIT = "fitted pts/s"
FP64_NOMINAL_TFLOPS = 1.25  # GB300 FP64 (non-tensor) nominal rate
# DRAM bytes (read + write) per row of k_tile_qr, from one ncu capture of the
# current kernel on the 3e5-point recipe (profiles/tile_qr_3e5pts_p8.md):
# 14.86 MB read + 51.45 MB written for 3e5 rows.  Scaled to a full launch by
# its rows; set to None whenever the kernel changes until it is re-captured.
TILE_QR_DRAM_BYTES_PER_ROW = (15.191296e6 + 48.828416e6) / 3.0e5


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["fmt", "reference"], default="fmt")
    ap.add_argument("--workload", choices=["scale", "small", "batch", "serve", "fig1", "sweep"], default="scale")
    ap.add_argument("--requests", type=int, default=48, help="serve: requests in the arrival stream")
    ap.add_argument("--rate", type=float, default=200.0, help="serve: mean arrivals per second")
    ap.add_argument("--slots", type=int, default=2, help="serve: worker slots (streams)")
    ap.add_argument("--problems", type=int, default=4096, help="problems of the batch workload")
    ap.add_argument("--points", type=int, default=0, help="override the number of points")
    ap.add_argument("--targets", type=int, default=0, help="override the number of targets")
    ap.add_argument("--cpu-points", type=int, default=200_000, help="oracle sample size for cpu_baseline")
    ap.add_argument("--cpu-points-serial", type=int, default=50_000,
                    help="oracle sample for cpu_baseline.single_core (0 = skip)")
    ap.add_argument("--ref-points", type=int, default=40_000, help="oracle sample per step for --impl reference")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--profile-only", action="store_true", help="run warmup+steps, print nothing (for ncu)")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64",
                    help="path of the headline value; the other path is reported in the 'mixed' / 'fp64' block")
    ap.add_argument("--no-second-path", action="store_true", help="skip the block of the other precision")
    ap.add_argument("--sweeps", type=int, default=0, help="mixed path: FP64 refinement sweeps (0 = library default)")
    ap.add_argument("--graph", action="store_true", help="capture each fit_level in a CUDA graph (FMT_OPT_GRAPH)")
    ap.add_argument("--autotune", action="store_true",
                    help="time QR launch configurations (fmt_autotune) for the workload's degrees before the run")
    ap.add_argument("--sweep-max-exp", type=int, default=7,
                    help="sweep: largest N = 8^E (E <= 9; degree 12 runs up to 8^7)")
    ap.add_argument("--sweep-min-exp", type=int, default=4, help="sweep: smallest N = 8^E (E >= 4)")
    ap.add_argument("--sweep-tols", default="1e-6,1e-8,1e-10,1e-12", help="sweep: comma-separated tol_rel values")
    ap.add_argument("--blocks", default="c3,batch,serve",
                    help="scale workload: extra blocks of the line (comma-separated: c3 = the precision form of "
                         "the small workload against the oracle, batch = the 4096-problem form in FP64 and mixed, "
                         "serve = the Poisson request stream); 'none' for none")
    return ap.parse_args()


def make_workload(args, rank=0):
    from paper_1511_01353_gb300 import workloads as W
    if args.workload == "batch":
        return W.batch(n_problems=args.problems, seed=W.SEED_BASE + 3 + 1000 * rank)
    if args.workload == "small":
        kw = {}
        if args.points:
            kw["n"] = args.points
        if args.targets:
            kw["n_targets"] = args.targets
        return W.small(**kw)
    kw = dict(seed=W.SEED_BASE + 1 + 1000 * rank)
    if args.points:
        kw["n"] = args.points
    if args.targets:
        kw["n_targets"] = args.targets
    return W.scale(**kw)


class ClockSampler:
    """nvidia-smi samples (every 200 ms) of SM clock and throttle reasons."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", self.gpu_id, "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
                pw.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None, "reasons": sorted(reasons), "samples": len(sm)}


def _morton_np(x, y, z, lo, side):
    import numpy as np

    def spread(v):
        out = np.zeros_like(v)
        for b in range(21):
            out |= ((v >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b)
        return out

    qs = []
    for a, arr in enumerate((x, y, z)):
        t = (np.asarray(arr, np.float64) - lo[a]) * (2097152.0 / side)
        q = np.where(t >= 2097152.0, 2097151.0, np.floor(np.where(t >= 0, t, 0.0)))
        qs.append(spread(q.astype(np.uint64)))
    return qs[0] | (qs[1] << np.uint64(1)) | (qs[2] << np.uint64(2))


def levels_visited(ex, xq, yq, zq, lo, side):
    """Sum over targets of the number of tree levels evaluate visits (for flops)."""
    import numpy as np
    code = _morton_np(xq, yq, zq, lo, side)
    alive = np.ones(code.shape[0], bool)
    total = 0
    off = 0
    for d, k in enumerate(ex.header["level_nodes"]):
        if k == 0:
            break
        pref = np.sort(ex.prefix[off:off + k])
        off += k
        P = code >> np.uint64(3 * (21 - d)) if d > 0 else np.zeros_like(code)
        idx = np.searchsorted(pref, P)
        hit = (idx < k) & (pref[np.minimum(idx, k - 1)] == P)
        alive &= hit
        total += int(alive.sum())
    return total


def reduce_max(values, dist=None, device="cpu"):
    """Max over ranks of a list of floats (the slowest rank's times); the
    identity when torch.distributed is not initialised or has one rank."""
    if dist is None or not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def job_throughput(world, units_per_rank, seconds_max):
    """Whole-job rate: every rank processed units_per_rank in at most seconds_max."""
    return world * units_per_rank / seconds_max


def run_reference(args, rank, world):
    """The FP64 CPU oracle as it stands, timed on this host's cores."""
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_1511_01353_gb300 import workloads as W
    n = args.ref_points
    w = W.scale(n=n, n_targets=n) if args.workload == "scale" else W.small()
    n = w.n
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        T = O.fit(w.x, w.y, w.z, w.f, w.degree, w.max_depth, w.min_pts, w.tol_rel, mode="omp")
        t1 = time.perf_counter()
        if i >= args.warmup:
            times.append(t1 - t0)
        del T
    t = sum(times) / len(times)
    value = n / t
    cores = O.num_threads()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "sample_points": n, "degree": w.degree, "max_depth": w.max_depth,
                       "min_pts": w.min_pts, "tol_rel": w.tol_rel},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d points of the same recipe per step, fit only, OpenMP over sibling "
                                       "subtrees" % n},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline_batch(args, w):
    """The oracle on the first problems of the batch, one after another (each
    with OpenMP over its sibling subtrees), until ~10 s of work."""
    from oracle import oracle as O
    t0 = time.perf_counter()
    pts = 0
    k = 0
    while k < w.n_problems and time.perf_counter() - t0 < 10.0:
        a, b = int(w.offsets[k]), int(w.offsets[k + 1])
        O.fit(w.x[a:b], w.y[a:b], w.z[a:b], w.f[a:b], int(w.degrees[k]), w.max_depth, w.min_pts, w.tol_rel,
              mode="omp")
        pts += b - a
        k += 1
    dt = time.perf_counter() - t0
    out = {"value": pts / dt, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
           "sample": "first %d problems of the batch (%d points), fitted one after another, %.1f s" % (k, pts, dt)}
    if args.cpu_points_serial > 0:
        # the same problems on one thread (depth-first as printed), up to the serial sample size
        t0 = time.perf_counter()
        ps, j = 0, 0
        while j < k and ps < args.cpu_points_serial:
            a, b = int(w.offsets[j]), int(w.offsets[j + 1])
            O.fit(w.x[a:b], w.y[a:b], w.z[a:b], w.f[a:b], int(w.degrees[j]), w.max_depth, w.min_pts, w.tol_rel,
                  mode="dfs")
            ps += b - a
            j += 1
        ds = time.perf_counter() - t0
        out["single_core"] = {"value": ps / ds, "unit": UNIT, "cores": 1, "kind": "oracle",
                              "sample": "first %d problems (%d points), depth-first on one thread, %.1f s"
                                        % (j, ps, ds)}
    return out


def cpu_baseline(args):
    from oracle import oracle as O
    from paper_1511_01353_gb300 import workloads as W
    n = args.cpu_points
    w = W.scale(n=n, n_targets=n) if args.workload == "scale" else W.small()
    t0 = time.perf_counter()
    T = O.fit(w.x, w.y, w.z, w.f, w.degree, w.max_depth, w.min_pts, w.tol_rel, mode="omp")
    t1 = time.perf_counter()
    T.evaluate(w.xq, w.yq, w.zq)
    t2 = time.perf_counter()
    out = {"value": w.n / (t1 - t0), "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
           "sample": "%s: %d points (same recipe, p, depth, min_pts, tol), fit %.2f s; OpenMP over sibling "
                     "subtrees, each node serial" % (w.name, w.n, t1 - t0),
           "evals_per_s": w.m / (t2 - t1)}
    ns = args.cpu_points_serial
    if ns > 0:
        # the same oracle on one core: Alg. 1's depth-first recursion as printed
        ws = W.scale(n=ns, n_targets=1) if args.workload == "scale" else W.small()
        t0 = time.perf_counter()
        O.fit(ws.x, ws.y, ws.z, ws.f, ws.degree, ws.max_depth, ws.min_pts, ws.tol_rel, mode="dfs")
        dt = time.perf_counter() - t0
        out["single_core"] = {"value": ws.n / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                              "sample": "%s: %d points, depth-first on one thread, fit %.2f s" % (ws.name, ws.n, dt)}
    return out


def run_experiments(args, rank, world):
    """The paper's experiments on the GPU path (FP64).  fig1: the unscoped fit
    (a single node, max_depth 0) of 8^6 random points at p = 6, 10, 14 (Fig. 1,
    Sec. 3).  sweep: tau x N x p (Figs. 2-4, Sec. 4): N_p = N_q = 8^4 .. 8^E
    random points and targets, error against the Franke function (Eq. eqF1)
    at the targets and the number of octree nodes.  The paper prints no
    numbers for these figures; this is a report."""
    import numpy as np
    import torch
    from paper_1511_01353_gb300 import fmt as F
    from paper_1511_01353_gb300 import workloads as W

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    F.load()
    seed = W.SEED_BASE + 5

    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(a)).cuda()

    def cloud(n, stream):
        x, y, z = W.uniform_points(seed, stream, n)
        return [dev(a) for a in (x, y, z, W.franke_paper(x, y, z))]

    prec = F.FMT_MIXED if args.precision == "mixed" else F.FMT_FP64

    def run(pts, tgt, p, D, tol, warm):
        n = pts[0].shape[0]
        prm = F.make_params(p, D, 0, tol, precision=prec, sweeps=args.sweeps)
        if warm:
            F.fit(prm, *pts[:4]).close()
        torch.cuda.synchronize()
        F.fmt_profile_enable(True)
        t0 = time.perf_counter()
        tree = F.fit(prm, *pts[:4])
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        prof = F.fmt_profile_read()
        F.fmt_profile_enable(False)
        kms = {k: round(v["ms"], 3) for k, v in prof.items() if v["launches"] and k != "graph_launch"}
        out = torch.empty(tgt[0].shape[0], dtype=torch.float64, device="cuda")
        F.evaluate(tree, *tgt[:3], out)
        torch.cuda.synchronize()
        st = F.fmt_tree_stats(tree)
        nodes = int(sum(st.nodes[d] for d in range(st.n_levels)))
        depth = st.n_levels - 1
        fl = F.parse_export(F.fmt_tree_export(tree)).flags
        tiers = {"tensor": int(np.sum(((fl & F.FMT_FLAG_MIXED) != 0) & ((fl & F.FMT_FLAG_MIXED_FP64) == 0))),
                 "fp64_normal_eq": int(np.sum((fl & F.FMT_FLAG_MIXED_FP64) != 0)),
                 "householder": int(np.sum((fl & F.FMT_FLAG_MIXED) == 0))}
        tree.close()
        erms, einf = W.errors(out.cpu().numpy(), tgt[3].cpu().numpy())
        return {"N": n, "N_q": int(tgt[0].shape[0]), "p": p, "nmono": F.fmt_nmono(p), "max_depth": D,
                "tol_rel": tol, "nodes": nodes, "depth": depth, "E_rms": erms, "E_inf": einf,
                "fit_ms": t * 1e3, "fitted_pts_per_s": n / t, "nodes_by_tier": tiers, "kernel_ms": kms}

    rows = []
    if args.workload == "fig1":
        pts = cloud(8 ** 6, 1 + 8 ** 6)
        tgt = cloud(100_000, 9)
        for p in (6, 10, 14):
            rows.append(run(pts, tgt, p, 0, 0.0, True))
        metric = "unscoped fit (Fig. 1): E_rms, E_inf vs p"
        targets = 100_000
    else:
        emax = max(4, min(9, args.sweep_max_exp))
        for e in range(max(4, args.sweep_min_exp), emax + 1):
            n = 8 ** e
            pts = cloud(n, 1 + n)
            tgt = cloud(n, 9)
            for p in (4, 8, 12):
                if p == 12 and e > 7:
                    continue  # about 100 s per fit at 8^8 on the FP64 path
                for k, tol in enumerate(float(v) for v in args.sweep_tols.split(",")):
                    rows.append(run(pts, tgt, p, 10, tol, k == 0))
            del pts, tgt
            torch.cuda.empty_cache()
        metric = "tau x N x p sweep (Figs. 2-4): E_rms, E_inf, nodes"
        targets = "N_q = N_p"
    line = {"metric": metric, "unit": "see rows", "n_gpus": world,
            "dtype": "f64" if prec == F.FMT_FP64 else "f64+bf16 (mixed path)", "data": "synthetic",
            "config": {"workload": args.workload, "points": "uniform [0,1)^3", "values": "Franke (Eq. eqF1)",
                       "targets": targets, "min_pts": 0}, "rows": rows}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def serve_measure(args, n_requests, rate, slots, seed_offset=0):
    """One Poisson stream of fit+evaluate requests through the library's
    serving engine (continuous batching over worker streams).  Latency =
    completion minus submission on the engine's clock, with the
    host->device copy of the request's arrays and the device->host copy of
    its results inside it."""
    import threading

    import numpy as np
    import torch
    from paper_1511_01353_gb300 import fmt as F
    from paper_1511_01353_gb300 import workloads as W

    reqs = W.serve_stream(n_requests=n_requests, rate=rate, seed=W.SEED_BASE + 4 + seed_offset)
    prec = {"fp64": F.FMT_FP64, "mixed": F.FMT_MIXED}

    def params(r):
        return F.make_params(r.degree, 8, 0, 1e-6, precision=prec[r.precision], sweeps=args.sweeps)

    sv = F.Server(slots=slots, budget_bytes=150e9, max_batch_points=4_000_000)
    for r in reqs[:max(args.warmup, 1)]:  # warm-up: contexts, pools, kernels
        sv.wait(sv.submit(params(r), r.x[:2000], r.y[:2000], r.z[:2000], r.f[:2000], r.xq[:100], r.yq[:100],
                          r.zq[:100]))
    sampler = ClockSampler("GPU-" + str(torch.cuda.get_device_properties(0).uuid))
    sampler.start()
    tickets = [None] * len(reqs)
    t0 = F.Server.clock()

    def submitter():
        for i, r in enumerate(reqs):
            dt = t0 + r.arrival - F.Server.clock()
            if dt > 0:
                time.sleep(dt)
            tickets[i] = sv.submit(params(r), r.x, r.y, r.z, r.f, r.xq, r.yq, r.zq, keep=True)

    th = threading.Thread(target=submitter)
    th.start()
    th.join()
    waited = [sv.wait(t) for t in tickets]
    infos = [w_[1] for w_ in waited]
    clocks = sampler.stop()
    # every tree stayed resident: evaluate-only requests against them (the
    # request's own first targets, up to 1e4), then release
    mem_fit = sv.memory()
    ev_lat, ev_ok, ev_t = [], True, 0
    for r, (out_fit, inf) in zip(reqs, waited):
        if inf["resident_id"] <= 0:
            continue
        k = min(10_000, r.xq.shape[0])
        t0e = F.Server.clock()
        out_e, ie = sv.wait(sv.submit_eval(inf["resident_id"], r.xq[:k], r.yq[:k], r.zq[:k]))
        ev_lat.append(ie["t_done"] - ie["t_submit"])
        ev_t += k
        ev_ok = ev_ok and ie["status"] == F.FMT_OK and bool(np.array_equal(out_e, out_fit[:k]))
    for inf in infos:
        if inf["resident_id"] > 0:
            sv.release(inf["resident_id"])
    mem_end = sv.memory()
    sv.close()
    resident = {"trees_kept": sum(1 for i in infos if i["resident_id"] > 0),
                "admitted_bytes_with_all_resident": mem_fit["admitted"],
                "peak_admitted_bytes": mem_end["peak_admitted"], "admitted_after_release": mem_end["admitted"],
                "eval_requests": len(ev_lat), "eval_targets": ev_t,
                "eval_p50_ms": float(np.percentile(ev_lat, 50) * 1e3) if ev_lat else None,
                "eval_p99_ms": float(np.percentile(ev_lat, 99) * 1e3) if ev_lat else None,
                "eval_equal_to_fit_time_values": ev_ok,
                "note": "each request kept its tree on the device; one evaluate-only request per tree "
                        "(its first <= 1e4 targets), one at a time, then every tree released"}
    lat = np.array([i["t_done"] - i["t_submit"] for i in infos])
    ok = all(i["status"] == F.FMT_OK for i in infos)
    pts = np.array([r.x.shape[0] for r in reqs], dtype=np.float64)
    tg = np.array([r.xq.shape[0] for r in reqs], dtype=np.float64)
    span = max(i["t_done"] for i in infos) - min(i["t_submit"] for i in infos)
    by = {}
    for name in ("fp64", "mixed"):
        sel = np.array([r.precision == name for r in reqs])
        if sel.any():
            by[name] = {"requests": int(sel.sum()), "p50_ms": float(np.percentile(lat[sel], 50) * 1e3),
                        "p99_ms": float(np.percentile(lat[sel], 99) * 1e3), "points": int(pts[sel].sum())}
    offered = pts.sum() / max(reqs[-1].arrival, 1e-9)
    return {"value": float(pts.sum() / span), "unit": UNIT, "span_ms": span * 1e3,
            "config": {"workload": "serve: %d requests, Poisson %.0f/s, points log-uniform [1e3, 2e6], targets "
                                   "log-uniform [1, 1e6], p 4..10, FP64 or mixed per request" % (len(reqs), rate),
                       "slots": slots, "budget_bytes": 150e9, "max_batch_points": 4_000_000,
                       "max_depth": 8, "tol_rel": 1e-6},
            "evals_per_s": float(tg.sum() / span), "all_ok": ok,
            "statuses": {str(k): sum(1 for i in infos if i["status"] == k) for k in set(i["status"] for i in infos)},
            "latency": by, "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "offered_points_per_s": float(offered), "completed_points_per_s": float(pts.sum() / span),
            "saturated": bool(offered > pts.sum() / span),
            "batches": len(set(i["batch_id"] for i in infos)),
            "mean_batch_requests": float(np.mean([i["batch_requests"] for i in infos])),
            "clocks": clocks, "resident": resident,
            "h2d_bytes": int(32 * pts.sum() + 24 * tg.sum()), "d2h_bytes": int(8 * tg.sum())}


def run_serve(args, rank, world):
    """Serving: the Poisson request stream as the headline line."""
    import torch
    from paper_1511_01353_gb300 import fmt as F

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    F.load()
    s = serve_measure(args, args.requests, args.rate, args.slots, 1000 * rank)
    line = {"metric": "fitted pts/s and p50/p99 request latency (serving)", "value": s["value"],
            "unit": UNIT, "n_gpus": world, "steps": 1, "warmup": max(args.warmup, 1),
            "ms_per_step": s["span_ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64 and f64+bf16 per request", "data": "synthetic"}
    line.update({k: v for k, v in s.items() if k not in ("value", "unit", "span_ms", "h2d_bytes", "d2h_bytes")})
    line["e2e"] = {"value": s["value"], "unit": UNIT, "h2d_bytes_per_step": s["h2d_bytes"],
                   "d2h_bytes_per_step": s["d2h_bytes"]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def block_c3(args, stream, flush):
    """The precision form of the small workload: its 4096 points and 1e4
    targets at p = 8, depth 7 (min 64 points, tol 1e-4), fitted and
    evaluated on the mixed path and on the FP64 path, each compared with the
    FP64 oracle at the targets and at the data points (error relative to
    max|f|; target for the mixed path 1e-6)."""
    import numpy as np
    import torch
    from oracle import oracle as O
    from paper_1511_01353_gb300 import fmt as F
    from paper_1511_01353_gb300 import workloads as W

    w = W.small()
    p, D, mp, tol = 8, 7, w.min_pts, w.tol_rel
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    x, y, z, f = dev(w.x), dev(w.y), dev(w.z), dev(w.f)
    xq, yq, zq = dev(w.xq), dev(w.yq), dev(w.zq)
    out = torch.empty(w.m, dtype=torch.float64, device="cuda")
    T = O.fit(w.x, w.y, w.z, w.f, p, D, mp, tol)
    ref_q, _ = T.evaluate(w.xq, w.yq, w.zq)
    ref_d, _ = T.evaluate(w.x, w.y, w.z)
    scale = max(T.maxabs, 1e-300)
    res = {"workload": "small_n4096_p8_d7_min64_tol1e-4", "points": w.n, "targets": w.m, "degree": p,
           "max_depth": D, "oracle_nodes": int(T.n_nodes)}
    steps, warm = max(args.steps, 5), max(args.warmup, 3)
    for name, prec in (("mixed", F.FMT_MIXED), ("fp64", F.FMT_FP64)):
        prm = F.make_params(p, D, mp, tol, precision=prec, sweeps=args.sweeps)
        fit_ms, ev_ms = [], []
        for i in range(warm + steps):
            with torch.cuda.stream(stream):
                flush.fill_(1.0)
                a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                a.record(stream)
                tr = F.fit(prm, x, y, z, f, stream)
                b.record(stream)
                F.evaluate(tr, xq, yq, zq, out, stream=stream)
                c.record(stream)
            stream.synchronize()
            if i >= warm:
                fit_ms.append(a.elapsed_time(b))
                ev_ms.append(b.elapsed_time(c))
            if i < warm + steps - 1:
                tr.close()
        gq = out.cpu().numpy()
        outd = torch.empty(w.n, dtype=torch.float64, device="cuda")
        F.evaluate(tr, x, y, z, outd, stream=stream)
        stream.synchronize()
        gd = outd.cpu().numpy()
        st = F.fmt_tree_stats(tr)
        nodes = int(sum(st.nodes[d] for d in range(st.n_levels)))
        tr.close()
        fm = float(np.mean(fit_ms))
        res[name] = {"value": w.n / (fm * 1e-3), "unit": UNIT, "fit_ms": fm, "eval_ms": float(np.mean(ev_ms)),
                     "evals_per_s": w.m / (float(np.mean(ev_ms)) * 1e-3),
                     "max_err_vs_oracle_over_max_f_targets": float(np.max(np.abs(gq - ref_q))) / scale,
                     "max_err_vs_oracle_over_max_f_data": float(np.max(np.abs(gd - ref_d))) / scale,
                     "nodes": nodes, "steps": steps, "warmup": warm}
    res["mixed"]["target_err"] = 1e-6
    res["fp64"]["target_err"] = 1e-10
    res["note"] = ("4096 points fit in a few ms: launch- and latency-bound at this size (no roofline claimed); "
                   "errors against the FP64 oracle run in the same job")
    return res


def block_batch(args, stream, flush):
    """The batched form: 4096 independent problems (degrees 4..10, log-uniform
    sizes, 4.76e7 points) as one forest, one timed step each on the FP64 and
    the mixed path after a warm-up on the first 256 problems; mixed against
    FP64 at every target, and both against the FP64 oracle on a sample of
    problems."""
    import numpy as np
    import torch
    from oracle import oracle as O
    from paper_1511_01353_gb300 import fmt as F
    from paper_1511_01353_gb300 import workloads as W

    t_gen = time.perf_counter()
    w = W.batch(n_problems=args.problems, seed=W.SEED_BASE + 3)
    t_gen = time.perf_counter() - t_gen
    N, M, P = int(w.offsets[-1]), int(w.xq.shape[0]), w.n_problems
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    x, y, z, f = dev(w.x), dev(w.y), dev(w.z), dev(w.f)
    xq, yq, zq, tp = dev(w.xq), dev(w.yq), dev(w.zq), dev(w.tprob)
    out = torch.empty(M, dtype=torch.float64, device="cuda")
    preds, res = {}, {}
    # the project's autotuner on the first 256 problems (all degrees, concurrent launches)
    k = min(256, P)
    nk = int(w.offsets[k])
    t_tune = time.perf_counter()
    tprm = F.make_params(4, w.max_depth, w.min_pts, w.tol_rel)
    tune = F.fmt_autotune_forest(tprm, w.offsets[:k + 1], x[:nk], y[:nk], z[:nk], f[:nk], degrees=w.degrees[:k],
                                 boxes=w.boxes[:k], stream=stream)
    tune["seconds"] = time.perf_counter() - t_tune
    tune["sample"] = "first %d problems (%d points), FP64 level loop timed per candidate" % (k, nk)
    tune["table"] = {str(d): {kk: F.fmt_tune_get(d)[kk] for kk in ("rows", "warps", "chunk_factor", "merge", "source")}
                     for d in sorted(set(int(v) for v in w.degrees))}
    # the problem of every data point, to evaluate each fit at its own data
    pp = torch.from_numpy(np.repeat(np.arange(P, dtype=np.int32), np.diff(w.offsets))).cuda()
    outd = torch.empty(N, dtype=torch.float64, device="cuda")
    at_data = {}
    for name, prec in (("fp64", F.FMT_FP64), ("mixed", F.FMT_MIXED)):
        prm = F.make_params(4, w.max_depth, w.min_pts, w.tol_rel, precision=prec, sweeps=args.sweeps)
        # warm-up on the first 256 problems (kernels, pools, tables)
        k = min(256, P)
        nk, mk = int(w.offsets[k]), int(w.toff[k])
        tw = F.fit_all(F.oct_build_batch(prm, w.offsets[:k + 1], x[:nk], y[:nk], z[:nk], f[:nk],
                                         degrees=w.degrees[:k], boxes=w.boxes[:k], stream=stream), stream)
        F.evaluate_batch(tw, tp[:mk], xq[:mk], yq[:mk], zq[:mk], out[:mk], stream=stream)
        stream.synchronize()
        tw.close()
        F.fmt_profile_enable(True)
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
            a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            a.record(stream)
            tr = F.fit_all(F.oct_build_batch(prm, w.offsets, x, y, z, f, degrees=w.degrees, boxes=w.boxes,
                                             stream=stream), stream)
            b.record(stream)
            F.evaluate_batch(tr, tp, xq, yq, zq, out, stream=stream)
            c.record(stream)
        stream.synchronize()
        prof = F.fmt_profile_read()
        F.fmt_profile_enable(False)
        preds[name] = out.cpu().numpy()
        F.evaluate_batch(tr, pp, x, y, z, outd, stream=stream)  # untimed: the interpolant at the data
        stream.synchronize()
        at_data[name] = outd.cpu().numpy()
        st = F.fmt_tree_stats(tr)
        fl = F.parse_export(F.fmt_tree_export(tr)).flags if name == "mixed" else None
        tr.close()
        fit_s, ev_s = a.elapsed_time(b) * 1e-3, b.elapsed_time(c) * 1e-3
        qr = prof.get("tile_qr", {})
        res[name] = {"value": N / fit_s, "unit": UNIT, "fit_ms": fit_s * 1e3, "eval_ms": ev_s * 1e3,
                     "evals_per_s": M / ev_s,
                     "nodes": int(sum(st.nodes[d] for d in range(st.n_levels))),
                     "kernels_ms": {kk: round(v["ms"], 2) for kk, v in prof.items()
                                    if v["launches"] and kk != "graph_launch"},
                     "gpu_launches": int(sum(v["launches"] for kk, v in prof.items() if kk != "graph_launch"))}
        if qr.get("ms") and qr.get("flops"):
            ach = qr["flops"] / (qr["ms"] * 1e-3) / 1e12
            res[name]["tile_qr_roofline"] = {"bound": "alu", "achieved": ach, "peak": FP64_NOMINAL_TFLOPS,
                                             "unit": "TFLOP/s", "frac": ach / FP64_NOMINAL_TFLOPS}
        if fl is not None:
            tc = (fl & F.FMT_FLAG_MIXED) != 0
            t2 = (fl & F.FMT_FLAG_MIXED_FP64) != 0
            res[name]["nodes_by_tier"] = {"tensor": int(np.sum(tc & ~t2)), "fp64_normal_eq": int(np.sum(t2)),
                                          "householder": int(np.sum(~tc))}
    # per-problem error of the mixed path against the FP64 path, relative to the problem's max|f|:
    # at the problem's targets and at its data points
    rel = np.empty(P)
    rel_data = np.empty(P)
    fmax = np.empty(P)
    for i in range(P):
        a_, b_ = int(w.toff[i]), int(w.toff[i + 1])
        da, db = int(w.offsets[i]), int(w.offsets[i + 1])
        fmax[i] = max(float(np.max(np.abs(w.f[da:db]))), 1e-300)
        rel[i] = float(np.max(np.abs(preds["mixed"][a_:b_] - preds["fp64"][a_:b_]))) / fmax[i]
        rel_data[i] = float(np.max(np.abs(at_data["mixed"][da:db] - at_data["fp64"][da:db]))) / fmax[i]
    del at_data
    # both paths against the oracle on a sample of problems, one per degree, the smallest of each
    sample, ora = [], {"fp64": 0.0, "mixed": 0.0}
    t_or = time.perf_counter()
    for d in sorted(set(int(v) for v in w.degrees)):
        idx = [i for i in range(P) if int(w.degrees[i]) == d]
        i = min(idx, key=lambda j: int(w.offsets[j + 1] - w.offsets[j]))
        a_, b_ = int(w.offsets[i]), int(w.offsets[i + 1])
        T = O.fit(w.x[a_:b_], w.y[a_:b_], w.z[a_:b_], w.f[a_:b_], d, w.max_depth, w.min_pts, w.tol_rel,
                  mode="omp")
        qa, qb = int(w.toff[i]), int(w.toff[i + 1])
        ref, _ = T.evaluate(w.xq[qa:qb], w.yq[qa:qb], w.zq[qa:qb])
        for name in ora:
            ora[name] = max(ora[name], float(np.max(np.abs(preds[name][qa:qb] - ref))) / max(T.maxabs, 1e-300))
        sample.append(i)
    # Targets where the two paths differ by more than the mixed bar lie where
    # a node's polynomial extrapolates beyond its data (a cluster's node box
    # far from its points), where rounding-sized changes of the data move the
    # fit by orders of magnitude more: the FP64 path against the oracle at
    # those problems' targets shows how ill-determined the value is there.
    over = [i for i in np.argsort(-rel) if rel[i] > 1e-6]
    context = []
    for i in over[:4]:
        a_, b_ = int(w.offsets[i]), int(w.offsets[i + 1])
        if b_ - a_ > 40000:
            continue
        T = O.fit(w.x[a_:b_], w.y[a_:b_], w.z[a_:b_], w.f[a_:b_], int(w.degrees[i]), w.max_depth, w.min_pts,
                  w.tol_rel, mode="omp")
        qa, qb = int(w.toff[i]), int(w.toff[i + 1])
        ref, _ = T.evaluate(w.xq[qa:qb], w.yq[qa:qb], w.zq[qa:qb])
        context.append({"problem": int(i), "points": b_ - a_, "degree": int(w.degrees[i]),
                        "mixed_vs_fp64": float(rel[i]), "mixed_vs_fp64_at_data": float(rel_data[i]),
                        "fp64_vs_oracle_at_targets": float(np.max(np.abs(preds["fp64"][qa:qb] - ref))) / T.maxabs})
    t_or = time.perf_counter() - t_or
    return {"workload": w.name, "problems": P, "points": N, "targets": M,
            "degree": "%d..%d per problem" % (w.degrees.min(), w.degrees.max()),
            "max_depth": w.max_depth, "min_pts": w.min_pts, "tol_rel": w.tol_rel,
            "fp64": res["fp64"], "mixed": res["mixed"],
            "mixed_over_fp64_fitted_pts_per_s": res["mixed"]["value"] / res["fp64"]["value"],
            "mixed_vs_fp64_max_err_over_max_f": float(np.max(rel)),
            "mixed_vs_fp64_median_err_over_max_f": float(np.median(rel)),
            "mixed_vs_fp64_at_data_max_err_over_max_f": float(np.max(rel_data)),
            "problems_above_1e-6_at_targets": len(over),
            "above_bar_context": context,
            "vs_oracle_max_err_over_max_f": ora,
            "oracle_sample": "problems %s (the smallest of each degree), oracle fit %.1f s" % (sample, t_or),
            "autotune": tune,
            "l2": "flushed before each timed step (256 MB write)",
            "warmup": "first 256 problems, each path", "steps": 1, "generation_s": t_gen,
            "target_err": {"mixed": 1e-6, "fp64": 1e-10}}


def block_serve(args):
    """The serving configuration as a block of the default line."""
    s = serve_measure(args, args.requests, args.rate, args.slots)
    s.pop("span_ms", None)
    return s


def mixed_rooflines(prof, degree, steps, probe_tflops, peaks):
    """Per-kernel roofline of the mixed path's kernels from their launch
    units (rows or nodes) and the algorithmic work per unit at `degree`."""
    L = (degree + 1) * (degree + 2) * (degree + 3) // 6
    m = L + 1
    Lp = (m + 15) // 16 * 16
    band1 = max(Lp - 128, 0)
    out = {}

    def entry(name, bound, work, unit, peak, peak_source, what):
        v = prof.get(name, {})
        if not v.get("ms"):
            return
        ach = work(v) / (v["ms"] * 1e-3) / (1e12 if unit == "TFLOP/s" else 1e9)
        out[name] = {"bound": bound, "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak,
                     "peak_source": peak_source, "ms_per_step": v["ms"] / steps, "work": what}

    fp64_src = "GB300 nominal FP64 (non-tensor) 1.25 TFLOP/s; live DFMA probe %.3f" % probe_tflops
    # tensor Gram: six digit-pair products of the 128-lane bands, M = 128, K = 64 per 64-row atom
    gram_flops_row = 6 * 2 * 128 * (Lp + band1)
    entry("mixed_gram", "tensor", lambda v: v["units"] * gram_flops_row, "TFLOP/s", peaks["bf16_tflops"],
          peaks["source"] + " (bf16 dense, burst)",
          "issued MMA flops: 6 digit-pair products x 2 x 128 x (%d + %d) per row" % (Lp, band1))
    # projection: the cached digit tiles (4 x Lp rows x 128 B per 64-row atom) and s (8 B) per row
    proj_bytes_row = 4 * Lp * 128 / 64 + 8
    entry("mixed_proj", "hbm", lambda v: v["units"] * proj_bytes_row, "GB/s", peaks["hbm_gbs"],
          peaks["source"] + " (copy)", "%.0f B per row (digit-tile cache + s)" % proj_bytes_row)
    # sweep residual: double-float Horner on the FP32 pipe, 18 FP32 instructions per multiply-add
    # (the library records 2 flops per multiply-add); peak = 152 SMs x 128 lanes x 2.07 GHz
    fp32_lane_instr_peak = 152 * 128 * 2.07e9 / 1e12
    entry("mixed_sresid", "alu", lambda v: v["flops"] / 2.0 * 18.0, "TFLOP/s", fp32_lane_instr_peak,
          "FP32 pipe issue rate (152 SMs x 128 lanes x 2.07 GHz, T lane-instructions/s)",
          "double-float Horner of s = r - Lambda F: 18 FP32 instructions per multiply-add (T lane-instr/s)")
    # factor: Cholesky of the m x m Gram (m^3 / 3 FMAs) + back substitution, per node
    entry("mixed_factor", "alu", lambda v: v["units"] * (2.0 * m ** 3 / 3.0 + 2.0 * L * L), "TFLOP/s",
          FP64_NOMINAL_TFLOPS, fp64_src, "2 m^3/3 + 2 L^2 flops per node (latency-bound: one node per CTA)")
    # update: two triangular solves, |R F| and the bias solves per node and sweep
    entry("mixed_update", "alu", lambda v: v["units"] * 6.0 * L * L, "TFLOP/s", FP64_NOMINAL_TFLOPS, fp64_src,
          "6 L^2 flops per node and sweep (latency-bound: one node per CTA)")
    entry("mixed_box", "hbm", lambda v: v["units"] * 32.0, "GB/s", peaks["hbm_gbs"], peaks["source"] + " (copy)",
          "32 B per row (x, y, z, r)")
    return out


def load_peaks():
    """The machine's measured peaks (generated MEASURED_PEAKS.json when
    present, else the figures it recorded for the GB300s)."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        hbm = float(d.get("hbm_gbs"))
        bf = float(d.get("bf16_tflops"))
        return {"hbm_gbs": hbm, "bf16_tflops": bf, "source": "MEASURED_PEAKS.json"}
    except Exception:
        return {"hbm_gbs": 6669.5, "bf16_tflops": 1982.8,
                "source": "measured peaks of this pool's GB300s (MEASURED_PEAKS.json not present in this run)"}


def main():
    args = parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return 0
    if args.workload == "serve":
        return run_serve(args, rank, world)
    if args.workload in ("fig1", "sweep"):
        return run_experiments(args, rank, world)

    import numpy as np
    import torch
    from paper_1511_01353_gb300 import fmt as F
    from paper_1511_01353_gb300 import workloads as W

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    F.load()
    stream = torch.cuda.Stream()
    w = make_workload(args, rank)
    prec_of = {"fp64": F.FMT_FP64, "mixed": F.FMT_MIXED}
    params = None if args.workload == "batch" else F.make_params(w.degree, w.max_depth, w.min_pts, w.tol_rel,
                                                                 precision=prec_of[args.precision],
                                                                 sweeps=args.sweeps, graph=args.graph)

    def dev(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")

    is_batch = args.workload == "batch"
    if is_batch:
        params = F.make_params(4, w.max_depth, w.min_pts, w.tol_rel, precision=prec_of[args.precision],
                               sweeps=args.sweeps, graph=args.graph)
        w.n = int(w.offsets[-1])
        w.m = int(w.xq.shape[0])
        w.name = w.name
        tprob = torch.from_numpy(w.tprob).to("cuda")
    x, y, z, f = dev(w.x), dev(w.y), dev(w.z), dev(w.f)
    xq, yq, zq = dev(w.xq), dev(w.yq), dev(w.zq)
    out = torch.empty(w.m, dtype=torch.float64, device="cuda")
    tuning = "built-in rule"
    if args.autotune:  # before any timed work; a level uses the entry of its largest degree
        tuning = {}
        for d in (sorted(set(int(v) for v in w.degrees)) if is_batch else [w.degree]):
            e = F.fmt_autotune(d, stream=stream)
            tuning[str(d)] = {k: e[k] for k in ("rows", "warps", "chunk_factor", "merge", "sample_points", "ms",
                                                "ms_builtin")}

    def build(xx, yy, zz, ff, prm=None):
        prm = params if prm is None else prm
        if is_batch:
            return F.oct_build_batch(prm, w.offsets, xx, yy, zz, ff, degrees=w.degrees, boxes=w.boxes,
                                     stream=stream)
        return F.oct_build(prm, xx, yy, zz, ff, stream)

    def evaluate(tree, qx, qy, qz):
        if is_batch:
            F.evaluate_batch(tree, tprob, qx, qy, qz, out, stream=stream)
        else:
            F.evaluate(tree, qx, qy, qz, out, stream=stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > L2 (129 MB)
    torch.cuda.synchronize()

    level_events = []

    def fit_with_level_events(lv, prm=None):
        # the driver loop of F.fit, with events around every fit_level
        tree = build(x, y, z, f, prm)
        d = 0
        while True:
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            F.fit_level(tree, d, stream)
            b.record(stream)
            lv.append((d, a, b))
            if F.refine(tree, d, stream) == 0:
                break
            d += 1
        return tree

    def step(timed, prm=None):
        with torch.cuda.stream(stream):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e2 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            tree = fit_with_level_events(level_events if timed else [], prm)
            e1.record(stream)
            evaluate(tree, xq, yq, zq)
            e2.record(stream)
        return tree, (e0, e1, e2)

    for _ in range(args.warmup):
        tree, _ = step(False)
        stream.synchronize()
        tree.close()

    gpu_name = torch.cuda.get_device_properties(local_rank).name
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local_rank).uuid)
    except Exception:
        uuid = str(local_rank)
    sampler = ClockSampler(uuid)
    sampler.start()
    time.sleep(0.3)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    F.fmt_profile_enable(True)
    evs, trees = [], []
    for _ in range(args.steps):
        tree, ev = step(True)
        evs.append(ev)
        trees.append(tree)
    stream.synchronize()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    prof = F.fmt_profile_read()
    F.fmt_profile_enable(False)
    clocks = sampler.stop()
    fit_ms = [a.elapsed_time(b) for a, b, _ in evs]
    eval_ms = [b.elapsed_time(c) for _, b, c in evs]
    last = trees[-1]
    ex = F.parse_export(F.fmt_tree_export(last))
    stats = F.fmt_tree_stats(last)
    for t in trees[:-1]:
        t.close()

    lvl_ms = {}
    for d, a, b in level_events:
        lvl_ms.setdefault(d, []).append(a.elapsed_time(b))
    level_fit_ms = [sum(lvl_ms[d]) / len(lvl_ms[d]) for d in sorted(lvl_ms)]
    fit_s = sum(fit_ms) / len(fit_ms) / 1e3
    eval_s = sum(eval_ms) / len(eval_ms) / 1e3
    fit_s, eval_s = reduce_max([fit_s, eval_s], dist, device="cuda")

    # accuracy of the interpolant against the closed form (last timed step)
    pred = out.cpu().numpy()
    acc_extra = {}
    if is_batch:
        rel = []
        for i in range(w.n_problems):
            a, b = int(w.toff[i]), int(w.toff[i + 1])
            tr = w.truth(i, w.xq[a:b], w.yq[a:b], w.zq[a:b])
            fi = w.f[int(w.offsets[i]):int(w.offsets[i + 1])]
            rel.append(W.errors(pred[a:b], tr)[0] / max(float(np.max(np.abs(fi))), 1e-300))
        rel = np.array(rel)
        truth = np.concatenate([w.truth(i, w.xq[w.toff[i]:w.toff[i + 1]], w.yq[w.toff[i]:w.toff[i + 1]],
                                        w.zq[w.toff[i]:w.toff[i + 1]]) for i in range(w.n_problems)])
        erms, einf = W.errors(pred, truth)
        acc_extra = {"per_problem_rel_rms_p50": float(np.median(rel)),
                     "per_problem_rel_rms_p90": float(np.percentile(rel, 90)),
                     "problems_rel_rms_below_1e-3": float(np.mean(rel < 1e-3)),
                     "note": "targets are fresh samples of each problem's cloud; clustered problems with "
                             "sparse tails extrapolate node polynomials there (E_inf)"}
    else:
        erms, einf = W.errors(pred, W.franke_bj(w.xq, w.yq, w.zq))

    # roofline of the dominant kernel (tile_qr, FP64 pipe); flops = 2 m^2 per row
    qr = prof.get("tile_qr", {})
    qr_tflops = qr["flops"] / (qr["ms"] * 1e-3) / 1e12 if qr.get("ms") else None
    dfma = F.fmt_probe_dfma(20000, stream)
    probe_tflops = 2.0 * dfma / 1e12
    fit_flops = sum(v["flops"] for k, v in prof.items() if k != "evaluate")
    deg = int(w.degrees.max()) if is_batch else w.degree
    ev_levels = 0 if is_batch else levels_visited(ex, w.xq, w.yq, w.zq, (0.0, 0.0, 0.0), 1.0)
    hf = 2.0 * (F.fmt_nmono(deg) + (deg + 1) * (deg + 2) / 2 + (deg + 1))
    ev = prof.get("evaluate", {})
    # a target inside its root cube evaluates one cumulative polynomial (its deepest node's)
    ev_tflops = w.m * hf * args.steps / (ev["ms"] * 1e-3) / 1e12 if ev.get("ms") else None
    total_ms = sum(v["ms"] for v in prof.values())
    kernels = {k: {"launches": v["launches"], "ms_per_step": v["ms"] / args.steps,
                   "share": (v["ms"] / total_ms if total_ms else None)} for k, v in prof.items() if v["launches"]}
    # kernel and memset launches (a graph launch replays launches counted here)
    gpu_launches = sum(v["launches"] for k, v in prof.items() if k != "graph_launch")

    # the other precision on the same inputs: throughput and its error against the headline path
    other = None
    if not args.no_second_path and not args.profile_only:
        oprec = "mixed" if args.precision == "fp64" else "fp64"
        oparams = F.make_params(params.degree, params.max_depth, params.min_pts, params.tol_rel,
                                precision=prec_of[oprec], sweeps=args.sweeps, graph=args.graph)
        for _ in range(max(1, min(args.warmup, 2))):
            tr, _ = step(False, oparams)
            stream.synchronize()
            tr.close()
        F.fmt_profile_enable(True)
        oev, otrees = [], []
        for _ in range(args.steps):
            tr, ev = step(False, oparams)
            oev.append(ev)
            otrees.append(tr)
        stream.synchronize()
        oprof = F.fmt_profile_read()
        F.fmt_profile_enable(False)
        ofit = reduce_max([sum(a.elapsed_time(b) for a, b, _ in oev) / len(oev) / 1e3,
                           sum(b.elapsed_time(c) for _, b, c in oev) / len(oev) / 1e3], dist, device="cuda")
        opred = out.cpu().numpy()
        ost = F.fmt_tree_stats(otrees[-1])
        oex = F.parse_export(F.fmt_tree_export(otrees[-1]))
        for tr in otrees:
            tr.close()
        fscale = max(float(np.max(np.abs(w.f))), 1e-300)
        mst = ost if oprec == "mixed" else stats
        mex = oex if oprec == "mixed" else ex
        def nodes_pts(sel):
            return int(np.sum(sel)), int(np.sum(mex.count[sel]))
        fl = mex.flags
        tc = (fl & F.FMT_FLAG_MIXED) != 0
        t2 = (fl & F.FMT_FLAG_MIXED_FP64) != 0
        # tensor-core tier: fitted there; its failures (small pivot / not converged / degree > 9) go to the
        # FP64 normal-equations tier, and what that tier cannot fit to the FP64 Householder path
        fallback = {"tensor_tier_nodes": nodes_pts(tc & ~t2)[0], "tensor_tier_points": nodes_pts(tc & ~t2)[1],
                    "fp64_tier_nodes": nodes_pts(t2)[0], "fp64_tier_points": nodes_pts(t2)[1],
                    "householder_nodes": nodes_pts(~tc)[0], "householder_points": nodes_pts(~tc)[1],
                    "tensor_tier_small_pivot_nodes": nodes_pts((fl & F.FMT_FLAG_MIXED_PIVOT) != 0)[0],
                    "tensor_tier_not_converged_nodes": nodes_pts((fl & F.FMT_FLAG_MIXED_SLOW) != 0)[0]}
        mixed_pts = sum(int(mst.mixed_points[d]) for d in range(mst.n_levels))
        all_pts = sum(int(mst.points[d]) for d in range(mst.n_levels))
        gram = oprof.get("mixed_gram", {}) if oprec == "mixed" else prof.get("mixed_gram", {})
        other = {"precision": oprec, "value": job_throughput(world, w.n, ofit[0]), "unit": UNIT,
                 "evals_per_s": job_throughput(world, w.m, ofit[1]), "fit_ms": ofit[0] * 1e3,
                 "eval_ms": ofit[1] * 1e3,
                 "fit_speedup_mixed_over_fp64": (fit_s / ofit[0]) if oprec == "mixed" else (ofit[0] / fit_s),
                 "max_abs_diff_vs_headline_over_max_f": float(np.max(np.abs(opred - pred))) / fscale,
                 "mixed_share_of_fitted_points": mixed_pts / max(all_pts, 1),
                 "mixed_nodes": int(sum(mst.mixed[d] for d in range(mst.n_levels))),
                 "tiers": fallback,
                 "kernels": {k: {"launches": v["launches"], "ms_per_step": v["ms"] / args.steps}
                             for k, v in oprof.items() if v["launches"]},
                 "rooflines": mixed_rooflines(oprof if oprec == "mixed" else prof, params.degree, args.steps,
                                              probe_tflops, load_peaks()),
                 "note": "error vs the FP64 GPU path, which matches the FP64 oracle to 1e-10 max|f|; "
                         "target for the mixed path: 1e-6 max|f|"}

    e2e = None
    if not args.no_e2e:
        # end to end through the public API: pinned host inputs -> device -> fit -> evaluate -> host
        hx, hy, hz, hf_ = (torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (w.x, w.y, w.z, w.f))
        hxq, hyq, hzq = (torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in (w.xq, w.yq, w.zq))
        hout = torch.empty(w.m, dtype=torch.float64).pin_memory()
        dx, dy, dz, df = (torch.empty_like(x) for _ in range(4))
        dxq, dyq, dzq = (torch.empty_like(xq) for _ in range(3))
        e2e_fit, e2e_eval = [], []
        for i in range(args.warmup + args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(1.0)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                c = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                for d_, h_ in ((dx, hx), (dy, hy), (dz, hz), (df, hf_)):
                    d_.copy_(h_, non_blocking=True)
                tr = F.fit_all(build(dx, dy, dz, df), stream)
                b.record(stream)
                for d_, h_ in ((dxq, hxq), (dyq, hyq), (dzq, hzq)):
                    d_.copy_(h_, non_blocking=True)
                evaluate(tr, dxq, dyq, dzq)
                hout.copy_(out, non_blocking=True)
                c.record(stream)
            stream.synchronize()
            if i >= args.warmup:
                e2e_fit.append(a.elapsed_time(b) / 1e3)
                e2e_eval.append(b.elapsed_time(c) / 1e3)
            tr.close()
        tf = sum(e2e_fit) / len(e2e_fit)
        te = sum(e2e_eval) / len(e2e_eval)
        e2e = {"value": world * w.n / tf, "unit": UNIT, "evals_per_s": world * w.m / te,
               "h2d_bytes_per_step": 32 * w.n + 24 * w.m, "d2h_bytes_per_step": 8 * w.m,
               "ms_per_step": (tf + te) * 1e3}

    if args.profile_only:
        return 0
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_batch(args, w) if is_batch else cpu_baseline(args)
    # the other configurations as blocks of the same line (one GPU only; not the headline)
    blocks = {}
    wanted = [b for b in args.blocks.split(",") if b and b != "none"]
    if rank == 0 and world == 1 and args.workload == "scale" and wanted:
        if "c3" in wanted:
            blocks["c3"] = block_c3(args, stream, flush)
        if "batch" in wanted:
            blocks["batch"] = block_batch(args, stream, flush)
            for d in range(F.FMT_MAX_DEGREE + 1):  # back to the built-in rule for what follows
                F.fmt_tune_set(dict(degree=d, source=0, rows=64, warps=4, chunk_factor=4, merge=0))
            torch.cuda.empty_cache()
        if "serve" in wanted:
            blocks["serve"] = block_serve(args)

    nodes = [int(stats.nodes[d]) for d in range(stats.n_levels)]
    points = [int(stats.points[d]) for d in range(stats.n_levels)]
    line = {
        "metric": METRIC, "value": job_throughput(world, w.n, fit_s), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": (fit_s + eval_s) * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f64+bf16 (tensor-core Gram and projection, FP64 factor/refine)",
        "data": "synthetic",
        "config": {"workload": w.name, "points": w.n, "targets": w.m,
                   "degree": ("%d..%d per problem" % (w.degrees.min(), w.degrees.max())) if is_batch else w.degree,
                   "problems": w.n_problems if is_batch else 1,
                   "nmono": F.fmt_nmono(deg), "max_depth": w.max_depth, "min_pts": w.min_pts,
                   "tol_rel": w.tol_rel,
                   "values": ("shifted/scaled Franke or Gaussian sums per problem" if is_batch
                              else "3-D Franke (benchmark form)"),
                   "l2": "flushed before every step (256 MB write)", "parallelism": "replicas",
                   "gpu": gpu_name, "graph": bool(args.graph), "qr_launch_config": tuning},
        "evals_per_s": job_throughput(world, w.m, eval_s), "fit_ms": fit_s * 1e3, "eval_ms": eval_s * 1e3,
        "roofline": {"bound": "alu", "kernel": "tile_qr", "achieved": qr_tflops, "peak": FP64_NOMINAL_TFLOPS,
                     "unit": "TFLOP/s", "frac": (qr_tflops / FP64_NOMINAL_TFLOPS if qr_tflops else None),
                     "traffic": (TILE_QR_DRAM_BYTES_PER_ROW * qr["units"] / qr["launches"]
                                 if TILE_QR_DRAM_BYTES_PER_ROW and qr.get("launches") else None),
                     "traffic_unit": "bytes per launch (ncu dram read+write, scaled per row from a "
                                     "3e5-point capture)",
                     "algorithmic_bytes": 32.0 * qr["units"] / qr["launches"] if qr.get("launches") else None,
                     "peak_source": "GB300 nominal FP64 (non-tensor) 1.25 TFLOP/s",
                     "probe_fp64_tflops": probe_tflops,
                     "frac_of_probe": (qr_tflops / probe_tflops if qr_tflops else None),
                     "flops_per_row": "2 m^2, m = nmono + 1 (Householder on [Lambda | r])"},
        "fit_roofline": {"bound": "alu", "achieved": fit_flops / args.steps / fit_s * 1e-12, "unit": "TFLOP/s",
                         "peak": FP64_NOMINAL_TFLOPS,
                         "frac": fit_flops / args.steps / fit_s * 1e-12 / FP64_NOMINAL_TFLOPS,
                         "what": "algorithmic flops of the whole fit phase / fit wall time"},
        "eval_roofline": {"bound": "alu", "achieved": ev_tflops, "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                          "frac": (ev_tflops / FP64_NOMINAL_TFLOPS if ev_tflops else None),
                          "flops_per_target": hf, "levels_on_target_paths": ev_levels,
                          "what": "one Horner evaluation of the deepest node's cumulative polynomial per target"},
        "kernels": kernels, "gpu_launches": gpu_launches, "clocks": clocks,
        "tree": {"nodes": nodes, "points": points, "level_fit_ms": level_fit_ms,
                 "level_items": [int(stats.items[d]) for d in range(stats.n_levels)],
                 "level_chunk_rows": [int(stats.chunk_rows[d]) for d in range(stats.n_levels)], "near_tau": int(sum(stats.near_tau[d] for d in range(22))),
                 "rank_flagged": int(sum(stats.rank_flagged[d] for d in range(22)))},
        "accuracy": dict({"E_rms": erms, "E_inf": einf,
                          "vs": ("generating function of each problem at its targets" if is_batch
                                 else "closed-form Franke at the targets")}, **acc_extra),
        "e2e": e2e, "cpu_baseline": cpu,
        "precision": args.precision, ("mixed" if args.precision == "fp64" else "fp64"): other,
    }
    line.update(blocks)
    last.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
