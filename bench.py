#!/usr/bin/env python
"""Benchmark: layered-media FMM matvec throughput (Mpts/s) on the C2 workload.

Workload (synthetic, seeded): three-layer medium with interfaces y = 0, -2,
k = (4, 6, 8), eta = (1, 2, 3); 64 circles/ellipses (radii in [0.2, 0.6],
centres in [-10, 10] x [-4, 2], seed 12452, some crossing interfaces) with
1024 boundary nodes each, N = 65536 Nystrom points; FMM order p = 20; FP64.

One step = one application of the Nystrom operator y = K x through
lfmm_matvec (gather, P2M, M2M, M2L free-space + reaction, L2L, L2P, near
field, scatter) with x and y resident in HBM; the L2 cache is flushed before
every step.  The GMRES solve to 1e-8 with the DD preconditioner and the
set-up time are reported beside it.  With --gpus N > 1 each rank solves its
own replica of the workload (the matvec of one geometry does not shard), and
`value` sums the ranks' throughput over the slowest rank's time.

--impl reference times the FP64 CPU oracle (dense Nystrom rows with direct
Sommerfeld quadrature) on the host cores on a bounded sample of rows.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

HBM_FALLBACK_GBS = 6800.0
# FP64 peak from unit counts and clock: 152 SMs x 2 DFMA/clk x 2 flops x 2.07 GHz
# (a DFMA microbenchmark on the same GPU model reached 1.194 TFLOP/s, 95 %)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# DRAM traffic per launch from the committed ncu captures (profiles/); null once the
# kernel changes after the capture
NCU_TRAFFIC_BYTES = {"k_m2l": 85761280.0 + 3519488.0, "k_near_leaf": 67980800.0 + 316160.0,
                     "k_near_leaf (precision form)": 38071040.0}


def run_combined(lfmm, wl, M, pts, w, nrm, x, flush, stream, args, dist, n):
    """The combined-field operator (opt-in second-kind form) on the same workload:
    matvec throughput timed like the headline, and the GMRES solve."""
    import torch

    t0 = time.perf_counter()
    Gc = lfmm.geometry_build(M, pts, w, nrm, p=wl.p, leaf_size=wl.leaf_size, combined=True)
    setup_s = time.perf_counter() - t0
    y = torch.empty_like(x)
    for _ in range(args.warmup):
        lfmm.matvec(Gc, x, y)
    torch.cuda.synchronize()
    times = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lfmm.matvec(Gc, x, y)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    value, slowest = whole_job_throughput(float(np.sum(times)) * 1e-3, n * args.steps, dist, "cuda")
    b = lfmm.rhs_plane_wave(Gc, [math.radians(float(wl.angles_deg[0]))], device=True)
    _, info = lfmm.gmres_solve(Gc, b, tol=1e-8, max_iter=1000, precond=True)
    _, im = lfmm.gmres_solve(Gc, b, tol=1e-8, max_iter=1000, precond=True, precision=1)
    return {"metric": "FMM matvec Mpts/s, combined-field operator", "value": value,
            "ms_per_step": slowest * 1e3 / args.steps, "setup_seconds": setup_s,
            "solve": {"seconds": info["solve_seconds"], "iterations": info["iterations"],
                      "true_rel_residual": info["true_rel_residual"], "converged": bool(info["converged"])},
            "solve_mixed": {"seconds": im["solve_seconds"], "iterations": im["iterations"],
                            "true_rel_residual": im["true_rel_residual"], "converged": bool(im["converged"])}}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2", choices=["c2", "c1"])
    ap.add_argument("--no-solve", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-c3", action="store_true", help="skip the million-point four-layer workload block")
    ap.add_argument("--serve-full", type=int, default=0,
                    help="run only the serving form on this many requests drawn like the serving "
                         "configuration itself (N up to 262,144, up to 512 bodies) and print it as one JSON line")
    ap.add_argument("--only-batch", action="store_true",
                    help="only the block right-hand side of one batching geometry (32 angles) and print it")
    ap.add_argument("--only-c3", action="store_true",
                    help="run only the million-point four-layer workload block (--steps timed matvecs per operator) "
                         "and print it as one JSON line")
    ap.add_argument("--autotune", type=int, default=0,
                    help="1: choose the M2L work-item schedule by timing at set-up")
    ap.add_argument("--replay", action="store_true",
                    help="replay the paper's Examples 1-3 (Sec. 5, Tables 5.1-5.3) as GPU solves and exit")
    ap.add_argument("--replay-max", type=int, default=192000, help="largest element count of the replay")
    return ap.parse_args()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": HBM_FALLBACK_GBS}, "fallback"


def workload(name):
    from workloads import config_c1, config_c2

    wl = config_c2() if name == "c2" else config_c1()
    desc = ("C2: 3-layer medium (interfaces y=0,-2; k=4,6,8; eta=1,2,3), 64 circles/ellipses x 1024 nodes, "
            "N=65536, p=20, FP64") if name == "c2" else "C1: 2-layer medium, 1 circle, N=256"
    return wl, desc


class Clocks:
    """nvidia-smi samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def whole_job_throughput(local_seconds, units_per_rank, dist=None, device="cpu"):
    """Units processed by all ranks over the slowest rank's time, in millions per second.

    Every rank passes its own timed seconds; the maximum over ranks is taken with
    one all-reduce (each rank runs an independent replica, so this is the only
    collective).  Returns (value, slowest seconds).
    """
    import torch

    t = torch.tensor([float(local_seconds)], dtype=torch.float64, device=device)
    world = 1
    if dist is not None and dist.is_available() and dist.is_initialized():
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        world = dist.get_world_size()
    slowest = float(t.item())
    return world * units_per_rank / slowest / 1e6, slowest


def setup_report(lf, G, seconds):
    """Set-up time of a geometry with its phases, and the reaction moment tables' FP64 rate: their
    complex multiply-adds (8 flop each; entries x quadrature nodes x 2 terms) over the far-field
    phase, which the tables dominate (an upper bound on their own time)."""
    ph = lf.geometry_query(G, "setup_times", np.float64)
    cm = lf.geometry_query(G, "table_work", np.float64)
    flops = 8.0 * float(cm[0] + cm[1])
    far_s = float(ph[2])
    tf = flops / far_s / 1e12 if far_s > 0 else None
    return {"seconds": seconds, "tree_and_lists_s": float(ph[0]), "near_field_s": float(ph[1]),
            "far_field_s": far_s, "table_gflop": flops / 1e9,
            "table_cmacs_cross_same": [float(cm[0]), float(cm[1])],
            "table_fp64_tflops": tf, "table_fp64_frac": (tf / FP64_PEAK_TFLOPS) if tf else None}


def algorithmic_work(lf, G, n):
    """Per-launch algorithmic FLOPs of M2L and bytes of the near field (one RHS column)."""
    lev = lf.geometry_query(G, "box_level")
    pl = lf.geometry_query(G, "p_level")
    vfp = lf.geometry_query(G, "vfree_ptr")
    vrp = lf.geometry_query(G, "vreact_ptr")
    nf = np.diff(vfp)
    nr = np.diff(vrp)
    coef = (2 * pl[lev] + 1).astype(np.float64)
    m2l_flops = float(np.sum((nf + nr) * 8.0 * coef * coef))
    tp = lf.geometry_query(G, "tree_params", np.float64)
    nnz = float(tp[8])
    near_bytes = 16.0 * nnz + 48.0 * n
    return {"m2l_flops": m2l_flops, "near_bytes": near_bytes, "near_nnz": nnz,
            "m2l_pairs_free": int(nf.sum()), "m2l_pairs_reaction": int(nr.sum()),
            "D": int(tp[3]), "l0": int(tp[4]), "reaction_tables": int(tp[9])}


def cpu_baseline(wl, rows_per_sample, n_samples=1):
    """Time the oracle on a bounded sample of full rows of K (FP64, host cores)."""
    from oracle import core, nystrom  # the oracle is only timed here (CPU baseline)

    pts, w, _, _ = nystrom.elements(wl.bodies)
    n = pts.shape[0]
    rng = np.random.default_rng(0)
    t0 = time.perf_counter()
    cnt = 0.0
    for _ in range(n_samples):
        r = rng.integers(0, n)
        cols = rng.permutation(n)[: int(rows_per_sample * n)] if rows_per_sample < 1 else None
        if cols is None:
            nystrom.dense_rows(wl.medium, pts, w, [r])
            cnt += 1.0
        else:
            # a random fraction of one row of the dense definition
            nystrom.dense_row_block(wl.medium, pts, w, r, cols)
            cnt += cols.size / n
    dt = time.perf_counter() - t0
    # full dense matvec time extrapolated from the per-row time: N rows
    t_full = dt / cnt * n
    return {"value": n / t_full / 1e6, "unit": "Mpts/s", "cores": core.num_threads(), "kind": "oracle",
            "sample": f"{cnt:g} full row(s) of the dense {n}x{n} Nystrom matrix with direct Sommerfeld "
                      f"quadrature, {dt:.1f} s; full matvec extrapolated to {t_full:.3g} s",
            "seconds": dt}


def run_serving(lfmm, n_requests=32, slots=8, seed=12455, n_max=131072.0, max_bodies=128, max_iter=2000):
    """Serving form on a bounded stand-in for the request stream (random 2-4 layer stacks,
    k in [2, 12], N log-uniform in [2k, n_max], up to max_bodies bodies): Poisson arrivals at
    1.5x the FP64 one-at-a-time capacity.  The arms see the same arrivals: FP64 one at a time
    (1 slot), FP64 served (``slots`` requests in flight, their GMRES steps advanced together
    with the FP64 products in shared launches), the served mixed-precision form and the served
    combined-field operator (second kind, opt-in); each solve to the FP64 residual 1e-8 within
    max_iter steps."""
    from workloads import config_c5_stream

    stream = config_c5_stream(n_requests, seed, n_max=n_max, max_bodies=max_bodies)
    reqs = []
    for wl in stream:
        pts, w, nrm = lfmm.polygon_elements(wl.bodies)
        reqs.append((wl.medium, pts, w, nrm, math.radians(float(wl.angles_deg[0]))))
    free, _total = __import__("torch").cuda.mem_get_info()
    budget = int(0.5 * free)

    def one_arm(n_slots, precision, arrivals, combined=False):
        srv = lfmm.Server(slots=n_slots, hbm_budget=budget)
        t0 = time.perf_counter()
        tickets = []
        for (med, pts, w, nrm, ang), ta in zip(reqs, arrivals):
            dt = ta - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            tickets.append(srv.submit(med.interfaces, med.k, med.eta, pts, w, ang, tol=1e-8,
                                      precision=precision, max_iter=max_iter, normals=nrm, combined=combined))
        lat, conv, res, its = [], 0, 0.0, 0
        for t in tickets:
            _x, info, tm = srv.wait(t)
            lat.append(tm["latency_seconds"])
            conv += int(info["converged"])
            res = max(res, info["true_rel_residual"])
            its += info["iterations"]
        wall = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        lat = np.array(lat) * 1e3
        return {"slots": n_slots, "precision": "mixed" if precision else "fp64",
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "solves_per_s": len(reqs) / wall, "converged": conv, "max_true_rel_residual": res,
                "iterations": its, "peak_running": st["peak_running"]}

    # capacity: every request submitted at once; latency: the same requests as a Poisson
    # stream at 1.5x the FP64 one-at-a-time capacity
    cap64 = one_arm(1, 0, [0.0] * len(reqs))
    rate = 1.5 * cap64["solves_per_s"]
    rng = np.random.default_rng(seed + 1)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=len(reqs)))
    out = {}
    for name, n_slots, prec, cf in (("fp64_one_at_a_time", 1, 0, False), ("fp64_served", slots, 0, False),
                                    ("mixed_served", slots, 1, False), ("combined_field_served", slots, 0, True)):
        cap = cap64 if name == "fp64_one_at_a_time" else one_arm(n_slots, prec, [0.0] * len(reqs), cf)
        lat = one_arm(n_slots, prec, arrivals, cf)
        out[name] = {"slots": n_slots, "precision": "mixed" if prec else "fp64",
                     "operator": "combined field" if cf else "single layer",
                     "capacity_solves_per_s": cap["solves_per_s"],
                     "p50_ms": lat["p50_ms"], "p99_ms": lat["p99_ms"],
                     "stream_solves_per_s": lat["solves_per_s"],
                     "converged": lat["converged"], "max_true_rel_residual": lat["max_true_rel_residual"],
                     "krylov_iterations": lat["iterations"], "peak_running": lat["peak_running"]}
    sizes = [int(r[2].size) for r in reqs]
    return {"metric": "served p50/p99 ms vs FP64 form",
            "workload": f"{len(reqs)} requests, random 2-4 layer stacks, k in [2,12], N {min(sizes)}..{max(sizes)}; "
                        f"latency under Poisson arrivals at 1.5x the FP64 one-at-a-time capacity "
                        f"({rate:.2f} requests/s); tol 1e-8 on the FP64 residual",
            "hbm_budget_bytes": budget, **out}


def run_c3(lfmm, steps=5):
    """The precision form's own workload, C3: four layers (interfaces y = 0, -6, -12; k = 6, 10,
    8, 12; eta = 1..4), 1024 circles/ellipses x 1024 nodes over [-40, 40] x [-18, 6] (seed
    12453), N = 1,048,576, p = 20.  Set-up time, the FP64 and precision-form matvec (L2 flushed,
    CUDA events, median), the errors of both against the 64 stored oracle rows (x non-zero on a
    seeded 4k-point subset) and of the precision form against FP64 on a dense random x, and the
    per-stage times of each operator."""
    import torch

    sys.path.insert(0, os.path.join(ROOT, "tests", "golden"))
    import make_c3_sampled_rows as gen
    from workloads import config_c3

    wl = config_c3()
    med = wl.medium
    M = lfmm.medium_create(med.interfaces, med.k, med.eta)
    pts, w, nrm = lfmm.polygon_elements(wl.bodies)
    t0 = time.perf_counter()
    G = lfmm.geometry_build(M, pts, w, nrm, p=wl.p, leaf_size=wl.leaf_size, profile=True)
    setup_s = time.perf_counter() - t0
    n = G.n
    with open(os.path.join(ROOT, "tests", "golden", "c3_sampled_rows.json")) as f:
        fx = json.load(f)
    cols, xs, rows = gen.sample(n)
    ref = np.array([complex(*v) for v in fx["y"]])
    xsp = np.zeros(n, dtype=np.complex128)
    xsp[cols] = xs
    xsp = torch.from_numpy(xsp).cuda()
    gen_t = torch.Generator(device="cpu").manual_seed(77)
    x = torch.complex(torch.randn(n, generator=gen_t, dtype=torch.float64),
                      torch.randn(n, generator=gen_t, dtype=torch.float64)).cuda()
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    out = {"workload": "C3: 4 layers (y=0,-6,-12; k=6,10,8,12; eta=1..4), 1024 circles/ellipses x 1024 nodes, "
                       "N=1048576, p=20", "N": n, "setup_seconds": setup_s,
           "setup": setup_report(lfmm, G, setup_s),
           "tree": {k: float(v) for k, v in zip(["D", "l0", "boxes", "components", "near_blocks", "near_entries",
                                                  "reaction_tables"], lfmm.geometry_query(G, "tree_params",
                                                                                          np.float64)[3:10])}}
    ys = {}
    for name, mixed in (("fp64", False), ("mixed", True)):
        y = torch.empty_like(x)
        for _ in range(2):
            lfmm.matvec(G, x, y, mixed=mixed)
        torch.cuda.synchronize()
        st0 = lfmm.stage_times(G)
        times = []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lfmm.matvec(G, x, y, mixed=mixed)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        st1 = lfmm.stage_times(G)
        ys[name] = y
        yr = lfmm.matvec(G, xsp, mixed=mixed).cpu().numpy()[rows]
        err = np.abs(yr - ref) / np.abs(ref)
        ms = float(np.median(times))
        out[name] = {"ms_per_matvec": ms, "Mpts_per_s": n / ms / 1e3,
                     "oracle_rows_max_rel_err": float(err.max()), "oracle_rows_median_rel_err": float(np.median(err)),
                     "stages_ms": {k: (st1[k]["ms"] - st0[k]["ms"]) / max(st1[k]["count"] - st0[k]["count"], 1)
                                   for k in st1}}
    out["mixed"]["op_rel_diff_vs_fp64"] = float(torch.linalg.norm(ys["mixed"] - ys["fp64"]) /
                                                torch.linalg.norm(ys["fp64"]))
    pf = lfmm.geometry_query(G, "precision_form", np.float64)
    out["mixed"]["fp32_from_level"] = int(pf[0])
    out["mixed"]["coarse_m2l"] = "double-float" if pf[1] == 1 else "FP64"
    out["mixed"]["coarse_log10_ranges"] = [float(v) for v in pf[2:]]
    # the precision form's near field against HBM (complex64 regular blocks, FP64 reaction
    # blocks and diagonal, x in FP64 and complex64, y read and written); the stage runs
    # beside the far field, so its live time includes the competition for the SMs
    ne = lfmm.geometry_query(G, "near_entries", np.float64)
    nbytes = 8.0 * ne[1] + 16.0 * ne[2] + 72.0 * n
    peaks, src = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", HBM_FALLBACK_GBS))
    t_near = out["mixed"]["stages_ms"]["near"] * 1e-3
    out["mixed"]["near_roofline"] = {"kernel": "k_near_leaf_w (precision form)", "bound": "hbm",
                                     "algorithmic_bytes": nbytes, "entries_complex64": int(ne[1]),
                                     "entries_fp64": int(ne[2]),
                                     "achieved": nbytes / t_near / 1e9 if t_near > 0 else None, "peak": hbm,
                                     "unit": "GB/s", "frac": (nbytes / t_near / 1e9 / hbm) if t_near > 0 else None,
                                     "peak_source": src, "note": "live stage time inside the matvec"}
    G.destroy()
    return out


def run_batch(lfmm, index=10, steps=5, solve=True):
    """Block right-hand side: one geometry of the batching configuration (C4 geometry
    `index`, 2-4 layers, k in [2, 12]) with its 32 incidence angles as one 32-column matvec,
    against 32 single-column matvecs; L2 flushed before every timed call."""
    import torch

    from workloads import config_c4

    wl = config_c4()[index]
    med = wl.medium
    M = lfmm.medium_create(med.interfaces, med.k, med.eta)
    pts, w, nrm = lfmm.polygon_elements(wl.bodies)
    G = lfmm.geometry_build(M, pts, w, nrm, p=wl.p, leaf_size=wl.leaf_size)
    n = G.n
    ang = np.radians(wl.angles_deg)
    B = lfmm.rhs_plane_wave(G, ang, device=True)          # [32, n]: column-major n x 32
    Y = torch.empty_like(B)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def timed(fn):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            tot += e0.elapsed_time(e1)
        return tot / steps * 1e-3

    t_block = timed(lambda: lfmm.matvec(G, B, Y))
    cols = [B[c] for c in range(B.shape[0])]
    outs = [torch.empty_like(c) for c in cols]

    def singles():
        for c, o in zip(cols, outs):
            lfmm.matvec(G, c, o)

    t_single = timed(singles)
    same = max(float(torch.linalg.norm(Y[c] - outs[c]) / torch.linalg.norm(outs[c])) for c in range(len(cols)))
    nr = B.shape[0]
    # precision form of the block: M2L of the FP32 levels on the tensor cores (3xTF32)
    # against the same operator with its M2L on the SIMT kernel
    Ym, Ys = torch.empty_like(B), torch.empty_like(B)
    t_mixed_tc = timed(lambda: lfmm.matvec(G, B, Ym, mixed=True))
    t_mixed_simt = timed(lambda: lfmm.matvec(G, B, Ys, mixed=True, simt_m2l=True))
    rel = lambda a, b: max(float(torch.linalg.norm(a[c] - b[c]) / torch.linalg.norm(b[c])) for c in range(nr))
    out = {"metric": "block right-hand side matvec, Mpts*rhs/s", "workload": f"C4 geometry {index}: {len(med.k)} layers, "
           f"N={n}, {nr} incidence angles", "block_value": n * nr / t_block / 1e6,
           "single_column_value": n * nr / t_single / 1e6, "block_ms": t_block * 1e3,
           "single_columns_ms": t_single * 1e3, "max_rel_diff_block_vs_single": same,
           "mixed_block_tensor_core_value": n * nr / t_mixed_tc / 1e6, "mixed_block_tensor_core_ms": t_mixed_tc * 1e3,
           "mixed_block_simt_value": n * nr / t_mixed_simt / 1e6, "mixed_block_simt_ms": t_mixed_simt * 1e3,
           "mixed_tensor_core_vs_fp64_max_rel_diff": rel(Ym, Y), "mixed_tensor_core_vs_simt_max_rel_diff": rel(Ym, Ys)}
    if not solve:
        return out
    # several angles solved together (one Krylov space per column, block matvecs) against
    # the same angles one by one; 8 of the 32 keep the section short
    na = 8
    B8 = B[:na].contiguous()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    X8, info8 = lfmm.gmres_solve(G, B8, tol=1e-8, max_iter=1000)
    torch.cuda.synchronize()
    t_simul = time.perf_counter() - t0
    t0 = time.perf_counter()
    xs1 = [lfmm.gmres_solve(G, B8[c].contiguous(), tol=1e-8, max_iter=1000)[0] for c in range(na)]
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    same_solve = max(float(torch.linalg.norm(X8[c] - xs1[c]) / torch.linalg.norm(xs1[c])) for c in range(na))
    out["angles_solved_together"] = {"angles": na, "seconds": t_simul, "one_by_one_seconds": t_seq,
                                     "converged": bool(info8["converged"]),
                                     "true_rel_residual": info8["true_rel_residual"],
                                     "max_rel_diff_vs_one_by_one": same_solve}
    return out


def run_batch16(lfmm, steps=3):
    """The whole batching configuration: 16 geometries of uneven size (N from 4k to 128k,
    2-4 layers, k in [2, 12]), each with its 32 incidence angles as a block right-hand side.
    One block matvec per geometry with its own launches, against all 16 in shared launches
    (lfmm_matvec_batch: one launch per stage for all geometries), in complex128 and
    complex64 vectors; every geometry's fused result must equal its own launches' bit for bit.
    The precision form (tensor-core M2L for the 32 columns) runs per geometry, with its
    difference from FP64 per geometry."""
    import torch

    from workloads import config_c4

    wls = config_c4()
    t0 = time.perf_counter()
    Gs, Bs = [], []
    for wl in wls:
        med = wl.medium
        M = lfmm.medium_create(med.interfaces, med.k, med.eta)
        pts, w, nrm = lfmm.polygon_elements(wl.bodies)
        G = lfmm.geometry_build(M, pts, w, nrm, p=wl.p, leaf_size=wl.leaf_size)
        Gs.append(G)
        Bs.append(lfmm.rhs_plane_wave(G, np.radians(wl.angles_deg), device=True))
    setup_s = time.perf_counter() - t0
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        tot = []
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            tot.append(e0.elapsed_time(e1))
        return float(np.median(tot)) * 1e-3

    Y1 = [torch.empty_like(b) for b in Bs]
    t_own = timed(lambda: [lfmm.matvec(G, b, y) for G, b, y in zip(Gs, Bs, Y1)])
    Y2 = [torch.empty_like(b) for b in Bs]
    t_fused = timed(lambda: lfmm.matvec_batch(Gs, Bs, Y2))
    same = all(bool(torch.equal(a, b)) for a, b in zip(Y1, Y2))
    B32 = [b.to(torch.complex64) for b in Bs]
    Y32 = [torch.empty_like(b) for b in B32]
    t_fused32 = timed(lambda: lfmm.matvec_batch(Gs, B32, Y32))
    Ym = [torch.empty_like(b) for b in Bs]
    t_mixed = timed(lambda: [lfmm.matvec(G, b, y, mixed=True) for G, b, y in zip(Gs, Bs, Ym)])
    diffs = [max(float(torch.linalg.norm(m[c] - y[c]) / torch.linalg.norm(y[c])) for c in range(m.shape[0]))
             for m, y in zip(Ym, Y1)]
    work = sum(G.n * b.shape[0] for G, b in zip(Gs, Bs))
    out = {"metric": "block right-hand side matvec over 16 uneven geometries, Mpts*rhs/s",
           "workload": f"16 geometries, N {min(G.n for G in Gs)}..{max(G.n for G in Gs)} (total "
                       f"{sum(G.n for G in Gs)}), 2-4 layers, 32 incidence angles each",
           "setup_seconds": setup_s,
           "own_launches_value": work / t_own / 1e6, "own_launches_ms": t_own * 1e3,
           "fused_value": work / t_fused / 1e6, "fused_ms": t_fused * 1e3,
           "fused_complex64_value": work / t_fused32 / 1e6, "fused_complex64_ms": t_fused32 * 1e3,
           "fused_equals_own_launches_bitwise": same,
           "mixed_tensor_core_value": work / t_mixed / 1e6, "mixed_tensor_core_ms": t_mixed * 1e3,
           "mixed_vs_fp64_max_rel_diff_per_geometry": diffs}
    for G in Gs:
        G.destroy()
    return out


# the paper's Tables 5.1-5.3 (Sec. 5): elements, GMRES iterations without / with the DD
# preconditioner, and for Example 1 the L_inf error column (CPU times on unstated hardware
# are context only and not compared)
PAPER_TABLES = {
    "E1": {"elements": [12000, 24000, 48000, 96000, 192000], "iters": [140, 163, 190, 278, 331],
           "iters_pc": [60, 68, 77, 86, 99], "linf": [2.282e-02, 1.151e-02, 5.782e-03, 2.897e-03, 1.450e-03]},
    "E2": {"elements": [12000, 24000, 48000, 96000, 192000], "iters": [93, 104, 115, 132, 162],
           "iters_pc": [59, 66, 72, 81, 93]},
    "E3": {"elements": [12000, 24000, 48000, 96000, 192000], "iters": [125, 138, 156, 173, 192],
           "iters_pc": [71, 79, 88, 101, 112]},
}


def run_replay(sizes=(12000, 24000, 48000, 96000, 192000)):
    """Examples 1-3 of Sec. 5 as GPU solves (FP64, p = 20, tol 1e-8): iterations with and
    without the DD preconditioner, solve seconds, and for Example 1 the error of the
    manufactured solution u^s = G(r, r') (source r' = (0, 0.375) inside the L-shape)."""
    from paper_2511_12450_gb300 import lfmm
    from workloads import example1, example2, example3

    out = {}
    for name, make in (("E1", example1), ("E2", example2), ("E3", example3)):
        rows = []
        for n in sizes:
            wl = make(n)
            med = wl.medium
            M = lfmm.medium_create(med.interfaces, med.k, med.eta)
            pts, w, nrm = lfmm.polygon_elements(wl.bodies)
            t0 = time.perf_counter()
            G = lfmm.geometry_build(M, pts, w, nrm, p=20, leaf_size=64)
            setup = time.perf_counter() - t0
            row = {"elements": int(pts.shape[0]), "setup_s": setup}
            if name == "E1":
                # exact solution: the field of a unit element at the source point, G(r, r')
                src = np.array([wl.extra["source"]], dtype=np.float64)
                Gs = lfmm.geometry_build(M, src, np.ones(1), p=20, leaf_size=64)
                one = np.ones(1, dtype=np.complex128)
                lay = np.searchsorted(-np.asarray(med.interfaces, dtype=float), -pts[:, 1], side="left")
                b = np.asarray(med.eta, dtype=float)[lay] * lfmm.eval_field(Gs, one, pts)
                th = np.linspace(0.0, 2.0 * np.pi, 400, endpoint=False)
                tg = np.stack([0.75 + 2.6 * np.cos(th), -0.875 + 2.6 * np.sin(th)], axis=1)
                keep = np.min(np.abs(tg[:, 1:2] - np.asarray(med.interfaces, dtype=float)[None, :]), axis=1) > 1e-3
                tg = tg[keep]
                exact = lfmm.eval_field(Gs, one, tg)
            else:
                b = lfmm.rhs_plane_wave(G, [math.radians(float(wl.angles_deg[0]))])
            for pc in (False, True):
                x, info = lfmm.gmres_solve(G, b, tol=1e-8, max_iter=1000, precond=pc)
                key = "pc" if pc else "plain"
                row["iters_" + key] = info["iterations"]
                row["solve_s_" + key] = info["solve_seconds"]
                row["true_rel_residual_" + key] = info["true_rel_residual"]
                if name == "E1" and pc:
                    u = lfmm.eval_field(G, x, tg)
                    row["linf_error"] = float(np.max(np.abs(u - exact)))
                    row["l2_rel_error"] = float(np.linalg.norm(u - exact) / np.linalg.norm(exact))
            rows.append(row)
            print(name, row, file=sys.stderr, flush=True)
        out[name] = {"ours": rows, "paper": PAPER_TABLES[name]}
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    wl, desc = workload(args.workload)
    frac = 0.25 if args.workload == "c2" else 1.0
    for _ in range(args.warmup):
        cpu_baseline(wl, min(frac, 0.02))
    res = cpu_baseline(wl, frac, n_samples=args.steps)
    n = wl.n_elements
    line = {
        "impl": "reference",
        "metric": "FMM matvec Mpts/s", "value": res["value"], "unit": "Mpts/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * res["seconds"] / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": desc, "N": n},
        "cpu_baseline": {k: res[k] for k in ("value", "unit", "cores", "kind", "sample")},
        "e2e": {"value": res["value"], "unit": "Mpts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_ours(args):
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    from paper_2511_12450_gb300 import lfmm

    wl, desc = workload(args.workload)
    med = wl.medium
    M = lfmm.medium_create(med.interfaces, med.k, med.eta)
    pts, w, nrm = lfmm.polygon_elements(wl.bodies)
    n = pts.shape[0]
    t0 = time.perf_counter()
    G = lfmm.geometry_build(M, pts, w, nrm, p=wl.p, leaf_size=wl.leaf_size, profile=True,
                            autotune=bool(args.autotune))
    setup_s = time.perf_counter() - t0
    work = algorithmic_work(lfmm, G, n)
    gen = torch.Generator(device="cpu").manual_seed(1234 + rank)
    x = torch.complex(torch.randn(n, generator=gen, dtype=torch.float64),
                      torch.randn(n, generator=gen, dtype=torch.float64)).cuda()
    y = torch.empty_like(x)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        lfmm.matvec(G, x, y)
    torch.cuda.synchronize()
    st0 = lfmm.stage_times(G)
    nl0 = float(lfmm.geometry_query(G, "launch_count", np.float64)[0])
    clocks = Clocks(local)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    times = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lfmm.matvec(G, x, y)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    st1 = lfmm.stage_times(G)
    launches = int(round(float(lfmm.geometry_query(G, "launch_count", np.float64)[0]) - nl0))
    value, slowest_s = whole_job_throughput(float(np.sum(times)) * 1e-3, n * args.steps, dist, "cuda")
    total_ms = slowest_s * 1e3
    stages = {k: {"count": st1[k]["count"] - st0[k]["count"], "ms": st1[k]["ms"] - st0[k]["ms"]} for k in st1}

    # end to end through the C ABI with host (pinned) buffers: H2D + matvec + D2H per step
    xh = torch.empty(n, dtype=torch.complex128).pin_memory()
    yh = torch.empty(n, dtype=torch.complex128).pin_memory()
    xh.copy_(x.cpu())
    xa, ya = xh.numpy(), yh.numpy()
    for _ in range(2):
        lfmm.matvec(G, xa, ya)
    e2e_times = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        lfmm.matvec(G, xa, ya)
        e2e_times.append(time.perf_counter() - t1)
    e2e_value, _ = whole_job_throughput(float(np.sum(e2e_times)), n * args.steps, dist, "cuda")
    assert np.allclose(ya, y.cpu().numpy(), rtol=1e-12, atol=1e-12 * float(np.abs(ya).max()))

    # roofline of the dominant stage
    peaks, src = measured_peaks()
    dom = max(("m2l", "near"), key=lambda k: stages[k]["ms"])
    if dom == "m2l":
        avg_s = stages["m2l"]["ms"] / max(stages["m2l"]["count"], 1) * 1e-3
        achieved = work["m2l_flops"] / avg_s / 1e12
        roof = {"kernel": "k_m2l", "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                "traffic": NCU_TRAFFIC_BYTES.get("k_m2l"),
                "peak_source": "FP64 from unit counts x clock (152 SMs x 2 DFMA/clk x 2.07 GHz)"}
    else:
        avg_s = stages["near"]["ms"] / max(stages["near"]["count"], 1) * 1e-3
        peak = float(peaks.get("hbm_gbs", HBM_FALLBACK_GBS))
        achieved = work["near_bytes"] / avg_s / 1e9
        roof = {"kernel": "k_near_leaf", "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": NCU_TRAFFIC_BYTES.get("k_near_leaf"), "peak_source": src}

    # precision form: the same matvec with FP32 multipole-to-local translations
    ym = torch.empty_like(x)
    for _ in range(args.warmup):
        lfmm.matvec(G, x, ym, mixed=True)
    torch.cuda.synchronize()
    stm0 = lfmm.stage_times(G)
    mtimes = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lfmm.matvec(G, x, ym, mixed=True)
        e1.record(stream)
        e1.synchronize()
        mtimes.append(e0.elapsed_time(e1))
    mixed_value, mixed_s = whole_job_throughput(float(np.sum(mtimes)) * 1e-3, n * args.steps, dist, "cuda")
    mixed = {"metric": "FMM matvec Mpts/s, precision form (FP32 far field on scaled expansions, complex64 "
                       "regular near field)",
             "value": mixed_value, "ms_per_step": mixed_s * 1e3 / args.steps,
             "op_rel_diff": float(torch.linalg.norm(ym - y) / torch.linalg.norm(y))}
    pf = lfmm.geometry_query(G, "precision_form", np.float64)
    mixed["fp32_from_level"] = int(pf[0])
    mixed["coarse_m2l"] = "double-float" if pf[1] == 1 else "FP64"
    # the precision form's near field against HBM: complex64 regular blocks, FP64 reaction
    # blocks, the FP64 diagonal, x in FP64 and complex64, y read and written
    ne = lfmm.geometry_query(G, "near_entries", np.float64)
    near32_bytes = 8.0 * ne[1] + 16.0 * ne[2] + (16.0 + 16.0 + 8.0 + 32.0) * n
    stm1 = lfmm.stage_times(G)
    mixed["stages_ms_per_step"] = {k: (stm1[k]["ms"] - stm0[k]["ms"]) / max(stm1[k]["count"] - stm0[k]["count"], 1)
                                   for k in stm1}
    near_s = mixed["stages_ms_per_step"]["near"] * 1e-3
    peaks_m, src_m = measured_peaks()
    hbm = float(peaks_m.get("hbm_gbs", HBM_FALLBACK_GBS))
    mixed["near_roofline"] = {"kernel": "k_near_leaf (precision form)", "bound": "hbm",
                              "achieved": near32_bytes / near_s / 1e9 if near_s > 0 else None, "peak": hbm,
                              "unit": "GB/s",
                              "frac": (near32_bytes / near_s / 1e9 / hbm) if near_s > 0 else None,
                              "peak_source": src_m, "traffic": NCU_TRAFFIC_BYTES.get("k_near_leaf (precision form)"),
                              "note": "timed inside the matvec, beside the far field"}
    mixed["near_entries_complex64"] = int(ne[1])
    mixed["near_entries_fp64"] = int(ne[2])
    mixed["near_bytes_per_launch"] = near32_bytes

    solve = None
    if not args.no_solve:
        b = lfmm.rhs_plane_wave(G, [math.radians(float(wl.angles_deg[0]))], device=True)
        xs, info = lfmm.gmres_solve(G, b, tol=1e-8, max_iter=1000, precond=True)
        solve = {"metric": "GMRES solve s @1e-8 resid", "seconds": info["solve_seconds"],
                 "iterations": info["iterations"], "true_rel_residual": info["true_rel_residual"],
                 "converged": bool(info["converged"]), "precond": "overlapping DD (Sec. 4.2)",
                 "setup_seconds": setup_s}
        xm, im = lfmm.gmres_solve(G, b, tol=1e-8, max_iter=1000, precond=True, precision=1)
        mixed["solve"] = {"metric": "GMRES solve s @1e-8 resid (FP64 residual), relaxed mixed precision",
                          "seconds": im["solve_seconds"], "iterations": im["iterations"],
                          "refinements": im["refinements"], "fp64_matvecs": im["fp64_matvecs"],
                          "true_rel_residual": im["true_rel_residual"],
                          "converged": bool(im["converged"]), "op_rel_diff_on_b": im["op_rel_diff"],
                          "rel_diff_to_fp64_solution": float(torch.linalg.norm(xm - xs) / torch.linalg.norm(xs))}

    combined = None
    if not args.no_solve:
        combined = run_combined(lfmm, wl, M, pts, w, nrm, x, flush, stream, args, dist, n)

    c3 = None
    if rank == 0 and not args.no_c3 and args.workload == "c2":
        c3 = run_c3(lfmm)
    batch = None
    if rank == 0 and not args.no_batch and args.workload == "c2":
        batch = run_batch(lfmm)
        batch["all_16_geometries"] = run_batch16(lfmm)
    serve = None
    if rank == 0 and not args.no_serve and args.workload == "c2":
        serve = run_serving(lfmm)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(wl, 1 if args.workload == "c2" else 1.0)
        cpu.pop("seconds", None)
    if rank == 0:
        line = {
            "metric": "FMM matvec Mpts/s", "value": value, "unit": "Mpts/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": desc, "N": n, "p": wl.p, "leaf_size": wl.leaf_size,
                       "l2": "flushed (512 MB write) before every step",
                       "parallelism": f"{world} independent replica(s), one per GPU"},
            "e2e": {"value": e2e_value, "unit": "Mpts/s", "h2d_bytes_per_step": 16 * n,
                    "d2h_bytes_per_step": 16 * n},
            "gpu_launches": launches,
            "roofline": roof,
            "cpu_baseline": cpu,
            "clocks": clk,
            "stages_ms_per_step": {k: v["ms"] / max(v["count"], 1) for k, v in stages.items()},
            "work": work,
            "solve": solve,
            "mixed": mixed,
            "combined_field": combined,
            "c3": c3,
            "batch": batch,
            "serve": serve,
            "setup_seconds": setup_s,
            "setup": setup_report(lfmm, G, setup_s),
            "m2l_schedule": lfmm.tuning(G),
        }
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.replay:
        sizes = tuple(n for n in (12000, 24000, 48000, 96000, 192000) if n <= args.replay_max)
        print(json.dumps({"replay": run_replay(sizes), "data": "synthetic (the paper's geometries and media)",
                          "dtype": "f64"}))
        return 0
    if args.impl == "reference":
        return run_reference(args)
    if args.serve_full > 0:
        import torch

        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        from paper_2511_12450_gb300 import lfmm

        print(json.dumps({"serve": run_serving(lfmm, n_requests=args.serve_full, n_max=262144.0, max_bodies=512),
                          "data": "synthetic", "dtype": "f64"}))
        return 0
    if args.only_batch:
        import torch

        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        from paper_2511_12450_gb300 import lfmm

        print(json.dumps({"batch": run_batch(lfmm, steps=args.steps, solve=not args.no_solve), "data": "synthetic",
                          "dtype": "f64"}))
        return 0
    if args.only_c3:
        import torch

        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        from paper_2511_12450_gb300 import lfmm

        print(json.dumps({"c3": run_c3(lfmm, steps=args.steps), "data": "synthetic", "dtype": "f64"}))
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
