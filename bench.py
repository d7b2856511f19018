#!/usr/bin/env python
"""Benchmark: PLSS time to ||b - A x||/||b|| <= 1e-8 on one GB300.

Workload (synthetic, seeded; stands in for the paper's large sparse
SuiteSparse systems): the consistent overdetermined 1,000,000 x 200,000 CSR
with 8 nonzeros per row at uniform columns, values N(0,1) times column scales
10**U(-2, 2) rounded to FP32 once, b = A x*, x0 = 0.

A step is one whole solve (every update of Algorithm 1 until the true
relative residual is <= tol), inputs resident in HBM. The line also carries
the roofline of the dominant sweep (CUDA events recorded on the solve's
stream between the captured kernels of the timed solves), the oracle's time
on the host cores for a bounded sample, and an end-to-end figure through the
C ABI with host buffers.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2207_07615_gb300 import synth  # noqa: E402

WORKLOAD = "plss_overdetermined_1e6x2e5_nnz8_colscale1e-2..1e2"
METRIC = "time to ||r||/||b||<=1e-8"
# Updates the FP64 W = I solve of this workload takes to the tolerance: the
# GPU arm's own count on GB300 (181,143 with the current kernels, the same in
# every run: its reductions have a fixed order). The reference arm runs
# without the GPU arm's result, so it scales its sampled per-update time by
# this count; the GPU arm's own cpu_baseline scales by the count its solve
# just took.
REF_UPDATES_TO_TOL = 181143
L2_FLUSH_BYTES = 512 << 20
PROFILE_PERIOD = 16


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="plss", choices=["plss", "reference"])
    ap.add_argument("--prec", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--w-mode", type=int, default=0)
    ap.add_argument("--layout", default="auto", choices=["auto", "csr"])
    ap.add_argument("--server-layout", default="csr", choices=["auto", "csr"], help="c5: arena layout")
    ap.add_argument("--m", type=int, default=1_000_000)
    ap.add_argument("--n", type=int, default=200_000)
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--maxit", type=int, default=3_000_000)
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--oracle-updates", type=int, default=100)
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the compact lines of the other workloads in the headline run")
    ap.add_argument("--omp-updates", type=int, default=1000,
                    help="updates of the all-cores oracle sample")
    ap.add_argument("--workload", default="c2", choices=["c1", "c2", "c3", "c4a", "c4b", "c5"],
                    help="c2 (default): the headline line; the others print one line each for "
                         "the other synthetic workloads (see suite_* below)")
    ap.add_argument("--requests", type=int, default=1000, help="c5: requests in the trace")
    ap.add_argument("--pool", type=int, default=64, help="c5: matrices in the request pool")
    return ap.parse_args()


# ---------------------------------------------------------------- helpers

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value, dist, device=None):
    """The slowest rank's value (replicas: every rank solves its own copy of
    the workload; the job's time per step is the last one to finish)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def host_info():
    cpu = "unknown"
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part", "hardware")):
                    cpu = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return cpu, os.cpu_count()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def kernels_hash(path):
    """sha256[:16] of the code of the grid-wide sweeps in plss_kernels.cu:
    the file with comments and blank lines removed (a comment edit does not
    invalidate recorded counters), cut to the lines before the cluster
    solver (the sweeps, the update and their helpers) plus the launchers from
    sweep_ctas_per_sm up to the cluster launcher -- everything the C2 sweeps
    and update are built and launched from, and nothing else. The whole
    file's code when those markers are missing."""
    import hashlib
    import re
    text = open(path, encoding="utf-8").read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lines = [re.sub(r"//.*$", "", ln).rstrip() for ln in text.splitlines()]
    lines = [ln for ln in lines if ln.strip()]
    try:
        a = next(i for i, ln in enumerate(lines) if "kClusterCtas" in ln)
        b = next(i for i, ln in enumerate(lines) if "int sweep_ctas_per_sm(int which" in ln)
        c = next(i for i, ln in enumerate(lines)
                 if ln.startswith("cudaError_t launch_cluster_solve("))
        if a < b < c:
            lines = lines[:a] + lines[b:c]
    except StopIteration:
        pass
    return hashlib.sha256("\n".join(lines).encode()).hexdigest()[:16]


def ncu_traffic(kernel):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, or
    None when absent or taken on a different version of the kernel source."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    src = os.path.join(ROOT, "paper_2207_07615_gb300", "csrc", "plss_kernels.cu")
    try:
        kv = {}
        with open(path) as f:
            for line in f:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
        sha = kernels_hash(src)
        if kv.get("kernels_sha256_16") != sha:
            return None
        return float(kv[f"{kernel}_dram_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.tmp, stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.tmp.flush()
        rows = []
        with open(self.tmp.name) as f:
            for line in f:
                p = [s.strip() for s in line.split(",")]
                if len(p) >= 8:
                    rows.append(p)
        os.unlink(self.tmp.name)
        if not rows:
            return None

        def num(s):
            try:
                return float(s)
            except ValueError:
                return float("nan")
        sm = np.array([num(r[0]) for r in rows])
        mx = np.array([num(r[1]) for r in rows])
        pw = np.array([num(r[2]) for r in rows])
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].lower() == "active"})
        load = sm[pw >= np.nanmedian(pw)] if np.isfinite(pw).any() else sm
        return {"sm_mhz": float(np.nanmedian(load if load.size else sm)),
                "sm_max_mhz": float(np.nanmax(mx)), "reasons": reasons,
                "samples": int(len(rows)), "power_w_max": float(np.nanmax(pw))}


def sweep_bytes(kind, m, n, nnz, sv):
    """Algorithmic HBM bytes of one launch (each array touched once)."""
    if kind == "row_sweep":      # CSR (col_idx, val, row_ptr), p gathered once, r read + written
        return nnz * (4 + sv) + (m + 1) * 4 + 2 * m * sv + n * sv
    if kind == "col_sweep":      # CSC (row_idx, val, col_ptr), r gathered once, W y written
        return nnz * (4 + sv) + (n + 1) * 4 + m * sv + n * sv
    if kind == "update":         # p, W y read; p written; x (double) read + written
        return n * (3 * sv + 16)
    raise KeyError(kind)


def gather_reference(torch, A, sv, dev, flush, reps=5):
    """PyTorch's own gather (index_select, library code) over the same index
    streams as the two sweeps: the column indices of A into a vector of n and
    the row indices of A^T into a vector of m, each nnz gathers with the
    indices read and the gathered values written once. Timed alone with CUDA
    events, L2 flushed before each repetition; the median is reported beside
    the sweeps, which do the same gathers plus the values, products, sums and
    vector writes."""
    dt = torch.float64 if sv == 8 else torch.float32
    order = np.argsort(A.col_idx, kind="stable")
    rows = np.repeat(np.arange(A.m, dtype=np.int32), np.diff(A.row_ptr).astype(np.int64))[order]
    out = {}
    for side, idx_np, length in (("row_sweep", A.col_idx, A.n), ("col_sweep", rows, A.m)):
        idx = torch.from_numpy(np.ascontiguousarray(idx_np, dtype=np.int32)).to(dev)
        vec = torch.rand(length, dtype=dt, device=dev)
        dst = torch.empty(idx.numel(), dtype=dt, device=dev)
        ts = []
        for _ in range(reps + 1):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.index_select(vec, 0, idx, out=dst)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) * 1e3)
        us = float(np.median(ts[1:]))
        out[side] = {"us": us, "gathers_per_s": idx.numel() / (us * 1e-6)}
        del idx, vec, dst
    out["kernel"] = "torch.index_select (int32 indices), median of %d" % reps
    return out


def make_workload(args):
    A, b, xs = synth.overdetermined_scaled(m=args.m, n=args.n, per_row=8, seed=1)
    if args.prec == "fp64":
        A = A.astype(np.float64)
    return A, b, xs


def cpu_baseline(A, b, args, updates_to_tol, all_cores=True):
    """The oracle (plain C, 1 thread) on a bounded sample: the time of a
    1-update solve (set-up included) plus the per-update time of the next
    `oracle_updates` updates, scaled to the updates the solve needs; and the
    same source built with OpenMP on every host core, sampled over
    `omp_updates` updates and scaled the same way."""
    import oracle
    oracle.build()
    prec = 1 if args.prec == "fp32" else 0
    w = oracle.colweights(A, args.w_mode) if args.w_mode else None

    def sample(updates, threads):
        t0 = time.perf_counter()
        oracle.residual(A, b, w=w, tol=0.0, maxit=1, prec=prec, threads=threads)
        t1 = time.perf_counter()
        oracle.residual(A, b, w=w, tol=0.0, maxit=1 + updates, prec=prec, threads=threads)
        t2 = time.perf_counter()
        per = ((t2 - t1) - (t1 - t0)) / updates
        return (t1 - t0) + per * max(0, updates_to_tol - 1), t1 - t0, per

    cpu, cores = host_info()
    value, t_setup, per = sample(args.oracle_updates, False)
    out = {"value": value, "unit": "s", "cores": 1, "kind": "oracle",
           "sample": (f"1 update ({t_setup:.2f} s incl. set-up) + {args.oracle_updates} updates "
                      f"({per * 1e3:.1f} ms/update) of the same system, scaled to "
                      f"{updates_to_tol} updates; host {cpu}, {cores} cores, 1 used")}
    if all_cores and prec == 0:
        try:
            v2, s2, p2 = sample(args.omp_updates, True)
            nthreads = int(os.environ.get("OMP_NUM_THREADS", cores or 1))
            out["all_cores"] = {"value": v2, "unit": "s", "cores": nthreads, "kind": "oracle (OpenMP build)",
                                "sample": (f"1 update ({s2:.2f} s) + {args.omp_updates} updates "
                                           f"({p2 * 1e3:.2f} ms/update), scaled to {updates_to_tol} updates")}
        except RuntimeError as e:
            out["all_cores"] = {"unavailable": str(e)}
    return out


# ------------------------------------------------------------ reference arm

def run_config(args, m, n, nnz, ws):
    """The workload's config, the same dict in both arms."""
    sv = 8 if args.prec == "fp64" else 4
    work = (sweep_bytes("row_sweep", m, n, nnz, sv) + sweep_bytes("col_sweep", m, n, nnz, sv)) / 1e6
    return {"workload": WORKLOAD, "m": m, "n": n, "nnz": int(nnz), "tol": args.tol,
            "w_mode": args.w_mode, "precision": args.prec,
            "parallelism": "replicas" if ws > 1 else "single",
            "l2": f"inputs larger than L2 (per-update working set {work:.0f} MB) and a 512 MB write "
                  "between GPU steps"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    if args.workload != "c2":
        print(json.dumps({"impl": "reference", "unavailable": "the oracle arm times the headline "
                          "workload (c2) only"}), flush=True)
        return
    A, b, _ = make_workload(args)
    cpu, cores = host_info()
    t_all = time.perf_counter()
    vals = []
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(A, b, args, REF_UPDATES_TO_TOL, all_cores=False)
        if i >= args.warmup:
            vals.append(cb["value"])
    wall = time.perf_counter() - t_all
    v = float(np.mean(vals))
    line = {"metric": METRIC, "value": v, "unit": "s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": wall / (args.warmup + args.steps) * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.prec == "fp64" else "f32+f64", "data": "synthetic",
            "impl": "reference",
            "config": run_config(args, args.m, args.n, int(A.nnz), ws),
            "cpu_baseline": {"value": v, "unit": "s", "cores": 1, "kind": "oracle",
                             "sample": cb["sample"]},
            "e2e": {"value": v, "unit": "s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm

def run_plss(args):
    import torch
    from paper_2207_07615_gb300 import plss
    import __graft_entry__ as g
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        g.build()
    if dist is not None:
        dist.barrier()
    plss.lib()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    A, b, xs = make_workload(args)
    m, n, nnz = A.m, A.n, A.nnz
    sv = 8 if args.prec == "fp64" else 4
    ctx = plss.Context(A, precision=args.prec, layout=args.layout)
    ctx_layout = dict(ctx.layout(), kind=args.layout)
    b_dev = torch.from_numpy(b).to(dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    kw = dict(tol=args.tol, maxit=args.maxit, stop_on_true=1, w_mode=args.w_mode)

    for _ in range(args.warmup):
        ctx.solve(b_dev, **kw)
        flush.zero_()
    ctx.kernel_times(reset=True)
    clocks = Clocks(local)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    results = []
    for _ in range(args.steps):
        # CUDA events around the kernels of one chunk of updates in every
        # PROFILE_PERIOD (timing every chunk would slow the solve)
        x, r = ctx.solve(b_dev, profile=PROFILE_PERIOD, **kw)
        results.append(r)
        flush.zero_()
    e1.record()
    barrier()
    clk = clocks.stop()
    ms_total = e0.elapsed_time(e1)
    kt = ctx.kernel_times(reset=True)
    ms_step = max_over_ranks(ms_total / args.steps, dist, dev)
    last = results[-1]
    x_np = x.cpu().numpy()
    err_xstar = float(np.linalg.norm(x_np - xs) / np.linalg.norm(xs))

    # roofline of the dominant sweep. CUDA events bracket every kernel of one
    # chunk of updates in PROFILE_PERIOD; an event between two kernels stops
    # the second from starting under the first's tail (programmatic
    # dependent launch), so the event-timed kernels of an update add up to
    # more than an unprofiled update takes. Each kernel's time is therefore
    # its event time scaled by (device time per update of the timed solves,
    # which carry events in 1 chunk of 16) / (sum of the event times of the
    # three kernels): its share of the measured update.
    peaks, peak_src = measured_peaks()
    kinds = ("row_sweep", "col_sweep", "update")
    per = {}
    for k in kinds:
        ms, cnt = kt[k]
        if cnt > 0:
            per[k] = {"ms_total_events": ms, "launches": cnt, "us_per_launch_events": ms / cnt * 1e3,
                      "bytes_per_launch": sweep_bytes(k, m, n, nnz, sv)}
    us_update = ms_step * 1e3 / max(1, last["iters"])
    ev_sum = sum(v["us_per_launch_events"] for v in per.values())
    share = us_update / ev_sum if len(per) == 3 and ev_sum > 0 else 1.0
    for k, v in per.items():
        v["us_per_launch"] = v["us_per_launch_events"] * share
        v["share_of_update"] = v["us_per_launch"] / us_update
        v["gbs"] = v["bytes_per_launch"] / (v["us_per_launch"] * 1e-6) / 1e9
        v["gbs_events"] = v["bytes_per_launch"] / (v["us_per_launch_events"] * 1e-6) / 1e9
        v["ms_total"] = v["us_per_launch"] * v["launches"] * 1e-3
    dom = max(per, key=lambda k: per[k]["ms_total"]) if per else None
    roof = None
    if dom:
        ach = per[dom]["gbs"]
        roof = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": peaks["hbm_gbs"],
                "unit": "GB/s", "frac": ach / peaks["hbm_gbs"],
                "traffic": ncu_traffic(dom), "peak_source": f"{peak_src} hbm_gbs (copy)",
                "algorithmic_bytes_per_launch": per[dom]["bytes_per_launch"],
                "us_per_launch": per[dom]["us_per_launch"],
                "us_per_launch_events": per[dom]["us_per_launch_events"],
                "timing": ("kernel time = its CUDA-event time x (device us per update of the timed "
                           f"solves {us_update:.2f}) / (sum of the three kernels' event times "
                           f"{ev_sum:.2f}): scale {share:.3f}"),
                "sweeps": per}

    if roof is not None and rank == 0:
        gref = gather_reference(torch, A, sv, dev, flush)
        for k in ("row_sweep", "col_sweep"):
            if k in per:
                gref[k]["sweep_us"] = per[k]["us_per_launch"]
                gref[k]["sweep_vs_index_select"] = gref[k]["us"] / per[k]["us_per_launch"]
        roof["gather_reference"] = gref
        # the sweeps' gather floor: the same index streams, grids and warp
        # ranges, gathers only (hand-written kernel in the library)
        gb = {}
        for side, k in ((0, "row_sweep"), (1, "col_sweep")):
            try:
                med, mn = ctx.gather_bound(side, reps=7)
            except plss.PlssError as e:
                gb[k] = {"unavailable": str(e)}
                continue
            gb[k] = {"us": med, "us_min": mn, "gathers_per_s": nnz / (med * 1e-6)}
            if k in per:
                gb[k]["sweep_us"] = per[k]["us_per_launch"]
                gb[k]["bound_over_sweep"] = med / per[k]["us_per_launch"]
                gb[k]["achieved_at_bound_gbs"] = per[k]["bytes_per_launch"] / (med * 1e-6) / 1e9
        gb["kernel"] = "plss_gather_bound (median of 7, L2 evicted, the gathered vector re-read into L2 before each)"
        roof["gather_bound"] = gb

    # end to end through the C ABI with host buffers
    torch.cuda.synchronize()
    te = []
    for _ in range(args.e2e_steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        xh, rh = ctx.solve(b, **kw)
        te.append(time.perf_counter() - t0)
    e2e = None
    if te:
        e2e = {"value": float(np.mean(te)), "unit": "s", "h2d_bytes_per_step": 8 * m,
               "d2h_bytes_per_step": 8 * n}

    variants = {}
    if not args.no_variants and rank == 0:
        variants = run_variants(args, A, b, xs, x_np, ctx, b_dev, flush)

    cb = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(A, b, args, last["iters"])

    extras = None
    if rank == 0 and ws == 1 and not args.no_extras:
        extras = run_extras(args)

    if rank == 0:
        line = {"metric": METRIC, "value": ms_step / 1e3, "unit": "s", "n_gpus": ws,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
                "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if args.prec == "fp64" else "f32+f64", "data": "synthetic",
                "config": run_config(args, m, n, int(nnz), ws),
                "solve": {"updates": last["iters"], "status": last["status"],
                          "relres_true": last["relres_true"], "relres_rec": last["relres_rec"],
                          "ms_per_update": ms_step / max(1, last["iters"]),
                          "rel_err_vs_xstar": err_xstar},
                "layout": ctx_layout, "roofline": roof, "cpu_baseline": cb, "e2e": e2e,
                "gpu_launches": int(kt["all_launches"]), "clocks": clk, "variants": variants,
                "workloads": extras}
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()


def run_variants(args, A, b, xs, x_ref, ctx, b_dev, flush):
    """One solve each of the other forms on the same system: PLSS W
    (W = diag(1/||A_j||^2) and diag(1/||A_j||), Sec. 4.1) and FP32 storage
    with FP64 refinement; error against the FP64 W = I answer."""
    import torch
    from paper_2207_07615_gb300 import plss
    out = {}

    def timed(c, bb, **kw):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        x, r = c.solve(bb, **kw)
        e1.record()
        torch.cuda.synchronize()
        xn = x.cpu().numpy()
        return {"seconds": e0.elapsed_time(e1) / 1e3, "updates": r["iters"], "status": r["status"],
                "relres_true": r["relres_true"],
                "rel_err_vs_fp64": float(np.linalg.norm(xn - x_ref) / np.linalg.norm(x_ref)),
                "rel_err_vs_xstar": float(np.linalg.norm(xn - xs) / np.linalg.norm(xs))}
    base = dict(tol=args.tol, maxit=args.maxit, stop_on_true=1)
    if args.prec == "fp64":
        out["fp64_w2"] = timed(ctx, b_dev, w_mode=2, **base)
        out["fp64_w1"] = timed(ctx, b_dev, w_mode=1, **base)
        c32 = plss.Context(A, precision="fp32")
        out["fp32_w2"] = timed(c32, b_dev, w_mode=2, **base)
        out["fp32_w1"] = timed(c32, b_dev, w_mode=1, **base)
        # W = I in FP32 storage: refinement by residual replacement every 100
        # updates (restarts stall on this system: the float recursion loses
        # its Krylov space at every restart), and the restart schedule beside it
        out["fp32_w0"] = timed(c32, b_dev, w_mode=0, refine_mode="replace", refine_period=100, inner_tol=0.0,
                               **dict(base, maxit=min(args.maxit, 400000)))
        out["fp32_w0_restarts"] = timed(c32, b_dev, w_mode=0, **dict(base, maxit=min(args.maxit, 200000)))
        c32.close()
    return out


# ------------------------------------------------------- other workloads
#
# One JSON line per workload, same clocks and device-timing rules as the
# headline: inputs resident in HBM (device buffers), CUDA events on the
# solve's stream, W warm-up solves. They cover the identity sketch (c3), the
# batched and many-right-hand-side forms (c4a, c4b) and serving (c5).

def _suite_common(args):
    import torch
    import __graft_entry__ as g
    from paper_2207_07615_gb300 import plss
    g.build()
    plss.lib()
    torch.cuda.set_device(0)
    return torch, plss


def _timed(torch, fn, warmup, steps):
    """Runs fn() warmup times, then steps times between CUDA events on the
    current stream; returns (seconds per step, last result)."""
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    out = None
    for _ in range(warmup):
        out = fn()
        flush.zero_()
    torch.cuda.synchronize()
    clocks = Clocks(0)
    tot = 0.0
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        out = fn()
        e1.record()
        torch.cuda.synchronize()
        tot += e0.elapsed_time(e1) / 1e3
    return tot / steps, out, clocks.stop()


def _line(metric, value, unit, args, workload, extra, hib=False, dtype="f32+f64"):
    line = {"metric": metric, "value": value, "unit": unit, "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": value * 1e3 if unit == "s" and value is not None else None,
            "higher_is_better": hib, "scaling": "weak", "vs_baseline": None, "dtype": dtype,
            "data": "synthetic", "config": {"workload": workload}}
    line.update(extra)
    print(json.dumps(line), flush=True)


def suite_c1(args):
    """2,000 x 2,000 diagonally dominant, FP64, tol 1e-10 (L2-resident,
    latency-bound: time per update rather than GB/s)."""
    torch, plss = _suite_common(args)
    import oracle
    A, b, xs = synth.square_diag_dominant()
    A = A.astype(np.float64)
    ctx = plss.Context(A)
    bd = torch.from_numpy(b).cuda()
    t, (x, r), clk = _timed(torch, lambda: ctx.solve(bd, tol=1e-10, maxit=2000, stop_on_true=1),
                            args.warmup, args.steps)
    oracle.build()
    t0 = time.perf_counter()
    ref = oracle.residual(A, b, tol=1e-10, maxit=2000)
    tcpu = time.perf_counter() - t0
    err = float(np.linalg.norm(x.cpu().numpy() - ref["x"]) / np.linalg.norm(ref["x"]))
    _line("time to ||r||/||b||<=1e-10", t, "s", args, "plss_square_2000_diagdom_nnz11", {
        "dtype": "f64",
        "solve": {"updates": r["iters"], "status": r["status"], "relres_true": r["relres_true"],
                  "us_per_update": t / max(1, r["iters"]) * 1e6, "rel_err_vs_oracle": err},
        "cpu_baseline": {"value": tcpu, "unit": "s", "cores": 1, "kind": "oracle",
                         "sample": f"the whole solve ({ref['iters']} updates)"},
        "clocks": clk})
    ctx.close()


def suite_c3(args):
    """100,000 x 1,000,000, power-law rows (mean 20, max 5,000), U(-1,1) in
    FP32: residual sketch (FP32 storage and FP64) and identity sketch."""
    torch, plss = _suite_common(args)
    A, b, xs = synth.powerlaw_underdetermined()
    bd = torch.from_numpy(b).cuda()
    out = {}
    for prec in ("fp32", "fp64"):
        Ap = A if prec == "fp32" else A.astype(np.float64)
        ctx = plss.Context(Ap, precision=prec)
        for w in (0, 2):
            t, (x, r), clk = _timed(torch, lambda: ctx.solve(bd, tol=1e-8, maxit=min(200000, args.maxit),
                                                             stop_on_true=1,
                                                             w_mode=w), 1, 1)
            out[f"residual_{prec}_w{w}"] = {"seconds": t, "updates": r["iters"], "status": r["status"],
                                            "relres_true": r["relres_true"],
                                            "us_per_update": t / max(1, r["iters"]) * 1e6}
        out[f"layout_{prec}"] = ctx.layout()
        ctx.close()
    ctx = plss.Context(A, precision="fp64")
    for K in (0, 8):
        t, (x, r), clk = _timed(torch, lambda: ctx.solve(bd, sketch="identity", tol=1e-8,
                                                         maxit=min(10 * A.m, args.maxit), kacz_hist=K, seed=7), 1, 1)
        out[f"identity_K{K}"] = {"seconds": t, "rows_visited": r["iters"], "status": r["status"],
                                 "relres_true": r["relres_true"],
                                 "passes": r["iters"] / A.m}
    ctx.close()
    conv = [v["seconds"] for k, v in out.items() if k.startswith(("residual", "identity"))
            and v["status"] == "converged"]
    _line("time to ||r||/||b||<=1e-8", min(conv) if conv else None, "s", args,
          "plss_underdetermined_1e5x1e6_zipf20_max5000",
          {"forms": out, "clocks": clk, "value_is": "fastest converged form (null: none within the caps)"})


def suite_c4a(args):
    """256 independent systems (m log-uniform [1e3, 2e5], n = m or m/2, 5-50
    nonzeros per row, N(0,1) in FP32) in one batched context."""
    torch, plss = _suite_common(args)
    systems = synth.batched_systems()
    As = [A for A, _, _ in systems]
    bs = [torch.from_numpy(b).cuda() for _, b, _ in systems]
    nnz = sum(A.nnz for A in As)
    out = {}
    for prec in ("fp32", "fp64"):
        Ap = As if prec == "fp32" else [A.astype(np.float64) for A in As]
        # plan chosen by the autotuner on every 8th system (32 of 256, the
        # whole size range), outside the timed region
        t0 = time.perf_counter()
        best, table = plss.tune(Ap[::8], updates=10, precision=prec, w_mode=2)
        tune_s = time.perf_counter() - t0
        ctx = plss.Context(Ap, precision=prec, layout=best["layout"], tile_shift=best["tile_shift"])
        t, (xs_, rs), clk = _timed(torch, lambda: ctx.solve_batched(bs, tol=1e-8, maxit=min(5000, args.maxit),
                                                                    stop_on_true=1, w_mode=2,
                                                                    schedule=best["schedule"]),
                                   args.warmup, args.steps)
        ups = sum(r["iters"] for r in rs)
        out[prec] = {"seconds": t, "converged": sum(r["status"] == "converged" for r in rs),
                     "systems": len(rs), "system_updates": ups, "max_updates": max(r["iters"] for r in rs),
                     "worst_relres_true": max(r["relres_true"] for r in rs),
                     "plan": dict(best, tuned_on_systems=len(Ap[::8]), tune_seconds=tune_s, candidates=table)}
        ctx.close()
    _line("time to ||r||/||b||<=1e-8 (all systems)", out["fp32"]["seconds"], "s", args,
          "plss_batched_256_systems", {"forms": out, "nnz_total": int(nnz), "w_mode": 2, "maxit": 5000,
                                       "clocks": clk})


def suite_c4b(args):
    """7-point Laplacian on 126^3 with 32 right-hand sides (SpMM sweeps),
    FP32 storage with FP64 refinement, tol 1e-8."""
    torch, plss = _suite_common(args)
    A = synth.laplacian7()
    B, Xs = synth.laplacian_rhs(A)
    Bd = torch.from_numpy(B).cuda()
    out = {}
    for prec in ("fp32", "fp64"):
        ctx = plss.Context(A if prec == "fp32" else A.astype(np.float64), precision=prec, symmetric=True)
        t, (X, rs), clk = _timed(torch, lambda: ctx.solve_rhs(Bd, tol=1e-8, maxit=min(50000, args.maxit),
                                                              stop_on_true=1),
                                 1, 1)
        Xh = X.cpu().numpy()
        out[prec] = {"seconds": t, "converged": sum(r["status"] == "converged" for r in rs),
                     "max_updates": max(r["iters"] for r in rs),
                     "worst_relres_true": max(r["relres_true"] for r in rs),
                     "rel_err_vs_xstar": float(np.linalg.norm(Xh - Xs) / np.linalg.norm(Xs))}
        ctx.close()
    _line("time to ||r||/||b||<=1e-8 (32 right-hand sides)", out["fp32"]["seconds"], "s", args,
          "plss_laplacian7_126cube_32rhs", {"forms": out, "nnz": int(A.nnz), "clocks": clk})


def suite_c5(args):
    """Open-loop Poisson arrivals (2,000 requests/s) of random sparse
    consistent systems (m log-uniform [1e3, 1e6], n/m in {0.5, 1, 2}, 8-32
    nonzeros per row, N(0,1)) into the continuous-batching server, FP32 with
    FP64 refinement, W = diag(1/||A_j||), tol 1e-6, maxit 3,000. Latency is
    completion minus arrival and includes the host-side preparation and the
    upload. Eight client threads submit (plss_submit prepares the request on
    the calling thread), each taking every eighth request at its arrival
    time."""
    torch, plss = _suite_common(args)
    arrivals, reqs = serving_requests(args.requests, args.pool)
    res = serve(plss, reqs, arrivals, maxit=min(3000, args.maxit), layout=args.server_layout)
    _line("served solves/s", res["solves_per_s"], "solves/s", args, "plss_serving_poisson2000", dict(
        res, higher_is_better=True, steps=1, warmup=0, ms_per_step=None, pool=args.pool,
        server_layout=args.server_layout))


# ------------------------------------------------ extras in the headline run
#
# Compact results of the other workloads, carried by the headline line
# (`workloads`), each with its own clock record: the latency-bound square
# system (C1), 32 right-hand sides (C4b, FP32 storage), serving at the
# configured arrival rate and below capacity (C5, a shortened trace), and
# the identity sketch with a whole-GPU history window on the power-law
# system (C3).

def extra_c1(torch, plss, warmup=3, steps=10):
    import oracle
    A, b, xs = synth.square_diag_dominant()
    A = A.astype(np.float64)
    ctx = plss.Context(A)
    bd = torch.from_numpy(b).cuda()
    t, (x, r), clk = _timed(torch, lambda: ctx.solve(bd, tol=1e-10, maxit=2000, stop_on_true=1), warmup, steps)
    ctx.close()
    ref = oracle.residual(A, b, tol=1e-10, maxit=2000)
    return {"metric": "time to ||r||/||b||<=1e-10", "seconds": t, "updates": r["iters"],
            "status": r["status"], "relres_true": r["relres_true"],
            "us_per_update": t / max(1, r["iters"]) * 1e6, "oracle_updates": ref["iters"],
            "rel_err_vs_oracle": float(np.linalg.norm(x.cpu().numpy() - ref["x"]) / np.linalg.norm(ref["x"])),
            "steps": steps, "warmup": warmup, "clocks": clk}


def extra_c4b(torch, plss):
    A = synth.laplacian7()
    B, Xs = synth.laplacian_rhs(A)
    Bd = torch.from_numpy(B).cuda()
    ctx = plss.Context(A, precision="fp32", symmetric=True)
    t, (X, rs), clk = _timed(torch, lambda: ctx.solve_rhs(Bd, tol=1e-8, maxit=50000, stop_on_true=1), 1, 1)
    ctx.close()
    Xh = X.cpu().numpy()
    ups = max(r["iters"] for r in rs)
    return {"metric": "time to ||r||/||b||<=1e-8 (32 right-hand sides)", "seconds": t,
            "precision": "fp32 storage + fp64 refinement",
            "converged": sum(r["status"] == "converged" for r in rs), "max_updates": ups,
            "ms_per_update": t / max(1, ups) * 1e3,
            "worst_relres_true": max(r["relres_true"] for r in rs),
            "rel_err_vs_xstar": float(np.linalg.norm(Xh - Xs) / np.linalg.norm(Xs)), "clocks": clk}


def serve(plss, reqs, arrivals, maxit=3000, layout="csr", nthreads=8):
    """Replays requests (A, b) at the given arrival times through the
    continuous-batching server (plss_submit / plss_poll); latency is
    completion minus arrival, host-side preparation and upload included."""
    import threading
    srv = plss.Server(max_slots=64, precision="fp32", layout=layout)
    done = {}
    t0 = time.perf_counter()
    tickets = [None] * len(reqs)
    submit_s = [0.0] * len(reqs)
    busy = [0]

    def submitter(k):
        for i in range(k, len(reqs), nthreads):
            A, b = reqs[i]
            while time.perf_counter() - t0 < arrivals[i]:
                time.sleep(0.0002)
            ts = time.perf_counter()
            t = None
            while t is None:
                t = srv.submit(A, b, tol=1e-6, maxit=maxit, w_mode=1)
                if t is None:
                    busy[0] += 1
                    time.sleep(0.001)
            submit_s[i] = time.perf_counter() - ts
            tickets[i] = t

    ths = [threading.Thread(target=submitter, args=(k,)) for k in range(nthreads)]
    clocks = Clocks(0)
    for th in ths:
        th.start()
    pending = set(range(len(reqs)))
    while pending:
        for i in list(pending):
            t = tickets[i]
            if t is None:
                continue
            r = srv.poll(t)
            if r is not None:
                done[i] = (time.perf_counter() - t0, r[1])
                pending.discard(i)
        time.sleep(0.002)
    for th in ths:
        th.join()
    clk = clocks.stop()
    srv.close()
    lat = np.array([done[i][0] - arrivals[i] for i in range(len(reqs))])
    span = max(v[0] for v in done.values())
    return {"solves_per_s": len(reqs) / span,
            "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                          "mean": float(lat.mean()), "max": float(lat.max())},
            "offered_per_s": float(len(reqs) / max(arrivals[-1], 1e-9)), "requests": len(reqs),
            "converged": int(sum(v[1]["status"] == "converged" for v in done.values())),
            "makespan_s": span, "client_threads": nthreads, "busy_retries": busy[0],
            "submit_s_max": float(max(submit_s)), "clocks": clk}


def serving_requests(nreq, pool, rate=2000.0):
    arrivals, pool_ids, mats = synth.serving_trace(nreq=nreq, pool=pool, rate=rate)
    reqs = []
    for i, pid in enumerate(pool_ids):
        A = mats[int(pid)]
        xs = synth.rng_for(3000 + 1_000_000 + i).standard_normal(A.n)
        reqs.append((A, synth.rhs(A, xs)))
    return arrivals, reqs


def extra_c5(plss, nreq=200, pool=16):
    """The configured arrival rate (2,000/s, far above what the GPU serves),
    then the same requests at 0.9x and 0.5x of the service rate measured
    there, so that p50/p99 show the server rather than the queue."""
    arrivals, reqs = serving_requests(nreq, pool)
    out = {"rate_2000": serve(plss, reqs, arrivals)}
    cap = out["rate_2000"]["solves_per_s"]
    for f in (0.9, 0.5):
        gaps = np.diff(np.concatenate([[0.0], arrivals]))
        arr = np.cumsum(gaps * (2000.0 / (f * cap)))      # the same Poisson gaps, stretched
        out[f"load_{f}"] = serve(plss, reqs, arr)
    out["trace"] = (f"{nreq} requests over a pool of {pool} matrices (the configuration's trace: "
                    "10,000 over 256); arrival gaps of the 2,000/s trace stretched for the lower loads")
    return out


def extra_c3_identity(torch, plss, rows=50000):
    """Identity sketch on the 1e5 x 1e6 power-law system: windows of 0, 8 and
    256 directions (256 runs on the whole GPU), a fixed number of rows."""
    A, b, xs = synth.powerlaw_underdetermined()
    bd = torch.from_numpy(b).cuda()
    ctx = plss.Context(A, precision="fp64")
    out = {}
    for K in (0, 8, 256):
        t, (x, r), clk = _timed(torch, lambda: ctx.solve(bd, sketch="identity", tol=0.0, maxit=rows,
                                                         kacz_hist=K, seed=7), 1, 1)
        out[f"K{K}"] = {"seconds": t, "rows": r["iters"], "us_per_row": t / max(1, r["iters"]) * 1e6,
                        "relres_true": r["relres_true"], "clocks": clk}
    ctx.close()
    out["workload"] = f"plss_underdetermined_1e5x1e6_zipf20_max5000, {rows} rows (half a pass), tol 0"
    return out


def extra_general(torch, plss, cols=300, K=64):
    """The general sketch (Sec. 2.4) on the headline system: random sign
    columns with a history of K directions, a fixed number of columns."""
    A, b, xs = synth.overdetermined_scaled(m=1_000_000, n=200_000, per_row=8, seed=1)
    A = A.astype(np.float64)
    bd = torch.from_numpy(b).cuda()
    ctx = plss.Context(A)
    t, (x, r), clk = _timed(torch, lambda: ctx.solve(bd, sketch="general", tol=0.0, maxit=cols, kacz_hist=K,
                                                     seed=11), 1, 1)
    ctx.close()
    # per column: y = A^T s and r = b - A x (CSR + CSC streams, x gathered), and the history of
    # on average about K/2 directions of n doubles streamed twice (c = Q^T y, q = y - Q d)
    nnz, n, m = A.nnz, A.n, A.m
    hist_bytes = 2 * (min(K, cols) / 2) * n * 8
    return {"seconds": t, "columns": r["iters"], "us_per_column": t / max(1, r["iters"]) * 1e6,
            "relres_true": r["relres_true"], "history": K,
            "history_bytes_per_column": hist_bytes,
            "sparse_bytes_per_column": 2 * nnz * 12 + 8 * (2 * m + 3 * n),
            "clocks": clk,
            "workload": f"{WORKLOAD}, FP64, {cols} sketch columns, history {K}"}


def run_extras(args):
    import torch
    from paper_2207_07615_gb300 import plss
    out = {}
    for name, fn in (("c1", lambda: extra_c1(torch, plss)), ("c4b_fp32", lambda: extra_c4b(torch, plss)),
                     ("c3_identity", lambda: extra_c3_identity(torch, plss)),
                     ("c2_general", lambda: extra_general(torch, plss)),
                     ("c5", lambda: extra_c5(plss))):
        t0 = time.perf_counter()
        try:
            out[name] = fn()
        except Exception as e:   # a failing extra must not cost the headline line
            out[name] = {"error": f"{type(e).__name__}: {e}"}
        out[name]["wall_s"] = time.perf_counter() - t0
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload != "c2":
        globals()[f"suite_{args.workload}"](args)
    else:
        run_plss(args)


if __name__ == "__main__":
    main()
