"""Benchmark: semi-discrete OT reconstruction on one GB300 (or N replicas).

Setup (untimed for the step metric): a damped-Newton solve from psi = 0 to
max|V - nu|/nu <= tol on the workload box (timed as the OT solve), continued to tol/10.

A step is one Laguerre evaluation (sdot_laguerre: security test, re-queue and FP64
re-clip passes, reductions, volumes, centroids and the CSR Hessian) at converged
weights, kNN excluded: the cells/s definition of the measurement plan. value = N / mean
step time, summed over ranks. Positions and weights are in device memory when the timed
region starts; ``e2e`` repeats the calls through host buffers (psi in, volumes and
centroids out, copied inside the timed region). ``extra.ot_solve_s`` holds the OT solve
time from psi = 0 (sdot_create + sdot_solve to tol) in both precisions, measured in the
same run. Every timed call certifies every cell, by its security walk or by the
certificate carried from the previous call when psi and the cell moved less than its
reserves; ``extra.eval_detail.carried`` counts the carried cells, and
``extra.cells_per_s_walk_only`` times the same calls on a context with carrying off.
``roofline`` is the first clipping pass against the derived FP32 peak, and
``extra.roofline_cg`` is the CG iteration against the measured HBM bandwidth. Their
``traffic`` fields are DRAM bytes from ncu captures of the current kernels on the 128^3
version of the box, scaled to a launch.
The default workload is the 256^3 Zel'dovich box with 5% clumped points (17.6 M
seeds), mixed precision. ``--impl reference`` times the CPU oracle instead on a
bounded sample of the same workload (certified cells at psi = 0, cells/s).

``--serving`` runs the serving workload instead: 64 reconstruction jobs of
N = n^3 seeds, n log-uniform in [32, 128], arriving as a Poisson stream at a server
(sdot_server_*) that admits them by device footprint and runs them concurrently;
it reports the p50 and p99 job latency (completion - arrival) and the throughput.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

DEFAULT_WORKLOAD = "zeldovich-256^3-kinv-0.3a+clumps"
# algorithmic FP32 work of one cell clip: ~24 plane tests x ~20 vertices x 6 flop,
# ~60 new vertices x 10, ~48 fan triangles x 45 (volume, first moment, area)
FLOP_PER_CELL = 6000.0
FP32_LANES_PER_SM = 128
N_SM = 152
# CG vector traffic per row and iteration: the update kernel reads u, p, w, s, x, r and
# the inverse diagonal and writes p, s, x, r, u and the FP32 copy of u (100 B); the SpMV
# reads u_i in FP64 and FP32 and writes w_i (20 B); the gathered FP32 neighbour values
# u_j are counted once per row (4 B)
CG_BYTES_PER_ROW = 124
# per off-diagonal entry of L: int32 column + FP32 weight
CG_BYTES_PER_ENTRY = 8
# DRAM bytes (read + write) per unit from ncu captures of the current kernels on the
# clumpy 128^3 box (N = 2,202,087), scaled to a launch by the units it processes (None:
# not captured since the kernel last changed): the first clipping pass per cell
# (1.569 + 7.206 GB), one CG iteration (SpMV 402.4 MB + update 162.8 MB) per row
CLIP_DRAM_PER_CELL = (1.569416e9 + 7.205903e9) / 2202087
CG_DRAM_PER_ROW = (385.858560e6 + 16.551168e6 + 123.337216e6 + 39.467264e6) / 2202087


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--box-n", type=int, default=0,
                    help="profiling aid: the workload's recipe at lattice side n (clump "
                         "counts scaled with n^3); the bench line names the smaller box")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--tol", type=float, default=1e-4)
    ap.add_argument("--no-fp64-compare", action="store_true",
                    help="skip the OT solve and evaluations in the other precision")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--laguerre-once", action="store_true",
                    help="profiling aid: build the context and evaluate one diagram at psi = 0")
    ap.add_argument("--serving", action="store_true",
                    help="serving workload: Poisson stream of jobs, p50/p99 latency")
    ap.add_argument("--jobs", type=int, default=64)
    ap.add_argument("--rate", type=float, default=0.0,
                    help="arrivals per second (0: 1 / the mean solo solve time, calibrated)")
    ap.add_argument("--max-active", type=int, default=8)
    ap.add_argument("--no-batch-clip", action="store_true",
                    help="serving: each job launches its own clipping passes")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(self.rows)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def max_over_ranks(ms, dist):
    """Step time of the slowest rank (the whole job's time); ms when running alone."""
    import torch

    t = torch.tensor([ms], dtype=torch.float64)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_config(workload, rank, world, box_n=0):
    """Replicas only: every rank solves its own box (seed offset by 1000 x rank). box_n:
    the same recipe at lattice side box_n (clump counts scaled with the seed count)."""
    from paper_2110_08868_gb300 import ics

    cfg = dict(ics.CONFIGS[workload])
    if box_n:
        f = (box_n / cfg["n"]) ** 3
        cfg["n"] = box_n
        if cfg.get("clumps"):
            c = dict(cfg["clumps"])
            c["n_clumps"] = max(1, int(round(c["n_clumps"] * f)))
            c["n_extra"] = max(1, int(round(c["n_extra"] * f)))
            cfg["clumps"] = c
    if world > 1:
        cfg["seed"] = cfg["seed"] + 1000 * rank
    return cfg


def _oracle_cells_worker(path, L, idx):
    """One host core: the certified oracle cells idx of the box stored at path (psi = 0),
    single-threaded. Returns the seconds it took."""
    os.environ["OMP_NUM_THREADS"] = "1"
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import sdot_oracle as O

    y = np.load(path, mmap_mode="r")
    y = np.ascontiguousarray(y)
    psi = np.zeros(y.shape[0])
    O.cells(y, psi, L, "certified", idx=np.asarray(idx[:1]))  # build / load first
    t0 = time.perf_counter()
    O.cells(y, psi, L, "certified", idx=np.asarray(idx))
    return time.perf_counter() - t0


_BASELINE_BOX = {}


def cpu_baseline(workload, cells=None):
    """The CPU oracle as it stands, on a bounded sample of the workload's cells.

    Each certified oracle cell sorts all N candidate seeds, so one sample is one random
    cell of the box at psi = 0 per host core, computed by single-threaded worker
    processes (started with spawn) that share the positions through a memory-mapped
    file. The rate is the sample's cells over the slowest worker's time.
    """
    import multiprocessing as mp
    import tempfile

    from paper_2110_08868_gb300 import ics

    if workload not in _BASELINE_BOX:
        y, nu, L = ics.make_config(**ics.CONFIGS[workload])
        fd, path = tempfile.mkstemp(suffix=".npy")
        os.close(fd)
        np.save(path, y)
        _BASELINE_BOX[workload] = (path, int(y.shape[0]), float(L))
    path, N, L = _BASELINE_BOX[workload]
    nproc = os.cpu_count() or 1
    cells = cells or nproc
    rng = np.random.default_rng(123)
    idx = rng.choice(N, cells, replace=False)
    parts = [idx[w::nproc].tolist() for w in range(min(nproc, cells))]
    ctx = mp.get_context("spawn")
    with ctx.Pool(len(parts)) as pool:
        secs = pool.starmap(_oracle_cells_worker, [(path, L, part) for part in parts])
    dt = max(secs)
    return {"value": cells / dt, "unit": "cells/s", "cores": len(parts), "kind": "oracle",
            "sample": f"{cells} random certified oracle cells of the {workload} box (N={N}) at "
                      f"psi=0 on {len(parts)} host cores (one single-threaded worker process "
                      f"per core), slowest worker {dt:.1f} s"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    steps = []
    base = None
    for s in range(args.warmup + args.steps):
        b = cpu_baseline(args.workload)
        if s >= args.warmup:
            steps.append(b["value"])
        base = b
    v = statistics.median(steps)
    line = {"impl": "reference", "metric": "Laguerre cells/s", "value": v, "unit": "cells/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload, "psi": 0,
                                             "mode": "certified oracle cells"},
            "cpu_baseline": {"value": v, "unit": "cells/s", "cores": base["cores"],
                             "kind": "oracle", "sample": base["sample"]},
            "e2e": {"value": v, "unit": "cells/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def timed_solve(B, pos_dev, box, prec, tol):
    """OT solve time from psi = 0: sdot_create (kNN) + sdot_solve(tol), wall clock with
    the device synchronised on both sides. Returns (seconds, stats, ctx)."""
    import torch

    opt = B.sdot_default_options(precision=prec)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc, ctx = B.sdot_create(pos_dev, None, box, opt)
    B.check(rc)
    st = B.sdot_stats()
    B.check(B.sdot_solve(ctx, tol, None, st))
    torch.cuda.synchronize()
    return time.perf_counter() - t0, st.as_dict(), ctx


def eval_steps(B, ctx, psis, vol, cen, hcsr, n, stream):
    """n evaluations (sdot_laguerre with volumes, centroids and the CSR Hessian) cycling
    through psis; per call its device time (CUDA events on the context's stream) and the
    library's report of the clipping passes."""
    import torch

    ms, info = [], []
    for k in range(n):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        B.check(B.sdot_laguerre(ctx, psis[k % len(psis)], vol, cen, hcsr))
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        ei = B.sdot_eval_info()
        B.check(B.sdot_last_eval(ctx, ei))
        info.append(ei.as_dict())
    return ms, info


def run_native(args, rank, world, local):
    import torch

    from paper_2110_08868_gb300 import binding as B

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    from paper_2110_08868_gb300 import ics

    y, nu, L = ics.make_config(**replica_config(args.workload, rank, world, args.box_n))
    N = int(y.shape[0])
    box = [L, L, L]
    pos_dev = torch.from_numpy(y).cuda()
    stream = torch.cuda.current_stream()
    other = "fp64" if args.precision == "mixed" else "mixed"

    # OT solve from psi = 0 in the bench precision; its weights psi_a (max|V - nu|/nu <=
    # tol) and their continuation psi_b (<= tol/10) are the converged weights at which
    # the evaluations are timed. The timed calls alternate between the two, so every
    # call computes a new diagram from the previous one (the solver's access pattern).
    solve_s, solve_st, ctx = timed_solve(B, pos_dev, box, args.precision, args.tol)
    try:
        psi_a = torch.empty(N, dtype=torch.float64, device="cuda")
        psi_b = torch.empty(N, dtype=torch.float64, device="cuda")
        B.check(B.sdot_get_psi(ctx, psi_a))
        st_b = B.sdot_stats()
        B.check(B.sdot_solve(ctx, 0.1 * args.tol, psi_a, st_b))
        B.check(B.sdot_get_psi(ctx, psi_b))
        vol = torch.empty(N, dtype=torch.float64, device="cuda")
        cen = torch.empty((N, 3), dtype=torch.float64, device="cuda")
        hcsr = B.sdot_csr()
        psis = [psi_a, psi_b]
        eval_steps(B, ctx, psis, vol, cen, hcsr, args.warmup, stream)
        torch.cuda.synchronize()
        sampler = ClockSampler(local)
        sampler.start()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        l0 = B.sdot_kernel_launches()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        torch.cuda.nvtx.range_push("bench_timed")
        ms_each, info = eval_steps(B, ctx, psis, vol, cen, hcsr, args.steps, stream)
        torch.cuda.nvtx.range_pop()
        ev1.record(stream)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        launches = B.sdot_kernel_launches() - l0
        clocks = sampler.stop()
        ms = ev0.elapsed_time(ev1) / args.steps
        ms_max = max_over_ranks(ms, dist)
        value = world * N / (ms_max / 1e3)
        hess_nnz = int(hcsr.nnz)

        # e2e: the same calls through pinned host buffers (psi in, volumes and centroids
        # out, the copies inside the timed region)
        e2e = None
        if not args.no_e2e:
            psis_h = [p.cpu().pin_memory() for p in psis]
            vol_h = torch.empty(N, dtype=torch.float64).pin_memory()
            cen_h = torch.empty((N, 3), dtype=torch.float64).pin_memory()
            if dist is not None:
                dist.barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for k in range(args.steps):
                B.check(B.sdot_laguerre(ctx, psis_h[k % 2], vol_h, cen_h, hcsr))
            torch.cuda.synchronize()
            e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3 / args.steps, dist)
            e2e = {"value": world * N / (e_ms / 1e3), "unit": "cells/s",
                   "h2d_bytes_per_step": 8 * N, "d2h_bytes_per_step": 8 * N + 24 * N}
        # the same calls on a context that carries no certificates (every cell walks)
        rc, ctx3 = B.sdot_create(pos_dev, None, box,
                                 B.sdot_default_options(precision=args.precision,
                                                        carry_certificates=0))
        B.check(rc)
        try:
            eval_steps(B, ctx3, psis, vol, cen, hcsr, 3, stream)
            ms3, info3 = eval_steps(B, ctx3, psis, vol, cen, hcsr, 4, stream)
        finally:
            B.sdot_destroy(ctx3)
    finally:
        B.sdot_destroy(ctx)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    peaks = measured_peaks()
    # clip roofline: the first clipping pass of each timed evaluation
    pass1 = [x["ms_pass"][0] for x in info]
    pass1_ms = statistics.median(pass1)
    clock_ghz = (clocks["sm_mhz"] or peaks.get("sm_max_mhz", 2070.0)) / 1e3
    peak_tf = N_SM * FP32_LANES_PER_SM * 2 * clock_ghz / 1e3
    achieved_tf = N * FLOP_PER_CELL / (pass1_ms / 1e3) / 1e12
    kname = "clip_kernel<float,CapS,certify>" if args.precision == "mixed" else \
        "clip_kernel<double,CapS,certify>"
    roofline = {"kernel": kname + " (first clipping pass)", "bound": "alu",
                "launches_timed": len(pass1), "achieved": achieved_tf, "peak": peak_tf,
                "unit": "TFLOP/s", "frac": achieved_tf / peak_tf,
                "traffic": None if CLIP_DRAM_PER_CELL is None else CLIP_DRAM_PER_CELL * N,
                "peak_source": f"derived: 152 SMs x 128 FP32 lanes x 2 flop x {clock_ghz:.3f} "
                               "GHz (median SM clock sampled under load)",
                "per_launch_ms": pass1_ms, "flop_per_cell": FLOP_PER_CELL}
    # CG (HBM-bound): algorithmic bytes per iteration = the off-diagonal entries of L
    # (int32 column + FP32 weight; the sliced-ELL padding is not counted) + the vectors
    # (see CG_BYTES_PER_ROW)
    cg = None
    if solve_st["cg_iters"] > 0:
        it_ms = solve_st["ms_cg"] / solve_st["cg_iters"]
        bytes_it = solve_st["hess_offdiag"] * CG_BYTES_PER_ENTRY + CG_BYTES_PER_ROW * N
        gbs = bytes_it / (it_ms / 1e3) / 1e9
        hbm = peaks.get("hbm_gbs", 6786.2)
        cg = {"kernel": "CG iteration (cg_spmv_kernel + cg_update_kernel)", "bound": "hbm",
              "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
              "traffic": None if CG_DRAM_PER_ROW is None else CG_DRAM_PER_ROW * N,
              "per_iter_ms": it_ms, "bytes_per_iter": bytes_it,
              "hess_slots": solve_st["hess_slots"], "hess_offdiag": solve_st["hess_offdiag"],
              "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
    keep = ("newton_iters", "laguerre_evals", "cg_iters", "max_rel_err", "ms_knn", "ms_clip",
            "ms_cg", "ms_pass", "refined_fp64")
    extra = {"ot_solve_s": {args.precision: solve_s},
             "solve": {args.precision: {k: solve_st[k] for k in keep}},
             "eval_ms_median": statistics.median(ms_each),
             "cells_per_s_median": N / (statistics.median(ms_each) / 1e3),
             "eval_detail": {"requeued": [x["requeued"] for x in info][:4],
                             "reclipped_fp64": [x["reclipped_fp64"] for x in info][:4],
                             "carried": [x["carried"] for x in info][:4],
                             "ms_pass_median": [statistics.median(x["ms_pass"][q] for x in info)
                                                for q in range(3)]},
             "cells_per_s_walk_only": N / (statistics.median(ms3) / 1e3),
             "ms_pass1_walk_only": statistics.median(x["ms_pass"][0] for x in info3),
             "hess_nnz": hess_nnz,
             "roofline_cg": cg}
    if not args.no_fp64_compare:
        # the other precision: its OT solve from psi = 0 in the same run, and its cells/s
        # at the same two converged weights
        s2, st2, ctx2 = timed_solve(B, pos_dev, box, other, args.tol)
        try:
            eval_steps(B, ctx2, psis, vol, cen, hcsr, 2, stream)
            ms2, info2 = eval_steps(B, ctx2, psis, vol, cen, hcsr, 4, stream)
        finally:
            B.sdot_destroy(ctx2)
        extra["ot_solve_s"][other] = s2
        extra["solve"][other] = {k: st2[k] for k in keep}
        extra["cells_per_s_" + other] = N / (statistics.median(ms2) / 1e3)
        extra["mixed_solve_faster"] = extra["ot_solve_s"]["mixed"] < extra["ot_solve_s"]["fp64"]
    cpu = None
    if not args.no_cpu_baseline:
        cpu = cpu_baseline(args.workload)
    line = {"metric": "Laguerre cells/s", "value": value, "unit": "cells/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": args.workload + (f" at n={args.box_n}" if args.box_n else ""),
                       "N": N, "precision": args.precision,
                       "tol": args.tol, "k": 24,
                       "step": "one sdot_laguerre (volumes, centroids, CSR Hessian) at the "
                               "converged weights of the solve to tol, alternating with its "
                               "continuation to tol/10; kNN excluded; every cell certified, "
                               "by its security walk or by the certificate carried from the "
                               "previous call (extra.eval_detail.carried cells; "
                               "extra.cells_per_s_walk_only with carrying off)",
                       "l2": "inputs larger than L2 (device working set >> 129 MB)",
                       "parallelism": "replicas" if world > 1 else "1 GPU"},
            "e2e": e2e, "gpu_launches": launches, "clocks": clocks, "roofline": roofline,
            "cpu_baseline": cpu, "extra": extra}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def laguerre_once(args):
    import torch

    from paper_2110_08868_gb300 import binding as B
    from paper_2110_08868_gb300 import ics

    y, nu, L = ics.make_config(**ics.CONFIGS[args.workload])
    s = B.Solver(torch.from_numpy(y).cuda(), [L, L, L], precision=args.precision)
    g = s.laguerre(allow_empty=True)
    torch.cuda.synchronize()
    print(json.dumps({"workload": args.workload, "N": int(y.shape[0]),
                      "sum_vol_rel_err": float(g["vol"].sum() / L ** 3 - 1.0)}))


def nearest_rank(sorted_vals, p):
    """p-quantile by the nearest-rank rule (rank ceil(p n), 1-based)."""
    n = len(sorted_vals)
    r = max(1, int(np.ceil(p * n)))
    return sorted_vals[min(r, n) - 1]


def run_serving(args, rank, world, local):
    import torch

    from paper_2110_08868_gb300 import binding as B
    from paper_2110_08868_gb300 import ics

    if rank != 0:  # replicas only: the serving stream runs on one GPU
        return
    torch.cuda.set_device(local)
    sides, gaps = ics.serving_stream(args.jobs)
    boxes = [np.ascontiguousarray(ics.zeldovich_box(int(n), 1.0, ics.spectrum_kinv, 0.3,
                                                    1000 + j)[0])
             for j, n in enumerate(sides)]
    srv = B.Server(max_active=args.max_active, batch_clip=not args.no_batch_clip)
    # warm-up and calibration: the solo solve time of a 64^3 job, scaled by N to the
    # stream's mean job size, sets the default arrival rate
    ycal = np.ascontiguousarray(ics.zeldovich_box(64, 1.0, ics.spectrum_kinv, 0.3, 999)[0])
    t_cal = 0.0
    for _ in range(2):
        t0 = time.perf_counter()
        jid = srv.submit(ycal, [1.0] * 3, args.tol)
        if not srv.wait(jid, 900.0):
            raise RuntimeError("serving: the calibration job did not finish in 900 s")
        srv.result(jid)
        t_cal = time.perf_counter() - t0
    mean_n = float(np.mean(sides.astype(np.float64) ** 3))
    mean_solo = t_cal * mean_n / 64 ** 3
    rate = args.rate if args.rate > 0 else 1.0 / mean_solo
    arrivals = np.cumsum(gaps) / rate
    sampler = ClockSampler(local)
    sampler.start()
    l0 = B.sdot_kernel_launches()
    t_start = time.perf_counter()
    ids = []
    for j in range(args.jobs):
        delay = arrivals[j] - (time.perf_counter() - t_start)
        if delay > 0:
            time.sleep(delay)
        ids.append(srv.submit(boxes[j], [1.0] * 3, args.tol))
    results = []
    for jid in ids:
        if not srv.wait(jid, 1800.0):
            raise RuntimeError(f"serving: job {jid} did not finish in 1800 s")
        results.append(srv.result(jid))
    wall = time.perf_counter() - t_start
    launches = B.sdot_kernel_launches() - l0
    clocks = sampler.stop()
    info = srv.info()
    srv.close()
    lat = sorted(float(r["times"][2] - r["times"][0]) for r in results)
    queue_wait = sorted(float(r["times"][1] - r["times"][0]) for r in results)
    t_first = min(float(r["times"][0]) for r in results)
    t_last = max(float(r["times"][2]) for r in results)
    cells = float(np.sum(sides.astype(np.float64) ** 3))
    converged = all(r["stats"]["max_rel_err"] <= args.tol for r in results)
    p50, p99 = nearest_rank(lat, 0.50), nearest_rank(lat, 0.99)
    line = {"metric": "serving job latency p50 (p99 beside)", "value": p50, "unit": "s",
            "n_gpus": 1, "steps": args.jobs, "warmup": 2, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "p50_s": p50, "p99_s": p99,
            "queue_wait_p50_s": nearest_rank(queue_wait, 0.50),
            "queue_wait_p99_s": nearest_rank(queue_wait, 0.99),
            "throughput": {"value": cells / (t_last - t_first), "unit": "cells/s"},
            "makespan_s": t_last - t_first, "wall_s": wall, "all_converged": converged,
            "config": {"workload": f"serving stream: {args.jobs} jobs, N = n^3 with n "
                                   "log-uniform in [32, 128], 1/k spectrum 0.3a, Poisson "
                                   "arrivals",
                       "rate_per_s": rate, "calibration_solo_64^3_s": t_cal,
                       "tol": args.tol, "precision": "mixed", "max_active": args.max_active,
                       "batch_clip": not args.no_batch_clip,
                       "hbm_budget": info["hbm_budget"], "total_cells": cells,
                       "l2": "each job's working set (>= 47 MB) and the mix exceed L2"},
            "e2e": {"value": p50, "unit": "s",
                    "h2d_bytes_per_step": 24.0 * cells / args.jobs,
                    "d2h_bytes_per_step": 32.0 * cells / args.jobs},
            "server": {"peak_used_bytes": info["peak_used_bytes"],
                       "peak_active": info["peak_active"]},
            "gpu_launches": launches, "clocks": clocks}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.laguerre_once:
        laguerre_once(args)
        return
    if args.serving:
        run_serving(args, rank, world, local)
        return
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_native(args, rank, world, local)


if __name__ == "__main__":
    main()
