"""Benchmark of the CSR SpMV / SpMM hot path on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload spmv|spmm|small] [--impl reference]

Default workload (one "step" = one pass over all of it): FP64 SpMV y <- A x
(paper Sec. 3) on three synthetic matrices shaped like the paper's test set
(Sec. 4, Table "tab:matrices"): a 3D 27-point stencil on 100^3 (regular mesh
class), a random banded FEM-like matrix with 2M rows and 50 nonzeros per row
(FEM class), and an R-MAT graph of scale 22, edge factor 16 (power-law
class).  Each matrix runs through an autotuned plan.  Inputs are resident in
HBM when timing starts; the L2 is flushed (a 256 MiB write, not timed)
before every step, and every matrix is larger than the L2 anyway.

Reported (one JSON line on rank 0): GFLOP/s = 2 * nnz * k / t over all
ranks, the per-launch roofline of the dominant kernel against the measured
HBM copy bandwidth (compulsory bytes, Sec. 4.2: 12 nnz + 4 (m+1) + 8 n k +
8 m k) and against the FP64 FMA rate measured live (GB300's second roof),
an end-to-end figure through the public API with host buffers, the CPU
oracle timed on the host cores, and the SM clocks sampled during timing.

--gpus N > 1 runs under torchrun: every rank multiplies its own independent
matrices (weak scaling, no collective on the data path; one all-reduce of
the timings).  --impl reference times the CPU oracle instead (rank 0 only).
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

import synth  # noqa: E402

METRIC = "CSR SpMV/SpMM GFLOP/s & % of HBM roofline at FP64; batched vs looped"
UNIT = "GFLOP/s"


# ------------------------------------------------------------------ workloads

def workload_matrices(name: str, rank: int):
    """(name, CSR, k list) of a workload; rank shifts the seeds so ranks hold independent problems."""
    s = synth.BASE_SEED + 1 + 1000 * rank
    if name == "small":
        return [("stencil2d_64", synth.stencil2d(64))], [1]
    if name in ("spmv", "spmm", "rcm", "bcsr"):
        mats = [("stencil3d_100", synth.stencil3d(100)),
                ("banded_2M_hbw1000_50", synth.banded(2_000_000, hbw=1000, per_row=50, seed=s)),
                ("rmat_s22_ef16", synth.rmat(22, ef=16, seed=s))]
        return mats, ([1, 4, 8, 16] if name == "spmm" else [1])
    raise ValueError(name)


WORKLOAD_TEXT = {
    "spmv": "FP64 CSR SpMV sweep: 3D 27-pt stencil 100^3 (m=1,000,000, nnz=26,463,592); random banded "
            "m=2,000,000 hbw 1000 50 nnz/row N(0,1) dominant diagonal; R-MAT scale 22 ef 16 "
            "(a,b,c=0.57,0.19,0.19) dedup, vals 1.0; x uniform[-1,1]",
    "spmm": "FP64 CSR SpMM Y=A X, X row-major n x k, k in {1,4,8,16}, on the 27-pt 100^3, banded 2M and "
            "R-MAT 22 matrices; X uniform[-1,1]",
    "small": "FP64 CSR SpMV, 2D 5-pt Laplacian 64x64 (m=4096, nnz=20,224)",
    "batched": "Batched FP64 SpMM, 512 CSR matrices (rows log-uniform 1k-200k, avg nnz/row 4-64, round-robin "
               "2D stencil / random banded / R-MAT), k=8 right-hand sides uniform[-1,1], one persistent launch "
               "replayed from a CUDA graph, per-matrix autotuned configuration",
    "rcm": "FP64 CSR SpMV on the sweep's three matrices before and after reverse Cuthill-McKee reordering "
           "B = P A P^T computed on the GPU (Sec. 4.4): time of the ordering and of the permutation, SpMV "
           "GFLOP/s, UCLD (32-byte sectors) and bandwidth max|i-j| of A and B",
    "bcsr": "FP64 SpMV from register-blocked CRS (Sec. 4.5: aligned a x b dense blocks, zeros stored and "
            "multiplied) against tuned CSR on the sweep's 27-pt 100^3, banded 2M and R-MAT 22 matrices and a "
            "blocky FEM-like matrix (27-pt stencil on 30^3 nodes with 8 x 8 node couplings, m=216,000, "
            "nnz=43,614,208); GFLOP/s count only stored entries (2 nnz)",
    "autograd": "Differentiable SpMV/SpMM on R-MAT scale 20 ef 16, vals uniform[0.5,1.5], k in {1,8}, FP64 and "
                "FP32: forward Y=A X, backward dX=A^T dY and dvals (transpose built once, timed separately)",
}


# Source files that define each variant's kernel: a DRAM-traffic figure recorded from an ncu
# capture (profiles/traffic.txt) is reported only while these files are unchanged.
KERNEL_SOURCES = {
    1: ["rows_kernel.cuh", "device_common.cuh"],
    2: ["merge_kernel.cuh", "device_common.cuh"],
    3: ["rows_tma.cuh", "rows_kernel.cuh", "device_common.cuh", "df64.cuh"],
    4: ["merge_kernel.cuh", "device_common.cuh"],
}


def kernel_source_hash(variant: int) -> str:
    import hashlib

    h = hashlib.sha256()
    for f in KERNEL_SOURCES.get(variant, []):
        with open(os.path.join(ROOT, "paper_1302_1078_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(variant: int, matrix: str):
    """DRAM bytes per launch from profiles/traffic.txt (lines: variant hash bytes matrix command...),
    or None when no capture matches the current kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    want = kernel_source_hash(variant)
    for line in open(path):
        f = line.split()
        if len(f) >= 4 and not line.startswith("#") and f[0] == str(variant) and f[1] == want and f[3] == matrix:
            return float(f[2])
    return None


def compulsory_bytes(m, n, nnz, k, es=8):
    """Sec. 4.2 / Sec. 5 application-bandwidth model with (m+1) row pointers:
    es*nnz + 4*nnz + 4*(m+1) + es*n*k + es*m*k."""
    return (es + 4) * nnz + 4 * (m + 1) + es * n * k + es * m * k


# --------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples (SM clock, max clock, throttle reasons) while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc is None:
            return
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
            except (ValueError, IndexError):
                continue
            for i, nm in enumerate(names):
                if len(r) > 4 + i and r[4 + i].lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_smi_id(torch, dev_index: int) -> str:
    try:
        p = torch.cuda.get_device_properties(dev_index)
        return f"{p.pci_domain_id:08X}:{p.pci_bus_id:02X}:{p.pci_device_id:02X}.0"
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        ids = [v for v in vis.split(",") if v.strip()]
        return ids[dev_index] if dev_index < len(ids) else str(dev_index)


# ----------------------------------------------------------------- CPU oracle

def cpu_oracle_rate(mats, ks, budget_s: float = 12.0, frac_rows: float | None = None, threads: int | None = None):
    """Time the CPU oracle (paper Sec. 4.1 row-parallel loop, all host cores unless `threads`)
    on the workload's matrices, repeating whole sweeps until `budget_s` is spent (at least one
    sweep, over a leading fraction of the rows if `frac_rows` is given).
    Returns (GFLOP/s, cores, text)."""
    import oracle

    threads = oracle.max_threads() if threads is None else threads
    xs = {}
    flops = 0.0
    t_total = 0.0
    sweeps = 0
    while True:
        for name, A in mats:
            r1 = A.m if frac_rows is None else max(1, int(A.m * frac_rows))
            rp = A.row_ptr[: r1 + 1]
            nz = int(rp[-1])
            for k in ks:
                key = (name, k)
                if key not in xs:
                    xs[key] = synth.uniform(A.n * k, seed=7, stream=k).reshape(A.n, k) if k > 1 else \
                        synth.uniform(A.n, seed=7)
                t0 = time.perf_counter()
                if k == 1:
                    oracle.spmv(r1, rp, A.col_idx, A.vals, xs[key], threads=threads)
                else:
                    oracle.spmm(r1, rp, A.col_idx, A.vals, xs[key], threads=threads)
                t_total += time.perf_counter() - t0
                flops += 2.0 * nz * k
        sweeps += 1
        if t_total >= budget_s or sweeps >= 50:
            break
    what = f"{sweeps} full sweep(s)" if frac_rows is None else f"{sweeps} sweep(s) over the first {frac_rows:.0%} of rows"
    return flops / t_total / 1e9, threads, f"{what} of the workload, {t_total:.1f} s timed on {threads} thread(s)"


# --------------------------------------------------------------- reference arm

def reference_matrices(workload: str):
    """Matrices and k values the reference arm multiplies for a workload: the workload's own
    matrices, the batch's members (k = 8) or the autograd R-MAT (k = 1 and 8)."""
    if workload == "batched":
        specs = synth.batch_specs(512)
        return [(f"batch_{i}", synth.batch_matrix(sp)) for i, sp in enumerate(specs)], [8]
    if workload == "autograd":
        return [("rmat_s20_ef16", synth.rmat(20, ef=16, seed=synth.BASE_SEED + 3, vals="u0.5_1.5"))], [1, 8]
    return workload_matrices(workload, 0)


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    mats, ks = reference_matrices(args.workload)
    import oracle

    threads = oracle.max_threads()
    # size each step so that warmup + steps stays within about two minutes
    total_nnz = sum(A.nnz for _, A in mats) * len(ks)
    est_step = total_nnz * 2e-9 * 8 / max(1, threads)  # rough seconds per full sweep
    nsteps = args.steps + args.warmup
    frac = None
    if est_step * nsteps > 120:
        frac = max(0.001, 120 / (est_step * nsteps))
    times, flops = [], []
    xs = {}
    for step in range(nsteps):
        f = 0.0
        t0 = time.perf_counter()
        for name, A in mats:
            r1 = A.m if frac is None else max(1, int(A.m * frac))
            rp = A.row_ptr[: r1 + 1]
            for k in ks:
                key = (name, k)
                if key not in xs:
                    xs[key] = synth.uniform(A.n * k, seed=7, stream=k).reshape(A.n, k) if k > 1 else \
                        synth.uniform(A.n, seed=7)
                if k == 1:
                    oracle.spmv(r1, rp, A.col_idx, A.vals, xs[key], threads=threads)
                else:
                    oracle.spmm(r1, rp, A.col_idx, A.vals, xs[key], threads=threads)
                f += 2.0 * int(rp[-1]) * k
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
            flops.append(f)
    value = sum(flops) / sum(times) / 1e9
    sample = "whole workload per step" if frac is None else f"first {frac:.1%} of the rows of each matrix per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT[args.workload]},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"CPU oracle (row-parallel OpenMP, dynamic,64), {sample}"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# -------------------------------------------------------------------- GPU arm

def launches_per_call(cfg: dict, k: int, dtype_vec: int = 2) -> int:
    """Kernels one product call launches: ROWS 1 per column panel; MERGE partition is
    precomputed by the plan, then kernel + carry fix-up per panel."""
    panel = 32 * dtype_vec if k > 1 else 1
    panels = (k + panel - 1) // panel
    return panels * (1 if cfg["variant"] == 1 else 2)


def run_gpu(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    import paper_1302_1078_gb300 as gbs

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    gbs.lib()

    mats, ks = workload_matrices(args.workload, rank)
    if args.only:
        keep = set(args.only.split(","))
        mats = [(name, A) for name, A in mats if name in keep]
        if not mats:
            raise SystemExit(f"--only {args.only}: no such matrix in the workload")
    # ---- resident inputs and tuned plans
    items = []
    for name, A in mats:
        rp = torch.from_numpy(A.row_ptr).to(dev)
        ci = torch.from_numpy(A.col_idx).to(dev)
        v = torch.from_numpy(A.vals).to(dev)
        # useful cacheline density of the x gathers (Sec. 4.1): 4 doubles = one 32-byte L2 sector,
        # 8 = the paper's 64-byte line; "x_sectors" = distinct sectors summed over rows
        u4, u8 = gbs.ucld(rp, ci, A.n, 4), gbs.ucld(rp, ci, A.n, 8)
        ucld = {"sector_4": u4["ucld"], "line_8": u8["ucld"], "x_sectors": u4["lines"]}
        for k in ks:
            X = synth.uniform(A.n * k, seed=synth.BASE_SEED + 11 + rank, stream=k)
            Xd = torch.from_numpy(X).to(dev).reshape(A.n, k) if k > 1 else torch.from_numpy(X).to(dev)
            Yd = torch.empty((A.m, k) if k > 1 else (A.m,), dtype=torch.float64, device=dev)
            if args.config:
                # a fixed configuration for every product (profiling runs): no tuning
                plan = gbs.Plan(rp, ci, A.n, torch.float64, k, config=json.loads(args.config))
            else:
                plan = gbs.Plan(rp, ci, A.n, torch.float64, k, tune=True, emulate=args.emulate)
            items.append(dict(name=name, A=A, k=k, rp=rp, ci=ci, v=v, X=Xd, Y=Yd, plan=plan, cfg=plan.config,
                              bytes=compulsory_bytes(A.m, A.n, A.nnz, k), flops=2.0 * A.nnz * k, ucld=ucld))
    stream = torch.cuda.current_stream(dev)

    def call(it):
        if it["k"] == 1:
            it["plan"].spmv(it["v"], it["X"], it["Y"])
        else:
            it["plan"].spmm(it["v"], it["X"], it["Y"])

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    # ---- FP64 FMA rate (second roof), measured live
    probe_out = torch.empty(152 * 8 * 256, dtype=torch.float64, device=dev)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks, threads_p, iters = sms * 8, 256, 2048
    L = gbs.lib()
    for _ in range(2):
        L.gbs_fp64_probe(probe_out.data_ptr(), blocks, threads_p, iters, stream.cuda_stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    L.gbs_fp64_probe(probe_out.data_ptr(), blocks, threads_p, iters, stream.cuda_stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    fp64_probe_gflops = 2.0 * 8 * iters * blocks * threads_p / (e0.elapsed_time(e1) * 1e-3) / 1e9

    # ---- warm-up
    for _ in range(args.warmup):
        flush.zero_()
        for it in items:
            call(it)
    torch.cuda.synchronize(dev)

    # ---- timed region: K steps; per-launch events on the launching stream
    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in items]
          for _ in range(args.steps)]
    sampler = ClockSampler(gpu_smi_id(torch, local_rank))
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    sampler.start()
    time.sleep(0.05)
    torch.cuda.nvtx.range_push("timed")
    t0 = time.perf_counter()
    for s in range(args.steps):
        flush.zero_()
        for j, it in enumerate(items):
            ev[s][j][0].record(stream)
            call(it)
            ev[s][j][1].record(stream)
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - t0
    torch.cuda.nvtx.range_pop()
    if world > 1:
        dist.barrier()
    sampler.stop()
    per_item_ms = [[ev[s][j][0].elapsed_time(ev[s][j][1]) for s in range(args.steps)] for j in range(len(items))]
    step_ms = sum(statistics.mean(t) for t in per_item_ms)

    # ---- warm figure (labelled, not the value): the same products back to back, no L2 flush
    warm_steps = max(3, min(args.steps, 20))
    wev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in items]
           for _ in range(warm_steps)]
    for s in range(warm_steps):
        for j, it in enumerate(items):
            wev[s][j][0].record(stream)
            call(it)
            wev[s][j][1].record(stream)
    torch.cuda.synchronize(dev)
    warm_ms = [statistics.mean(wev[s][j][0].elapsed_time(wev[s][j][1]) for s in range(warm_steps))
               for j in range(len(items))]
    flops_step = sum(it["flops"] for it in items)

    # ---- end to end through the public API with host buffers (H2D inputs, D2H result, each step)
    pinned = []
    for it in items:
        A = it["A"]
        hb = dict(rp=torch.from_numpy(A.row_ptr).pin_memory(), ci=torch.from_numpy(A.col_idx).pin_memory(),
                  v=torch.from_numpy(A.vals).pin_memory(), X=it["X"].cpu().pin_memory(),
                  Y=torch.empty(it["Y"].shape, dtype=torch.float64).pin_memory())
        pinned.append(hb)
    h2d = sum(h["rp"].numel() * 4 + h["ci"].numel() * 4 + h["v"].numel() * 8 + h["X"].numel() * 8 for h in pinned)
    d2h = sum(h["Y"].numel() * 8 for h in pinned)
    e2e_steps = max(3, min(args.steps, 10))
    # copies overlap the products: a copy stream brings in product j + 1's inputs while the
    # launching stream computes product j, and a third stream returns each result.  The copy
    # of the next step into a product's buffers waits for that product's previous compute.
    h2d_stream, d2h_stream = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    copied = [torch.cuda.Event() for _ in items]
    computed = [torch.cuda.Event() for _ in items]
    returned = [torch.cuda.Event() for _ in items]
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    ee0, ee1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h2d_stream.wait_stream(stream)
    d2h_stream.wait_stream(stream)
    # step 0 is an untimed warm-up (first copies from freshly pinned pages); timing starts after it
    for s_ in range(e2e_steps + 1):
        if s_ == 1:
            torch.cuda.synchronize(dev)
            ee0.record(stream)
            h2d_stream.wait_stream(stream)
            d2h_stream.wait_stream(stream)
        for j, (it, hb) in enumerate(zip(items, pinned)):
            with torch.cuda.stream(h2d_stream):
                if s_ > 0:
                    h2d_stream.wait_event(computed[j])  # the buffers are free again
                it["rp"].copy_(hb["rp"], non_blocking=True)
                it["ci"].copy_(hb["ci"], non_blocking=True)
                it["v"].copy_(hb["v"], non_blocking=True)
                it["X"].copy_(hb["X"], non_blocking=True)
                copied[j].record(h2d_stream)
            stream.wait_event(copied[j])
            if s_ > 0:
                stream.wait_event(returned[j])  # the previous result has left Y
            call(it)
            computed[j].record(stream)
            with torch.cuda.stream(d2h_stream):
                d2h_stream.wait_event(computed[j])
                hb["Y"].copy_(it["Y"], non_blocking=True)
                returned[j].record(d2h_stream)
    stream.wait_stream(h2d_stream)
    stream.wait_stream(d2h_stream)
    ee1.record(stream)
    torch.cuda.synchronize(dev)
    e2e_ms = ee0.elapsed_time(ee1) / e2e_steps

    # ---- max over ranks
    t = torch.tensor([step_ms, e2e_ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    step_ms_max, e2e_ms_max = float(t[0]), float(t[1])

    # ---- per-matrix report, dominant kernel roofline
    hbm_peak = None
    peaks_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(peaks_path):
        hbm_peak = json.load(open(peaks_path)).get("hbm_gbs")
    peak_src = "measured"
    if not hbm_peak:
        hbm_peak, peak_src = 6800.0, "fallback"
    # FP64 roof from the unit counts: 2 DFMA per clock per SM (ncu: sm__sass_thread_inst_executed_op_dfma
    # peak_sustained = 2), 2 flops each, at the median SM clock sampled during the timed region
    clk = sampler.summary()
    sm_mhz = clk["sm_mhz"] or clk["sm_max_mhz"] or 2070.0
    fp64_peak_gflops = 2.0 * 2.0 * sms * sm_mhz * 1e6 / 1e9
    per = []
    for j, it in enumerate(items):
        ms = statistics.mean(per_item_ms[j])
        per.append({"matrix": it["name"], "k": it["k"], "m": it["A"].m, "nnz": it["A"].nnz, "config": it["cfg"],
                    "ms": ms, "gflops": it["flops"] / ms / 1e6, "hbm_gbs": it["bytes"] / ms / 1e6,
                    "hbm_frac": it["bytes"] / ms / 1e6 / hbm_peak,
                    "fp64_frac": it["flops"] / ms / 1e6 / fp64_peak_gflops,
                    "warm_ms_no_l2_flush": warm_ms[j], "ucld": it["ucld"]})
    dom = max(range(len(items)), key=lambda j: per[j]["ms"])
    d = per[dom]
    t_hbm = items[dom]["bytes"] / (hbm_peak * 1e9)
    t_alu = items[dom]["flops"] / (fp64_peak_gflops * 1e9)
    hbm_roof = {"bound": "hbm", "achieved": d["hbm_gbs"], "peak": hbm_peak, "unit": "GB/s", "frac": d["hbm_frac"],
                "traffic": recorded_traffic(d["config"]["variant"], d["matrix"]) if d["k"] == 1 else None,
                "algorithmic_bytes": items[dom]["bytes"], "kernel": f"{d['matrix']} k={d['k']} {d['config']}",
                "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else "fallback"}
    alu_roof = {"bound": "alu", "achieved": d["gflops"], "peak": fp64_peak_gflops, "unit": "GFLOP/s",
                "frac": d["fp64_frac"],
                "peak_source": f"derived: 2 DFMA/clk/SM x 2 flop x {sms} SMs x {sm_mhz:.0f} MHz (median sampled clock); "
                               f"the gbs_fp64_probe kernel reaches {fp64_probe_gflops:.0f} GFLOP/s"}
    roofline = hbm_roof
    roofline["binding_roof"] = "fp64_alu" if t_alu > t_hbm else "hbm"
    roofline["fp64_alu"] = alu_roof

    launches = args.steps * sum(launches_per_call(it["cfg"], it["k"]) for it in items)
    line = {
        "metric": METRIC, "value": world * flops_step / (step_ms_max * 1e-3) / 1e9, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms_max, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT[args.workload], "parallelism": f"independent problems per GPU x{world}",
                   "l2": "256 MiB write before every step (untimed); every matrix exceeds the L2",
                   "timing": "CUDA events around each product on the launching stream; value uses their sum",
                   "wall_s_timed_region": wall},
        "roofline": roofline,
        "e2e": {"value": world * flops_step / (e2e_ms_max * 1e-3) / 1e9, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": e2e_steps,
                "note": "pinned host buffers; one untimed warm-up step; copies on their own streams overlap "
                        "the products; host-to-device copies on this GPU peak near 211 GB/s"},
        "clocks": sampler.summary(),
        "gpu_launches": launches,
        "fp64_peak_gflops_derived": fp64_peak_gflops, "fp64_probe_gflops": fp64_probe_gflops,
        "fp64_emulation": bool(args.emulate),
        "per_matrix": per,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, cores, what = cpu_oracle_rate(mats, ks)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": what}
        v1, _, what1 = cpu_oracle_rate(mats, ks, budget_s=4.0, threads=1)
        line["cpu_baseline_1core"] = {"value": v1, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": what1}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


# --------------------------------------------------------------- batched mode

def shard_for_rank(costs, world: int, rank: int):
    """Indices of the batch members rank `rank` multiplies: greedy longest-processing-time
    assignment of the costs to `world` ranks (deterministic: ties broken by index)."""
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    owner = [0] * len(costs)
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        owner[i] = r
        load[r] += costs[i]
    return [i for i in range(len(costs)) if owner[i] == rank]


def run_batched(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    import paper_1302_1078_gb300 as gbs

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    k = 8
    if args.shard:
        # one batch split across the ranks (strong scaling)
        specs = synth.batch_specs(args.batch_size)
        costs = [sp.rows * (5 if sp.kind == "stencil2d" else sp.avg) for sp in specs]
        mine = shard_for_rank(costs, world, rank)
    else:
        # every rank its own independent batch (weak scaling)
        specs = synth.batch_specs(args.batch_size, seed=synth.BASE_SEED + 4 + 1000 * rank)
        mine = list(range(len(specs)))
    mats, Xs, Ys, flops, bytes_ = [], [], [], 0.0, 0
    for i in mine:
        A = synth.batch_matrix(specs[i])
        rp = torch.from_numpy(A.row_ptr).to(dev)
        ci = torch.from_numpy(A.col_idx).to(dev)
        v = torch.from_numpy(A.vals).to(dev)
        X = torch.from_numpy(synth.uniform(A.n * k, seed=synth.BASE_SEED + 4, stream=i).reshape(A.n, k)).to(dev)
        mats.append((rp, ci, v, A.n))
        Xs.append(X)
        Ys.append(torch.empty((A.m, k), dtype=torch.float64, device=dev))
        flops += 2.0 * A.nnz * k
        bytes_ += compulsory_bytes(A.m, A.n, A.nnz, k)
    plan = gbs.BatchedPlan(mats, Xs, Ys, tune=True)
    info = plan.info()
    # the baseline a per-matrix user would run: each matrix's own standalone-tuned configuration
    plan_pm = gbs.BatchedPlan(mats, Xs, Ys, tune=True, configs=[None] * len(mats))
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def timed(fn, steps):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for s_ in range(steps):
            flush.zero_()
            evs[s_][0].record(stream)
            fn()
            evs[s_][1].record(stream)
        torch.cuda.synchronize(dev)
        return [a.elapsed_time(b) for a, b in evs]

    for _ in range(args.warmup):
        plan.run()
        plan.run_looped()
        plan_pm.run_looped()
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(gpu_smi_id(torch, local_rank))
    if world > 1:
        dist.barrier()
    sampler.start()
    time.sleep(0.05)
    torch.cuda.nvtx.range_push("timed")
    t_batched = timed(plan.run, args.steps)
    torch.cuda.nvtx.range_pop()
    t_looped = timed(plan.run_looped, args.steps)
    t_looped_pm = timed(plan_pm.run_looped, args.steps)
    sampler.stop()
    ms_b, ms_l, ms_lpm = statistics.mean(t_batched), statistics.mean(t_looped), statistics.mean(t_looped_pm)
    t = torch.tensor([ms_b, ms_l, ms_lpm], dtype=torch.float64, device=dev)
    tot = torch.tensor([flops, float(bytes_)], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(tot, op=dist.ReduceOp.SUM)
    ms_b, ms_l, ms_lpm = float(t[0]), float(t[1]), float(t[2])
    flops_all, bytes_all = float(tot[0]), float(tot[1])
    hbm_peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", 6800.0) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6800.0
    variants = {}
    for c in info["configs"]:
        key = "ROWS" if c["variant"] == 1 else "MERGE"
        variants[key] = variants.get(key, 0) + 1
    line = {
        "metric": METRIC, "value": flops_all / (ms_b * 1e-3) / 1e9, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_b, "higher_is_better": True,
        "scaling": "strong" if args.shard else "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT["batched"].replace("512", str(args.batch_size)),
                   "matrices_per_rank": len(mine),
                   "grid": info["grid"], "work_items": info["total_items"], "variants": variants,
                   "l2": "256 MiB write before every step (untimed)"},
        "batched_vs_looped": ms_l / ms_b, "looped_gflops": flops_all / (ms_l * 1e-3) / 1e9,
        "looped_ms": ms_l,
        "looped_note": "looped = the batch's own per-matrix configurations, one launch per matrix; "
                       "looped_tuned = each matrix's standalone-tuned configuration, one launch per matrix",
        "batched_vs_looped_tuned": ms_lpm / ms_b, "looped_tuned_ms": ms_lpm,
        "roofline": {"bound": "hbm", "achieved": bytes_all / (ms_b * 1e-3) / 1e9 / world, "peak": hbm_peak,
                     "unit": "GB/s", "frac": bytes_all / (ms_b * 1e-3) / 1e9 / world / hbm_peak, "traffic": None,
                     "kernel": "batched_kernel (whole batch per launch)"},
        "clocks": sampler.summary(),
        "gpu_launches": args.steps,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------------ reordering

def run_rcm(args, rank, world, local_rank):
    import torch

    import paper_1302_1078_gb300 as gbs

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    mats, _ = workload_matrices("spmv", rank)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def timed_ms(fn, steps):
        evs = []
        for _ in range(steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize(dev)
        return statistics.mean(a.elapsed_time(b) for a, b in evs)

    def bandwidth(rp, ci):
        rows = torch.repeat_interleave(torch.arange(rp.numel() - 1, device=dev, dtype=torch.int64),
                                       (rp[1:] - rp[:-1]).long())
        return int((rows - ci.long()).abs().max().item()) if ci.numel() else 0

    def measure(rp, ci, v, n):
        x = torch.from_numpy(synth.uniform(n, seed=synth.BASE_SEED + 11)).to(dev)
        y = torch.empty(rp.numel() - 1, dtype=torch.float64, device=dev)
        plan = gbs.Plan(rp, ci, n, torch.float64, 1, tune=True)
        for _ in range(args.warmup):
            plan.spmv(v, x, y)
        ms = timed_ms(lambda: plan.spmv(v, x, y), args.steps)
        return {"ms": ms, "gflops": 2.0 * ci.numel() / ms / 1e6, "config": plan.config,
                "ucld_sector_4": gbs.ucld(rp, ci, n, 4)["ucld"], "bandwidth": bandwidth(rp, ci)}

    per, flops, t_before, t_after = [], 0.0, 0.0, 0.0
    for name, A in mats:
        rp = torch.from_numpy(A.row_ptr).to(dev)
        ci = torch.from_numpy(A.col_idx).to(dev)
        v = torch.from_numpy(A.vals).to(dev)
        before = measure(rp, ci, v, A.n)
        gbs.rcm(rp, ci)  # warm-up (allocator, module load)
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        perm = gbs.rcm(rp, ci)
        e1.record(stream)
        brp, bci, bv = gbs.permute_csr(rp, ci, v, perm)
        e2.record(stream)
        torch.cuda.synchronize(dev)
        after = measure(brp, bci, bv, A.n)
        per.append({"matrix": name, "m": A.m, "nnz": A.nnz, "rcm_ms": e0.elapsed_time(e1),
                    "permute_ms": e1.elapsed_time(e2), "before": before, "after": after,
                    "speedup": before["ms"] / after["ms"]})
        flops += 2.0 * A.nnz
        t_before += before["ms"]
        t_after += after["ms"]
        del rp, ci, v, brp, bci, bv, perm
    line = {
        "metric": METRIC, "value": flops / (t_after * 1e-3) / 1e9, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_after, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT["rcm"], "l2": "256 MiB write before every product (untimed)"},
        "value_before_reordering": flops / (t_before * 1e-3) / 1e9, "rcm": per,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------ register blocking

def run_bcsr(args, rank, world, local_rank):
    import torch

    import paper_1302_1078_gb300 as gbs

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    mats, _ = workload_matrices("spmv", rank)
    mats = mats + [("stencil3d_30_dof8", synth.stencil3d_blocks(30, 8))]
    shapes = {"rmat_s22_ef16": [(8, 1), (1, 8)]}  # larger blocks of a power-law matrix are mostly zeros
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    hbm_peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", 6800.0) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6800.0

    def timed_ms(fn):
        for _ in range(args.warmup):
            fn()
        evs = []
        for _ in range(args.steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize(dev)
        return statistics.mean(a.elapsed_time(b) for a, b in evs)

    per = []
    for name, A in mats:
        rp = torch.from_numpy(A.row_ptr).to(dev)
        ci = torch.from_numpy(A.col_idx).to(dev)
        v = torch.from_numpy(A.vals).to(dev)
        x = torch.from_numpy(synth.uniform(A.n, seed=synth.BASE_SEED + 11)).to(dev)
        y = torch.empty(A.m, dtype=torch.float64, device=dev)
        plan = gbs.Plan(rp, ci, A.n, torch.float64, 1, tune=True)
        csr_ms = timed_ms(lambda: plan.spmv(v, x, y))
        entry = {"matrix": name, "m": A.m, "nnz": A.nnz,
                 "csr": {"ms": csr_ms, "gflops": 2.0 * A.nnz / csr_ms / 1e6, "config": plan.config,
                         "hbm_frac": compulsory_bytes(A.m, A.n, A.nnz, 1) / csr_ms / 1e6 / hbm_peak}, "bcsr": []}
        for a, b in shapes.get(name, [(8, 1), (1, 8), (2, 8), (8, 8)]):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            B = gbs.BCSR(rp, ci, v, A.n, a, b)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms = timed_ms(lambda: B.spmv(x, y))
            stored = B.nblocks * a * b
            moved = stored * 8 + B.nblocks * 4 + (B.block_rows + 1) * 4 + 8 * A.n + 8 * A.m
            entry["bcsr"].append({"a": a, "b": b, "blocks": B.nblocks, "fill": A.nnz / max(stored, 1),
                                  "convert_ms": e0.elapsed_time(e1), "ms": ms, "gflops": 2.0 * A.nnz / ms / 1e6,
                                  "relative_to_csr": csr_ms / ms, "block_bytes_hbm_frac": moved / ms / 1e6 / hbm_peak})
            del B
        per.append(entry)
        del rp, ci, v
    best = sum(min([e["csr"]["ms"]] + [b["ms"] for b in e["bcsr"]]) for e in per)
    flops = sum(2.0 * e["nnz"] for e in per)
    line = {
        "metric": METRIC, "value": flops / (best * 1e-3) / 1e9, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": best, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT["bcsr"], "value": "each matrix at its better of CSR and the best block "
                   "size", "l2": "256 MiB write before every product (untimed)"},
        "register_blocking": per,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ autograd

def run_autograd(args, rank, world, local_rank):
    import torch

    import paper_1302_1078_gb300 as gbs

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    A = synth.rmat(20, ef=16, seed=synth.BASE_SEED + 3 + 1000 * rank, vals="u0.5_1.5")
    rp = torch.from_numpy(A.row_ptr).to(dev)
    ci = torch.from_numpy(A.col_idx).to(dev)
    stream = torch.cuda.current_stream(dev)
    op = gbs.CsrOperator(rp, ci, A.n, tune=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    op.tplan  # the one-time transpose
    e1.record(stream)
    torch.cuda.synchronize(dev)
    transpose_ms = e0.elapsed_time(e1)
    results = []
    for dtype in (torch.float64, torch.float32):
        v = torch.from_numpy(A.vals).to(dev).to(dtype)
        for k in (1, 8):
            X = torch.from_numpy(synth.uniform(A.n * k, seed=5, stream=k)).to(dev).to(dtype)
            X = X if k == 1 else X.reshape(A.n, k)
            W = torch.rand((A.m,) if k == 1 else (A.m, k), dtype=dtype, device=dev)
            op.forward_raw(v, X)
            op.tplan.prepare(dtype, k, tune=True)  # tuned dX plan (one-time, like the forward plan)
            for _ in range(args.warmup):
                op.forward_raw(v, X)
                op.tplan.backward(v, X, W)
            torch.cuda.synchronize(dev)
            fwd, bwd = [], []
            for _ in range(args.steps):
                a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                a.record(stream)
                op.forward_raw(v, X)
                b.record(stream)
                op.tplan.backward(v, X, W)
                c.record(stream)
                fwd.append((a, b))
                bwd.append((b, c))
            torch.cuda.synchronize(dev)
            f = statistics.mean(x.elapsed_time(y) for x, y in fwd)
            bw = statistics.mean(x.elapsed_time(y) for x, y in bwd)
            results.append({"dtype": str(dtype).replace("torch.", ""), "k": k, "fwd_ms": f, "bwd_ms": bw,
                            "bwd_over_fwd": bw / f, "fwd_gflops": 2.0 * A.nnz * k / (f * 1e-3) / 1e9,
                            "bwd_gflops": 4.0 * A.nnz * k / (bw * 1e-3) / 1e9,
                            "fwd_config": op.plan(dtype, k).config, "dX_config": op.tplan.config(dtype, k)})
    main_r = results[0]
    line = {
        "metric": METRIC, "value": main_r["fwd_gflops"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": main_r["fwd_ms"] + main_r["bwd_ms"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT["autograd"], "m": A.m, "nnz": A.nnz},
        "transpose_ms_one_time": transpose_ms, "autograd": results,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="spmv", choices=["spmv", "spmm", "small", "batched", "autograd", "rcm", "bcsr"])
    ap.add_argument("--impl", default="gbspmv", choices=["gbspmv", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--shard", action="store_true", help="batched: split one batch across ranks (strong scaling)")
    ap.add_argument("--config", default=None,
                    help='spmv/spmm: one fixed configuration for every product instead of the tuner\'s, as JSON '
                         '(e.g. \'{"variant": 3, "lanes": 4, "threads": 128}\'); for profiling runs')
    ap.add_argument("--only", default=None,
                    help="spmv/spmm: comma-separated matrix names to keep (e.g. stencil3d_100); for profiling runs")
    ap.add_argument("--batch-size", type=int, default=512,
                    help="batched: matrices per batch (512 is the benchmark configuration; smaller for profiling)")
    ap.add_argument("--emulate", action="store_true",
                    help="let the tuner run part of the FP64 products on the FP32 pipe (float-float, within the "
                         "FP64 accuracy bound); off by default, so the default line is native FP64 arithmetic")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus)))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if world != args.gpus and "WORLD_SIZE" not in os.environ:
        world = 1
    if args.warmup < 3 and args.impl != "reference":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload == "batched":
        return run_batched(args, rank, world, local_rank)
    if args.workload == "autograd":
        return run_autograd(args, rank, world, local_rank)
    if args.workload == "rcm":
        return run_rcm(args, rank, world, local_rank)
    if args.workload == "bcsr":
        return run_bcsr(args, rank, world, local_rank)
    return run_gpu(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
