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
an end-to-end figure through the public API with host buffers (with the
host-to-device copy rate measured alone), the CPU oracle timed on the host
cores, and the SM clocks sampled during timing.  The same line carries the
rest of the metric, each part timed with its own CUDA events after an L2
flush: "spmm" (Sec. 5: k = 4, 8, 16 on the sweep's matrices), "batched" (512
uneven matrices, k = 8, one graph-replayed persistent launch against the
per-matrix launch loops: batched_vs_looped) and "autograd" (R-MAT scale 20:
forward, backward, bwd_over_fwd).  --sweep-only skips those three.

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
    1: ["rows_kernel.cuh", "device_common.cuh", "launch_impl.cuh"],
    2: ["merge_kernel.cuh", "device_common.cuh", "launch_impl.cuh"],
    3: ["rows_tma.cuh", "rows_kernel.cuh", "device_common.cuh", "df64.cuh", "launch_impl.cuh"],
    4: ["merge_kernel.cuh", "device_common.cuh", "launch_impl.cuh"],
    5: ["rows_kernel.cuh", "device_common.cuh", "launch_impl.cuh"],
}


def kernel_source_hash(variant: int) -> str:
    import hashlib

    h = hashlib.sha256()
    for f in KERNEL_SOURCES.get(variant, []):
        with open(os.path.join(ROOT, "paper_1302_1078_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_key(variant: int, relabel: int = 0) -> str:
    """Key of a configuration in profiles/traffic.txt: the variant, with rN appended for a plan that
    relabels its columns (gbs_config.relabel N)."""
    return f"{variant}r{relabel}" if relabel else str(variant)


def recorded_traffic(variant: int, matrix: str, relabel: int = 0):
    """DRAM bytes per launch from profiles/traffic.txt (lines: key hash bytes matrix command...),
    or None when no capture matches the configuration and the current kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    want = kernel_source_hash(variant)
    key = traffic_key(variant, relabel)
    for line in open(path):
        f = line.split()
        if len(f) >= 4 and not line.startswith("#") and f[0] == key and f[1] == want and f[3] == matrix:
            return float(f[2])
    return None


def compulsory_bytes(m, n, nnz, k, es=8):
    """Sec. 4.2 / Sec. 5 application-bandwidth model with (m+1) row pointers:
    es*nnz + 4*nnz + 4*(m+1) + es*n*k + es*m*k."""
    return (es + 4) * nnz + 4 * (m + 1) + es * n * k + es * m * k


def measured_hbm_peak():
    """(GB/s, source): the measured HBM copy bandwidth (MEASURED_PEAKS.json hbm_gbs), else the fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        v = json.load(open(path)).get("hbm_gbs")
        if v:
            return float(v), "measured"
    return 6800.0, "fallback"


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
        if t_total >= budget_s or sweeps >= 1000:
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
    """Kernels one product call launches: ROWS and ROWS_TMA 1 per column panel; MERGE partition
    is precomputed by the plan, then kernel + carry fix-up per panel; a relabelling plan adds
    the scatter of x into the relabelled order."""
    panel = 32 * dtype_vec if k > 1 else 1
    panels = (k + panel - 1) // panel
    return panels * (1 if cfg["variant"] in (1, 3) else 2) + (1 if cfg.get("relabel", 0) else 0)


def measure_spmm(gbs, torch, dev, items, steps, warmup, ks=(4, 8, 16)):
    """SpMM Y = A X (Sec. 5) at k in `ks` on the sweep's resident matrices, each product through
    an autotuned plan, timed cold (256 MiB L2 flush before every product) with CUDA events."""
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    hbm_peak = measured_hbm_peak()[0]
    out = []
    sampler = ClockSampler(gpu_smi_id(torch, dev.index or 0))
    for it in items:
        A = it["A"]
        for k in ks:
            X = torch.from_numpy(synth.uniform(A.n * k, seed=synth.BASE_SEED + 12, stream=k).reshape(A.n, k)).to(dev)
            Y = torch.empty((A.m, k), dtype=torch.float64, device=dev)
            plan = gbs.Plan(it["rp"], it["ci"], A.n, torch.float64, k, tune=True)
            for _ in range(warmup):
                plan.spmm(it["v"], X, Y)
            torch.cuda.synchronize(dev)
            if not sampler.rows:
                sampler.start()
                time.sleep(0.05)
            evs = []
            for _ in range(steps):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                plan.spmm(it["v"], X, Y)
                b.record(stream)
                evs.append((a, b))
            torch.cuda.synchronize(dev)
            ms = statistics.mean(a.elapsed_time(b) for a, b in evs)
            by = compulsory_bytes(A.m, A.n, A.nnz, k)
            out.append({"matrix": it["name"], "k": k, "ms": ms, "flops": 2.0 * A.nnz * k, "bytes": by,
                        "gflops": 2.0 * A.nnz * k / ms / 1e6, "hbm_frac": by / ms / 1e6 / hbm_peak,
                        "config": plan.config})
            del plan, X, Y
    sampler.stop()
    return {"products": out, "clocks": sampler.summary(), "steps": steps}


def reduce_max(torch, dev, values, world):
    """Element-wise maximum of a list of floats over the ranks."""
    if world == 1 or not values:
        return list(values)
    import torch.distributed as dist

    t = torch.tensor(values, dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t]


def host_numa_info(torch, dev_index: int) -> dict:
    """Where the host side of the end-to-end copies lives: the CPUs this process may run on, and
    the NUMA node of those CPUs and of the GPU's PCI function (Linux sysfs; empty where absent)."""
    info = {}
    try:
        cpus = sorted(os.sched_getaffinity(0))
        info["process_cpus"] = f"{cpus[0]}-{cpus[-1]} ({len(cpus)})" if cpus else ""
        nodes = set()
        for c in cpus:
            for d in os.listdir(f"/sys/devices/system/cpu/cpu{c}"):
                if d.startswith("node") and d[4:].isdigit():
                    nodes.add(int(d[4:]))
        info["process_cpu_numa_nodes"] = sorted(nodes)
    except OSError:
        pass
    try:
        p = torch.cuda.get_device_properties(dev_index)
        bus = f"{p.pci_domain_id:04x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0"
        with open(f"/sys/bus/pci/devices/{bus}/numa_node") as fh:
            info["gpu_pci_numa_node"] = int(fh.read().strip())
    except (OSError, ValueError, AttributeError):
        pass
    return info


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

    # ---- the host-to-device copy rate alone: the step's input copies from the same pinned
    # buffers on the same copy stream, nothing else running (best of three passes)
    h2d_ms = []
    for _ in range(3):
        torch.cuda.synchronize(dev)
        hc0, hc1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        hc0.record(h2d_stream)
        with torch.cuda.stream(h2d_stream):
            for it, hb in zip(items, pinned):
                it["rp"].copy_(hb["rp"], non_blocking=True)
                it["ci"].copy_(hb["ci"], non_blocking=True)
                it["v"].copy_(hb["v"], non_blocking=True)
                it["X"].copy_(hb["X"], non_blocking=True)
        hc1.record(h2d_stream)
        torch.cuda.synchronize(dev)
        h2d_ms.append(hc0.elapsed_time(hc1))
    h2d_gbs = h2d / (min(h2d_ms) * 1e-3) / 1e9
    del pinned

    # ---- max over ranks
    step_ms_max, e2e_ms_max = reduce_max(torch, dev, [step_ms, e2e_ms], world)

    # ---- per-matrix report, dominant kernel roofline
    hbm_peak, peak_src = measured_hbm_peak()
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
                "traffic": recorded_traffic(d["config"]["variant"], d["matrix"], d["config"].get("relabel", 0))
                if d["k"] == 1 else None,
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
                "d2h_bytes_per_step": d2h, "steps": e2e_steps, "ms_per_step": e2e_ms_max,
                "h2d_gbs_measured": h2d_gbs, "h2d_ms_alone": min(h2d_ms),
                "h2d_bound_ms": h2d / (h2d_gbs * 1e9) * 1e3, "host": host_numa_info(torch, local_rank),
                "note": "pinned host buffers; one untimed warm-up step; copies on their own streams overlap "
                        "the products; h2d_gbs_measured = the step's input copies alone on the copy stream "
                        "(best of three), so h2d_bound_ms is the floor the copies set on ms_per_step"},
        "clocks": sampler.summary(),
        "gpu_launches": launches,
        "fp64_peak_gflops_derived": fp64_peak_gflops, "fp64_probe_gflops": fp64_probe_gflops,
        "fp64_emulation": bool(args.emulate),
        "per_matrix": per,
    }
    # ---- the rest of the metric on the same line: SpMM k = 4, 8, 16 on the sweep's matrices,
    # the 512-matrix batch against its launch loops, and backward / forward on R-MAT 20
    if args.workload == "spmv" and not args.sweep_only and not args.only and not args.config:
        ksteps = max(3, min(args.steps, 20))
        sp = measure_spmm(gbs, torch, dev, [it for it in items if it["k"] == 1], ksteps, args.warmup)
        ms = reduce_max(torch, dev, [p["ms"] for p in sp["products"]], world)
        for p, t_ in zip(sp["products"], ms):
            p["ms"] = t_
            p["gflops"] = p["flops"] / t_ / 1e6
            p["hbm_frac"] = p["bytes"] / t_ / 1e6 / hbm_peak
            p["fp64_frac"] = p["flops"] / t_ / 1e6 / fp64_peak_gflops
        tot_ms = sum(p["ms"] for p in sp["products"])
        line["spmm"] = {"gflops": world * sum(p["flops"] for p in sp["products"]) / (tot_ms * 1e-3) / 1e9,
                        "workload": WORKLOAD_TEXT["spmm"].replace("k in {1,4,8,16}", "k in {4,8,16}"),
                        "steps": sp["steps"], "l2": "256 MiB write before every product (untimed)",
                        "clocks": sp["clocks"],
                        "per_product": [{k_: v_ for k_, v_ in p.items() if k_ not in ("flops", "bytes")}
                                        for p in sp["products"]]}
        b = measure_batched(gbs, torch, dev, args, rank, world, ksteps, args.warmup)
        b["ms"], b["looped_ms"], b["looped_tuned_ms"] = reduce_max(
            torch, dev, [b["ms"], b["looped_ms"], b["looped_tuned_ms"]], world)
        b["flops"], b["bytes"] = b["flops"] * world, b["bytes"] * world
        line["batched"] = batched_report(b, world, hbm_peak, fp64_peak_gflops)
        line["batched"]["workload"] = WORKLOAD_TEXT["batched"]
        line["batched_vs_looped"] = line["batched"]["batched_vs_looped"]
        line["batched_vs_looped_tuned"] = line["batched"]["batched_vs_looped_tuned"]
        ag = measure_autograd(gbs, torch, dev, rank, ksteps, args.warmup)
        fb = reduce_max(torch, dev, [v_ for r_ in ag["results"] for v_ in (r_["fwd_ms"], r_["bwd_ms"])], world)
        for j, r_ in enumerate(ag["results"]):
            r_["fwd_ms"], r_["bwd_ms"] = fb[2 * j], fb[2 * j + 1]
            r_["bwd_over_fwd"] = r_["bwd_ms"] / r_["fwd_ms"]
        line["autograd"] = dict(ag, workload=WORKLOAD_TEXT["autograd"])
        line["bwd_over_fwd"] = {f"{r_['dtype']}_k{r_['k']}": r_["bwd_over_fwd"] for r_ in ag["results"]}
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


def measure_batched(gbs, torch, dev, args, rank, world, steps, warmup, shard=False, batch_size=512):
    """The 512-matrix k = 8 batch (one persistent launch replayed from a CUDA graph) against
    the per-matrix launch loops.  Returns the timings and ratios as a dict (per-rank times;
    the caller reduces them across ranks)."""
    k = 8
    if shard:
        # one batch split across the ranks (strong scaling)
        specs = synth.batch_specs(batch_size)
        costs = [sp.rows * (5 if sp.kind == "stencil2d" else sp.avg) for sp in specs]
        mine = shard_for_rank(costs, world, rank)
    else:
        # every rank its own independent batch (weak scaling)
        specs = synth.batch_specs(batch_size, seed=synth.BASE_SEED + 4 + 1000 * rank)
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
    t_plan0 = time.perf_counter()
    plan = gbs.BatchedPlan(mats, Xs, Ys, tune=True)
    t_plan = time.perf_counter() - t_plan0
    info = plan.info()
    # the baseline a per-matrix user would run: each matrix's own standalone-tuned configuration
    plan_pm = gbs.BatchedPlan(mats, Xs, Ys, tune=True, configs=[None] * len(mats))
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def timed(fn, n):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        for s_ in range(n):
            flush.zero_()
            evs[s_][0].record(stream)
            fn()
            evs[s_][1].record(stream)
        torch.cuda.synchronize(dev)
        return [a.elapsed_time(b) for a, b in evs]

    for _ in range(warmup):
        plan.run()
        plan.run_looped()
        plan_pm.run_looped()
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(gpu_smi_id(torch, dev.index or 0))
    sampler.start()
    time.sleep(0.05)
    torch.cuda.nvtx.range_push("timed_batched")
    t_batched = timed(plan.run, steps)
    torch.cuda.nvtx.range_pop()
    t_looped = timed(plan.run_looped, steps)
    t_looped_pm = timed(plan_pm.run_looped, steps)
    sampler.stop()
    variants = {}
    for c in info["configs"]:
        key = "ROWS" if c["variant"] == 1 else "MERGE"
        variants[key] = variants.get(key, 0) + 1
    ms_b, ms_l, ms_lpm = statistics.mean(t_batched), statistics.mean(t_looped), statistics.mean(t_looped_pm)
    del plan, plan_pm, mats, Xs, Ys
    return {"ms": ms_b, "looped_ms": ms_l, "looped_tuned_ms": ms_lpm, "flops": flops, "bytes": float(bytes_),
            "matrices": len(mine), "grid": info["grid"], "work_items": info["total_items"], "variants": variants,
            "plan_s": t_plan, "clocks": sampler.summary(), "steps": steps}


def batched_report(r, world, hbm_peak, fp64_peak=None):
    """Public fields of a batched measurement (after the cross-rank reduction)."""
    out = {"ms": r["ms"], "gflops": r["flops"] / (r["ms"] * 1e-3) / 1e9,
           "hbm_frac": r["bytes"] / (r["ms"] * 1e-3) / 1e9 / world / hbm_peak,
           "batched_vs_looped": r["looped_ms"] / r["ms"], "looped_ms": r["looped_ms"],
           "looped_gflops": r["flops"] / (r["looped_ms"] * 1e-3) / 1e9,
           "batched_vs_looped_tuned": r["looped_tuned_ms"] / r["ms"], "looped_tuned_ms": r["looped_tuned_ms"],
           "looped_note": "looped = the batch's own per-matrix configurations, one launch per matrix; "
                          "looped_tuned = each matrix's standalone-tuned configuration, one launch per matrix",
           "matrices_per_rank": r["matrices"], "grid": r["grid"], "work_items": r["work_items"],
           "variants": r["variants"], "plan_build_s": r["plan_s"], "steps": r["steps"], "clocks": r["clocks"]}
    if fp64_peak:
        out["fp64_frac"] = r["flops"] / world / (r["ms"] * 1e-3) / 1e9 / fp64_peak
    return out


def run_batched(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    import paper_1302_1078_gb300 as gbs

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    if world > 1:
        dist.barrier()
    r = measure_batched(gbs, torch, dev, args, rank, world, args.steps, args.warmup, shard=args.shard,
                        batch_size=args.batch_size)
    t = torch.tensor([r["ms"], r["looped_ms"], r["looped_tuned_ms"]], dtype=torch.float64, device=dev)
    tot = torch.tensor([r["flops"], r["bytes"]], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(tot, op=dist.ReduceOp.SUM)
    r["ms"], r["looped_ms"], r["looped_tuned_ms"] = float(t[0]), float(t[1]), float(t[2])
    r["flops"], r["bytes"] = float(tot[0]), float(tot[1])
    rep = batched_report(r, world, measured_hbm_peak()[0])
    line = {
        "metric": METRIC, "value": rep["gflops"], "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms"], "higher_is_better": True,
        "scaling": "strong" if args.shard else "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT["batched"].replace("512", str(args.batch_size)),
                   "matrices_per_rank": r["matrices"], "grid": r["grid"], "work_items": r["work_items"],
                   "variants": r["variants"], "l2": "256 MiB write before every step (untimed)"},
        "batched_vs_looped": rep["batched_vs_looped"], "looped_gflops": rep["looped_gflops"],
        "looped_ms": r["looped_ms"], "looped_note": rep["looped_note"],
        "batched_vs_looped_tuned": rep["batched_vs_looped_tuned"], "looped_tuned_ms": r["looped_tuned_ms"],
        "roofline": {"bound": "hbm", "achieved": r["bytes"] / (r["ms"] * 1e-3) / 1e9 / world,
                     "peak": measured_hbm_peak()[0], "unit": "GB/s", "frac": rep["hbm_frac"], "traffic": None,
                     "kernel": "batched_kernel (whole batch per launch)"},
        "clocks": r["clocks"],
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
    hbm_peak = measured_hbm_peak()[0]

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

def measure_autograd(gbs, torch, dev, rank, steps, warmup, dtypes=None):
    """Forward Y = A X and backward (dX = A^T dY, dvals) on R-MAT scale 20, edge factor 16,
    vals uniform[0.5, 1.5], k in {1, 8}; the transpose is built once and timed separately."""
    import torch as _t

    dtypes = dtypes or (_t.float64, _t.float32)
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
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    results = []
    sampler = ClockSampler(gpu_smi_id(torch, dev.index or 0))
    for dtype in dtypes:
        v = torch.from_numpy(A.vals).to(dev).to(dtype)
        for k in (1, 8):
            X = torch.from_numpy(synth.uniform(A.n * k, seed=5, stream=k)).to(dev).to(dtype)
            X = X if k == 1 else X.reshape(A.n, k)
            W = torch.rand((A.m,) if k == 1 else (A.m, k), dtype=dtype, device=dev)
            op.forward_raw(v, X)
            op.tplan.prepare(dtype, k, tune=True)  # tuned dX plan (one-time, like the forward plan)
            for _ in range(warmup):
                op.forward_raw(v, X)
                op.tplan.backward(v, X, W)
            torch.cuda.synchronize(dev)
            if not sampler.rows:
                sampler.start()
                time.sleep(0.05)
            fwd, bwd, bdx, bdv = [], [], [], []
            for _ in range(steps):
                # each pass starts cold, like the sweep's products: the forward after an L2 flush,
                # the backward after another one; the backward's two parts are also timed alone
                a, b, c, d, e, f_, g, h = (torch.cuda.Event(enable_timing=True) for _ in range(8))
                flush.zero_()
                a.record(stream)
                op.forward_raw(v, X)
                b.record(stream)
                flush.zero_()
                c.record(stream)
                op.tplan.backward(v, X, W)
                d.record(stream)
                flush.zero_()
                e.record(stream)
                op.tplan.backward(v, X, W, need_dvals=False)
                f_.record(stream)
                flush.zero_()
                g.record(stream)
                op.tplan.backward(v, X, W, need_dX=False)
                h.record(stream)
                fwd.append((a, b))
                bwd.append((c, d))
                bdx.append((e, f_))
                bdv.append((g, h))
            torch.cuda.synchronize(dev)
            f = statistics.mean(x.elapsed_time(y) for x, y in fwd)
            bw = statistics.mean(x.elapsed_time(y) for x, y in bwd)
            results.append({"dtype": str(dtype).replace("torch.", ""), "k": k, "fwd_ms": f, "bwd_ms": bw,
                            "bwd_dX_alone_ms": statistics.mean(x.elapsed_time(y) for x, y in bdx),
                            "bwd_dvals_alone_ms": statistics.mean(x.elapsed_time(y) for x, y in bdv),
                            "bwd_over_fwd": bw / f, "fwd_gflops": 2.0 * A.nnz * k / (f * 1e-3) / 1e9,
                            "bwd_gflops": 4.0 * A.nnz * k / (bw * 1e-3) / 1e9,
                            "fwd_config": op.plan(dtype, k).config, "dX_config": op.tplan.config(dtype, k)})
    sampler.stop()
    del op
    return {"m": A.m, "nnz": A.nnz, "transpose_ms_one_time": transpose_ms, "results": results,
            "clocks": sampler.summary(), "steps": steps,
            "l2": "256 MiB write before the forward and again before the backward (untimed)"}


def run_autograd(args, rank, world, local_rank):
    import torch

    import paper_1302_1078_gb300 as gbs

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    r = measure_autograd(gbs, torch, dev, rank, args.steps, args.warmup)
    main_r = r["results"][0]
    line = {
        "metric": METRIC, "value": main_r["fwd_gflops"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": main_r["fwd_ms"] + main_r["bwd_ms"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_TEXT["autograd"], "m": r["m"], "nnz": r["nnz"], "l2": r["l2"]},
        "transpose_ms_one_time": r["transpose_ms_one_time"], "autograd": r["results"], "clocks": r["clocks"],
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
    ap.add_argument("--sweep-only", action="store_true",
                    help="spmv: time only the SpMV sweep (no SpMM, batched or autograd sections)")
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
