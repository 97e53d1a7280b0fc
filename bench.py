#!/usr/bin/env python3
"""Benchmark: GB300 symbolic LU (gSoFa method); default workload the 1024^2
nested-dissection 5-point grid (n = 1,048,576), the largest single-matrix workload.

One step = one pass of the whole hot path over the matrix: CSR validation,
maxId traversal of every source row, supernode detection, L/U CSR emission
(one ``gsofa_symbolic_device`` call on device-resident input).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload nd1024|grid3d|grid2d|batch512|served]

Prints ONE JSON line (rank 0).  ``value`` is nnz(L+U) per second over all
ranks (each rank factors its own replica: the method needs no exchange);
``e2e`` is the same metric through ``gsofa_symbolic`` with host buffers
(pinned input, host->device and device->host copies inside the timed region);
``roofline`` relates the traversal kernel's algorithmic bytes to the measured
HBM copy bandwidth; ``cpu_baseline`` times the CPU oracle on a row sample.
``--impl reference`` times the CPU oracle itself as the reference arm.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "nd512": (-1, "grid2d_nd_512x512_p0.8"),  # the served stream's large request (first of its pool)
    "grid3d": (1, "grid3d_32^3_p0.6_extra1024"),
    "grid2d": (0, "grid2d_64x64_p0.7"),
    "nd1024": (2, "grid2d_nd_1024x1024_p0.8"),
    "batch512": (3, "batch512_mix"),
    "served": (4, "served_poisson_mix"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="nd1024", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--requests", type=int, default=20000, help="served: stream length")
    ap.add_argument("--rate-frac", type=float, default=0.7, help="served: arrival rate / saturated req/s")
    ap.add_argument("--streams", type=int, default=2, help="served: server stream slots")
    ap.add_argument("--max-batch", type=int, default=512, help="served: requests per batch at most")
    ap.add_argument("--opt", action="append", default=[], help="library option NAME=VALUE (repeatable)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(t: float, world: int, device) -> float:
    """Largest value of t over the ranks (the timed region of the slowest replica).
    Replicas share nothing else: this is the only cross-rank operation."""
    if world <= 1:
        return t
    import torch
    x = torch.tensor([t], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(x, op=torch.distributed.ReduceOp.MAX)
    return float(x.item())


def sum_over_ranks(x: float, world: int, device) -> float:
    """Sum of x over the ranks (whole-job totals of independent replicas)."""
    if world <= 1:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.SUM)
    return float(t.item())


L2_NOTE = "GPU arm: L2 flushed between steps (256 MB write)"


def workload_matrix(k):
    """The CSR of a single-matrix workload (k < 0: the 512^2 ND grid of the served pool)."""
    import synth
    if k < 0:
        return synth.grid2d_nd(512, 0.8, seed=synth.config_seed(4), name="served_nd512_0")
    return synth.config(k)


def workload_config(name, A, nnz_lu, extra, world):
    """The `config` object of both arms (the GPU line and the reference line)."""
    return {"workload": name, "n": int(A.n), "nnz_A": int(A.nnz), "nnz_LU": int(nnz_lu), "options": extra,
            "l2": L2_NOTE, "parallelism": f"replicas x{world}"}


def kernel_source_digest():
    """SHA-256 of the traversal kernel sources; a stored DRAM-traffic figure is
    reported only for the kernel build it was measured on."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2007_00840_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.startswith("traverse_") or f == "internal.cuh":
            h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()


def stored_traffic(name):
    """DRAM bytes per traversal launch from profiles/traffic.json, if it was
    measured on the current kernel sources (else None)."""
    try:
        ent = json.load(open(os.path.join(ROOT, "profiles", "traffic.json"))).get(name)
    except Exception:
        return None
    if not isinstance(ent, dict) or ent.get("kernel_sources_sha256") != kernel_source_digest():
        return None
    return ent.get("bytes_per_launch")


def algorithmic_bytes(vscan, escan, nnz_rows, n):
    """Per-row minimum work of a fill-path search (oracle counts) summed over rows:
    8 B per expanded vertex (two row pointers), 4 B column + 4 B maxId per scanned
    adjacency entry, 4 B per output column, plus 16 B of per-row metadata."""
    return float(8 * vscan.sum() + 8 * escan.sum() + 4 * nnz_rows.sum() + 16 * n)


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in out.strip().splitlines():
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(A, stride: int, min_wall: float = 1.0):
    """The CPU oracle, as it stands, on every `stride`-th row, all host cores;
    the sample is repeated until it has run for min_wall seconds (a workload of
    a few milliseconds gives no stable rate alone)."""
    import oracle
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    rows = np.arange(0, A.n, stride, dtype=np.int32)
    reps, nnz = 0, 0
    t0 = time.perf_counter()
    while True:
        r = oracle.symbolic(A, rows=rows, nthreads=cores)
        nnz += int(r["L_rowptr"][-1] + r["U_rowptr"][-1])
        reps += 1
        dt = time.perf_counter() - t0
        if dt >= min_wall:
            break
    return {"value": nnz / dt, "unit": "nnz(L+U)/s", "cores": cores, "kind": "oracle",
            "sample": f"every {stride}th row ({rows.size} of {A.n} rows) x {reps} passes, "
                      f"{nnz} nnz(L+U), {dt:.2f} s wall",
            "rows_per_s": reps * rows.size / dt, "nnz": nnz // reps}


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle timed on the host cores (rank 0 only), on the
    same rows as the GPU arm (every row of the workload)."""
    import synth
    if rank != 0:
        return 0
    if args.workload in ("batch512", "served"):
        print(json.dumps({"impl": "reference", "unavailable":
                          "the reference arm times single-matrix workloads; use --workload nd1024|grid3d|grid2d"}))
        return 0
    k, name = WORKLOADS[args.workload]
    A = workload_matrix(k)
    extra = {kv.split("=")[0]: int(kv.split("=")[1]) for kv in args.opt}
    for _ in range(args.warmup):
        cpu_baseline(A, 16, min_wall=0.0)
    vals, rows = [], []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        cb = cpu_baseline(A, 1, min_wall=0.0)
        vals.append(cb["value"])
        rows.append(cb["rows_per_s"])
    wall = time.perf_counter() - t0
    v = statistics.median(vals)
    line = {
        "impl": "reference", "metric": "nnz(L+U)/s", "value": v, "unit": "nnz(L+U)/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * wall / max(args.steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic (seeded)",
        "config": workload_config(name, A, cb["nnz"], extra, world),
        "cpu_baseline": {"value": v, "unit": "nnz(L+U)/s", "cores": cb["cores"], "kind": "oracle",
                         "sample": cb["sample"]},
        "e2e": {"value": v, "unit": "nnz(L+U)/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "rows_per_s": statistics.median(rows),
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import paper_2007_00840_gb300 as gs
    from paper_2007_00840_gb300 import build as gbuild
    import synth

    if not torch.cuda.is_available():
        print(json.dumps({"error": "no CUDA device"}))
        return 1
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    gbuild.build()
    gs.load()

    if args.workload == "batch512":
        return run_batch_bench(args, rank, world, local)
    if args.workload == "served":
        return run_served_bench(args, rank, world, local)
    k, name = WORKLOADS[args.workload]
    A = workload_matrix(k)
    n = A.n
    dev = torch.device("cuda", local)
    rp = torch.from_numpy(A.rowptr).to(dev)
    ci = torch.from_numpy(A.colidx).to(dev)
    stream = torch.cuda.current_stream(dev)
    extra = {kv.split("=")[0]: int(kv.split("=")[1]) for kv in args.opt}
    opts = gs.options(collect_stats=2, **extra)  # phase times; the work counters come from one extra call
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # 256 MB > 129 MB L2

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    # warm-up (also sizes the row pool and JIT-free first-touch of every kernel)
    for _ in range(args.warmup):
        r = gs.symbolic_device(rp, ci, opts=opts, stream=stream)
        del r
    torch.cuda.synchronize(dev)

    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    trav_ms, launches, nnz_step, stats0 = [], 0, 0, None
    barrier()
    w0 = time.perf_counter()
    for s in range(args.steps):
        flush.fill_(s & 0xFF)  # evict L2 between steps (outside the step's events)
        ev0[s].record(stream)
        r = gs.symbolic_device(rp, ci, opts=opts, stream=stream)
        ev1[s].record(stream)
        trav_ms.append(r.stats["ms_traverse_smem"] + r.stats["ms_traverse_global"])
        launches += r.stats["kernel_launches"]
        nnz_step = r.nnz_L + r.nnz_U
        stats0 = r.stats
        del r
    barrier()
    wall = time.perf_counter() - w0
    clocks = sampler.stop() if sampler else None
    # work counters (expanded vertices, scanned entries) from one untimed call that records them
    r = gs.symbolic_device(rp, ci, opts=gs.options(collect_stats=1, **extra), stream=stream)
    work = {k2: r.stats[k2] for k2 in ("vertices_expanded", "edges_scanned")}
    del r
    torch.cuda.synchronize(dev)
    step_ms = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    t_dev = sum(step_ms) / 1000.0
    t_dev = max_over_ranks(t_dev, world, dev)
    value = world * args.steps * nnz_step / t_dev
    rows_per_s = world * args.steps * n / t_dev

    # end to end through the host entry point: pinned input, copies in the timed region
    e2e = None
    if not args.no_e2e:
        h_rp = torch.from_numpy(A.rowptr).pin_memory().numpy()
        h_ci = torch.from_numpy(A.colidx).pin_memory().numpy()
        for _ in range(2):
            gs.free_raw(gs.symbolic_host_raw(h_rp, h_ci))
        ts = []
        for _ in range(args.steps):
            flush.fill_(1)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            raw = gs.symbolic_host_raw(h_rp, h_ci)
            ts.append(time.perf_counter() - t0)
            nnz_h = raw.nnz_L + raw.nnz_U
            nsup = raw.n_super
            gs.free_raw(raw)
        te = sum(ts)
        te = max_over_ranks(te, world, dev)
        h2d = 4 * (n + 1) + 4 * A.nnz
        d2h = 16 * (n + 1) + 4 * nnz_h + 4 * n + 4 * (nsup + 1)
        e2e = {"value": world * args.steps * nnz_h / te, "unit": "nnz(L+U)/s",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "ms_per_step": 1000.0 * te / args.steps}

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0

    import oracle
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    # algorithmic bytes of the traversal launch from the oracle's per-row minimum work
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    orc = oracle.symbolic(A, nthreads=cores)
    nnz_rows = np.diff(orc["L_rowptr"]) + np.diff(orc["U_rowptr"])
    alg = algorithmic_bytes(orc["vscan"], orc["escan"], nnz_rows, n)
    t_trav = statistics.mean(trav_ms) / 1000.0
    achieved = alg / t_trav / 1e9
    # DRAM bytes per launch from an ncu capture of this kernel source (default options only)
    traffic = stored_traffic(name) if not extra else None

    # the dominant traversal tier of this matrix
    if stats0["ms_traverse_global"] > stats0["ms_traverse_smem"]:  # the class-ordered kernel's time
        kernel_name = "trav_class_kernel (class-ordered maxId traversal on a visited bitmap, one warp per source)"
    else:
        kernel_name = "trav_smem_kernel (maxId traversal, one CTA per source)"
    line = {
        "metric": "nnz(L+U)/s", "value": value, "unit": "nnz(L+U)/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * t_dev / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic (seeded)",
        "config": workload_config(name, A, nnz_step, extra, world),
        "rows_per_s": rows_per_s,
        "wall_s": wall,
        "e2e": e2e,
        "gpu_launches": launches,
        "roofline": {"bound": "hbm", "kernel": kernel_name,
                     "achieved": achieved, "peak": hbm_peak, "unit": "GB/s", "frac": achieved / hbm_peak,
                     "peak_source": f"{peak_src} (copy bandwidth, burst)", "traffic": traffic,
                     "algorithmic_bytes_per_launch": alg, "ms_per_launch": t_trav * 1000.0},
        "clocks": clocks,
        "stats": {**{k2: stats0[k2] for k2 in ("ms_validate", "ms_traverse", "ms_traverse_smem", "ms_traverse_global",
                                               "ms_supernode", "ms_emit", "ms_total", "pool_retries")}, **work},
        "oracle_min_work": {"vscan": int(orc["vscan"].sum()), "escan": int(orc["escan"].sum())},
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(A, 1)
        if args.workload in ("grid2d", "grid3d"):
            # the same oracle on one host core, on a row sample
            import oracle
            stride = 8 if args.workload == "grid3d" else 1
            rows1 = np.arange(0, A.n, stride, dtype=np.int32)
            t0 = time.perf_counter()
            r1 = oracle.symbolic(A, rows=rows1, nthreads=1)
            dt1 = time.perf_counter() - t0
            nnz1 = int(r1["L_rowptr"][-1] + r1["U_rowptr"][-1])
            line["cpu_baseline"]["single_thread"] = {
                "value": nnz1 / dt1, "unit": "nnz(L+U)/s", "cores": 1,
                "sample": f"every {stride}th row ({rows1.size} rows, {nnz1} nnz(L+U)), {dt1:.2f} s"}
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def _peak_hbm():
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(peaks["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _oracle_alg_bytes(mats, cores):
    import oracle
    tot = 0.0
    for A in mats:
        r = oracle.symbolic(A, nthreads=cores)
        nnz_rows = np.diff(r["L_rowptr"]) + np.diff(r["U_rowptr"])
        tot += algorithmic_bytes(r["vscan"], r["escan"], nnz_rows, A.n)
    return tot


def run_batch_bench(args, rank, world, local):
    """512 matrices of uneven size per gsofa_batch call (one persistent traversal launch)."""
    import torch
    import paper_2007_00840_gb300 as gs
    from paper_2007_00840_gb300 import build as gbuild
    import synth
    torch.cuda.set_device(local)
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    gbuild.build()
    mats = synth.config(3)
    dev = torch.device("cuda", local)
    dmats = [(torch.from_numpy(A.rowptr).to(dev), torch.from_numpy(A.colidx).to(dev)) for A in mats]
    rows = sum(A.n for A in mats)
    extra = {kv.split("=")[0]: int(kv.split("=")[1]) for kv in args.opt}
    opts = gs.options(**{"collect_stats": 2, "autotune": 1, **extra})
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    import tempfile
    tune_file = os.path.join(tempfile.mkdtemp(prefix="gsofa_tune_"), "shapes.txt")
    os.environ["GSOFA_TUNE_FILE"] = tune_file  # the autotuner appends the shape it picks
    for _ in range(max(args.warmup, 1)):
        res = gs.batch_device(dmats, opts=opts)
        del res
    torch.cuda.synchronize(dev)
    tuned = None
    if os.path.exists(tune_file):
        f = open(tune_file).read().split()
        if len(f) >= 7:
            tuned = {"threads_per_source": int(f[1]), "ctas_per_sm": int(f[2]), "list_capacity": int(f[3]),
                     "work_chunk": int(f[4]), "kernel": ["cta_per_source_bfs", "warp_per_source_class"][int(f[5])],
                     "class_slots": int(f[6]), "fill_first": int(f[7]) if len(f) >= 8 else 0}
    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    nnz, trav, launches = 0, [], 0
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    for s_ in range(args.steps):
        flush.fill_(s_ & 0xFF)
        e0[s_].record(stream)
        res = gs.batch_device(dmats, opts=opts)
        e1[s_].record(stream)
        nnz = sum(r.nnz_L + r.nnz_U for r in res)
        trav.append(res[0].stats["ms_traverse"])
        launches += res[0].stats["kernel_launches"]
        del res
    torch.cuda.synchronize(dev)
    clocks = sampler.stop() if sampler else None
    t = sum(a.elapsed_time(b) for a, b in zip(e0, e1)) / 1000.0
    t = max_over_ranks(t, world, dev)
    # end to end: pinned host CSRs in, every result array back to the host
    e2e = None
    if not args.no_e2e:
        hmats = [(torch.from_numpy(A.rowptr).pin_memory(), torch.from_numpy(A.colidx).pin_memory()) for A in mats]
        ts = []
        # device staging buffers reused every step (as a pipeline would), so the
        # batch plan and its captured graph are reused too
        dm = [(torch.empty_like(a, device=dev), torch.empty_like(b, device=dev)) for a, b in hmats]
        for it in range(1 + max(1, args.steps // 2)):  # the first pass (pinned host blocks) is not timed
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            for (da, db), (a, b) in zip(dm, hmats):
                da.copy_(a, non_blocking=True)
                db.copy_(b, non_blocking=True)
            res = gs.batch_device(dm, opts=opts)
            outs = gs.results_to_host(res)
            if it > 0:
                ts.append(time.perf_counter() - t0)
            d2h = sum(8 * (o.n + 1) * 2 + 4 * (o.nnz_L + o.nnz_U) + 4 * o.n + 4 * (o.n_super + 1) for o in outs)
            del res, outs
        h2d = sum(4 * (A.n + 1) + 4 * A.nnz for A in mats)
        te = max_over_ranks(sum(ts), world, dev)
        e2e = {"value": world * len(ts) * nnz / te, "unit": "nnz(L+U)/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": 1000 * sum(ts) / len(ts)}
    if rank != 0:
        return 0
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    alg = _oracle_alg_bytes(mats, cores)
    t_trav = statistics.mean(trav) / 1000.0
    if t_trav <= 0:
        t_trav = t / args.steps  # whole step as an upper bound when the launch was not timed
    peak, src = _peak_hbm()
    # CPU baseline: the oracle on every 16th matrix (all rows)
    import oracle
    sample = mats[::16]
    t0 = time.perf_counter()
    cnnz = 0
    for A in sample:
        r = oracle.symbolic(A, nthreads=cores)
        cnnz += int(r["L_rowptr"][-1] + r["U_rowptr"][-1])
    dt = time.perf_counter() - t0
    line = {
        "metric": "nnz(L+U)/s", "value": world * args.steps * nnz / t, "unit": "nnz(L+U)/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * t / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic (seeded)",
        "config": {"workload": "batch512_mix", "matrices": len(mats), "rows": rows, "nnz_LU": int(nnz),
                   "options": extra, "tuned_shape": tuned,
                   "l2": "flushed between steps (256 MB write)", "parallelism": f"replicas x{world}"},
        "rows_per_s": world * args.steps * rows / t, "matrices_per_s": world * args.steps * len(mats) / t,
        "e2e": e2e, "gpu_launches": launches,
        "roofline": {"bound": "hbm", "kernel": ("trav_class_kernel (batched, class-ordered, one warp per source)"
                                                if tuned and tuned["kernel"] == "warp_per_source_class"
                                                else "trav_smem_kernel (batched, one CTA per source)"),
                     "achieved": alg / t_trav / 1e9,
                     "peak": peak, "unit": "GB/s", "frac": alg / t_trav / 1e9 / peak, "traffic": None,
                     "peak_source": f"{src} (copy bandwidth, burst)", "algorithmic_bytes_per_launch": alg,
                     "ms_per_launch": t_trav * 1000},
        "clocks": clocks,
        "cpu_baseline": {"value": cnnz / dt, "unit": "nnz(L+U)/s", "cores": cores, "kind": "oracle",
                         "sample": f"every 16th matrix ({len(sample)} matrices, all rows), {dt:.2f} s wall"},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_served_bench(args, rank, world, local):
    """Poisson stream of requests (the 512-matrix mix plus 2% ND grids of order 262,144)."""
    import torch
    import paper_2007_00840_gb300 as gs
    from paper_2007_00840_gb300 import build as gbuild
    import synth
    torch.cuda.set_device(local)
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    gbuild.build()
    dev = torch.device("cuda", local)
    small, big = synth.served_pool()
    pool = small + big
    dpool = [(torch.from_numpy(A.rowptr).to(dev), torch.from_numpy(A.colidx).to(dev)) for A in pool]
    # batched throughput of the small mix sets the arrival rate
    opts = gs.options(autotune=1)
    for _ in range(2):
        res = gs.batch_device(dpool[:len(small)], opts=opts)
        del res
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    res = gs.batch_device(dpool[:len(small)], opts=opts)
    torch.cuda.synchronize(dev)
    t_small = (time.perf_counter() - t0) / len(small)
    batched_rps = 1.0 / t_small
    del res
    # the large requests run on their own; their mean service time enters the rate
    r = gs.symbolic_device(*dpool[len(small)])
    torch.cuda.synchronize(dev)
    del r
    t0 = time.perf_counter()
    for j in range(len(big)):
        r = gs.symbolic_device(*dpool[len(small) + j])
        torch.cuda.synchronize(dev)
        del r
    t_big = (time.perf_counter() - t0) / len(big)
    mean_service = 0.98 * t_small + 0.02 * t_big
    # saturated served throughput: a burst of requests submitted at once
    nreq = args.requests
    burst = min(2000, nreq)
    which_b, _ = synth.served_choices(burst, len(small), len(big), seed=5)
    srv = gs.Server(streams=args.streams, max_batch=args.max_batch, mem_cap_bytes=150 << 30)
    t0 = time.perf_counter()
    tk = [srv.submit(*dpool[int(k)]) for k in which_b]
    for t_ in tk:
        srv.wait(t_, keep_result=False)
    sat_rps = burst / (time.perf_counter() - t0)
    srv.close()
    lam = args.rate_frac * sat_rps
    which, arrivals = synth.served_choices(nreq, len(small), len(big), seed=4)
    arrivals = arrivals / lam
    # every pattern of the pool run alone: each served result is compared with it
    # on the device after the stream (the comparison is outside the latency)
    ref = [gs.symbolic_device(*d) for d in dpool]
    torch.cuda.synchronize(dev)
    srv = gs.Server(streams=args.streams, max_batch=args.max_batch, mem_cap_bytes=150 << 30, opts=gs.options())
    sampler = ClockSampler(local)
    sampler.start()
    tickets = []
    start = time.perf_counter()
    for i in range(nreq):
        due = start + arrivals[i]
        while time.perf_counter() < due:
            pass
        tickets.append(srv.submit(*dpool[int(which[i])]))
    mismatches = 0
    lat_small, lat_large = [], []
    for i, t in enumerate(tickets):
        r, lat = srv.wait(t, keep_result=True)
        (lat_large if int(which[i]) >= len(small) else lat_small).append(lat)
        g = ref[int(which[i])]
        for f in ("L_rowptr", "L_colidx", "U_rowptr", "U_colidx", "fill_count", "super_start"):
            if not torch.equal(getattr(r, f), getattr(g, f)):
                mismatches += 1
                break
        del r
    wall = time.perf_counter() - start
    clocks = sampler.stop()
    st = srv.stats()
    srv.close()
    # end to end: a shorter stream at the same rate with host CSR in and every
    # result array copied back to the host
    e2e = None
    if not args.no_e2e:
        ne = min(2000, nreq)
        hpool = [(torch.from_numpy(A.rowptr).pin_memory().numpy(), torch.from_numpy(A.colidx).pin_memory().numpy())
                 for A in pool]
        srv = gs.Server(streams=args.streams, max_batch=args.max_batch, mem_cap_bytes=150 << 30, opts=gs.options())
        h2d = d2h = nnz_e = 0
        tickets = []
        start = time.perf_counter()
        for i in range(ne):
            due = start + arrivals[i]
            while time.perf_counter() < due:
                pass
            k = int(which[i])
            tickets.append(srv.submit(*hpool[k]))
            h2d += 4 * (pool[k].n + 1) + 4 * pool[k].nnz
        for t in tickets:
            r, _ = srv.wait(t)
            h = r.to_host()
            nnz_e += h.nnz_L + h.nnz_U
            d2h += 16 * (h.n + 1) + 4 * (h.nnz_L + h.nnz_U) + 4 * h.n + 4 * (h.n_super + 1)
            del r
        te = time.perf_counter() - start
        srv.close()
        te = max_over_ranks(te, world, dev)
        e2e = {"value": sum_over_ranks(nnz_e, world, dev) / te, "unit": "nnz(L+U)/s",
               "h2d_bytes_per_step": h2d / ne, "d2h_bytes_per_step": d2h / ne, "requests": ne,
               "note": "per request: host CSR submitted, result copied back"}
    span = max_over_ranks(st["span_s"], world, dev)
    total_nnz = sum_over_ranks(st["total_nnz"], world, dev)
    total_rows = sum_over_ranks(st["total_rows"], world, dev)
    completed = sum_over_ranks(st["completed"], world, dev)
    launches_all = sum_over_ranks(st["kernel_launches"], world, dev)
    if rank != 0:
        torch.distributed.destroy_process_group()
        return 0
    line = {
        "metric": "nnz(L+U)/s", "value": total_nnz / span, "unit": "nnz(L+U)/s", "n_gpus": world,
        "steps": nreq, "warmup": 2, "ms_per_step": 1000 * st["span_s"] / nreq, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic (seeded)",
        "config": {"workload": "served_poisson_mix", "requests": nreq, "rate_per_s": lam,
                   "rate": f"{args.rate_frac} x saturated served throughput ({sat_rps:.1f} req/s; batched small "
                           f"{1000 * t_small:.3f} ms/request, large alone {1000 * t_big:.1f} ms)",
                   "batched_small_req_per_s": batched_rps, "big_fraction": 0.02,
                   "mem_cap_bytes": 150 << 30, "streams": args.streams, "max_batch": args.max_batch},
        "requests_per_s": completed / span, "rows_per_s": total_rows / span, "e2e": e2e,
        "gpu_launches": int(launches_all), "latency_scope": "rank 0" if world > 1 else "all requests",
        "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "max_ms": st["max_ms"], "batches": st["batches"],
        "peak_projected_mem_bytes": st["peak_mem_in_use"], "peak_device_bytes": st["peak_device_bytes"],
        "completed": st["completed"], "failed": st["failed"],
        "latency_by_kind_ms": {
            "small": {"count": len(lat_small), "p50": float(np.percentile(lat_small, 50)) if lat_small else None,
                      "p99": float(np.percentile(lat_small, 99)) if lat_small else None},
            "large_nd512": {"count": len(lat_large), "p50": float(np.percentile(lat_large, 50)) if lat_large else None,
                            "p99": float(np.percentile(lat_large, 99)) if lat_large else None}},
        "checked_against_alone": nreq, "mismatches": mismatches, "wall_s": wall, "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
