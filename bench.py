"""Benchmark of the GB300 Friends-of-Friends group finder.

One step = one pass of the whole path (fof_link + fof_groups: binning,
linking, finalisation, outputs, catalogue) over one synthetic box.  The
default workload is the 1024^3-particle clustered box (box side 100, 500,000
Plummer blobs holding half of the particles, l_x = 0.2 x mean separation,
min group size 20).  Prints ONE JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference ...    # the CPU oracle on a bounded sample

Under torchrun each rank runs its own independent box (seed offset by rank):
weak scaling, no collective on the data path; rank 0 prints.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "particles grouped/s"
UNIT = "particles/s"

# Algorithmic bytes per launch of each phase, per particle (p) and per cell
# (c): what the phase must move at least, not what it happens to move.
ALG_BYTES = {
    "bin_count": (12, 0),      # read positions
    "bin_scatter": (28, 0),    # read positions, write binned float4
    "brick_sort": (44, 4),     # read float4, write float4 + parent/minorig/cnt, cell starts
    "link": (20, 4),           # read binned float4 + parent once, cell starts once
    "finalize": (8, 0),        # read parent + own index of non-roots
    "outputs": (20, 0),        # read parent, root data, own index; write ids, sizes
    "catalogue": (4, 0),       # read sizes
    "scan_bricks": (0, 0),
}
# The whole path's algorithmic bytes: 60 per particle + 8 per cell.
PATH_BYTES = (60, 8)


def workloads():
    from paper_2003_11468_gb300 import synth
    return {
        "1024": synth.clustered_1024,
        # 1/64 of the 1024^3 box at the same density, blob recipe and l_x:
        # the small case the per-kernel ncu captures run on
        "1024s": lambda: synth.clustered_sample_of_1024(4),
        "256": synth.clustered_256,
        "32k": synth.uniform_32k,
    }


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2003_11468_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources for this workload; else None."""
    path = os.path.join(ROOT, "profiles", "traffic_by_kernel.txt")
    if not os.path.exists(path):
        return None
    want = source_hash()
    with open(path) as f:
        for line in f:
            parts = line.split()
            if len(parts) >= 4 and not line.startswith("#"):
                k, wl, nbytes, src = parts[:4]
                if k == kernel and wl == workload and src == want:
                    return float(nbytes)
    return None


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rank_seed(seed: int, rank: int) -> int:
    """Every rank groups its own independent box of the same recipe."""
    return seed + 1000 * rank


def max_over_ranks(value: float, world: int, device=None) -> float:
    """The slowest rank's time (all ranks get it); no-op for one rank."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(n_per_rank: int, world: int, seconds: float) -> float:
    """Whole-job throughput: the particles all ranks grouped / the slowest rank's time."""
    return world * n_per_rank / seconds


# ---------------------------------------------------------------------------
# the CPU oracle arm (and the cpu_baseline key)
# ---------------------------------------------------------------------------

_SAMPLES = {}


def cpu_sample(k: int = 8):
    """The oracle on a periodic 1/k^3-volume box of the 1024^3 recipe
    (generated once, then only the oracle is timed)."""
    import oracle
    from paper_2003_11468_gb300 import synth
    if k not in _SAMPLES:
        c = synth.clustered_sample_of_1024(k)
        _SAMPLES[k] = (c, c["make"]())
    c, pos = _SAMPLES[k]
    oracle.build()
    t0 = time.perf_counter()
    ids, sizes = oracle.groups(pos, c["box"], c["l_x"])
    oracle.catalogue(sizes, c["min_size"])
    dt = time.perf_counter() - t0
    return c, dt


def run_reference(args):
    world, rank, _ = dist_setup()
    if rank != 0:
        return 0
    wl = workloads()[args.workload]()
    times = []
    c = None
    for _ in range(args.warmup):
        c, _ = cpu_sample(args.cpu_k)
    for _ in range(args.steps):
        c, dt = cpu_sample(args.cpu_k)
        times.append(dt)
    v = c["n"] * len(times) / sum(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": wl["name"], "n": wl["n"], "box": wl["box"], "l_x": wl["l_x"],
                   "min_size": wl["min_size"]},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{c['name']}: n={c['n']}, box={c['box']}, same density, "
                                   f"blob recipe and l_x as the full workload"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------

def run_gpu(args):
    import numpy as np
    import torch

    from paper_2003_11468_gb300 import fof

    world, rank, local = dist_setup()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    fof.load()

    wl = workloads()[args.workload]()
    t_gen = time.perf_counter()
    # every rank its own independent box of the same recipe
    pos_np = wl["make"](seed=rank_seed(wl["seed"], rank))
    t_gen = time.perf_counter() - t_gen
    n, box, l_x, min_size = wl["n"], wl["box"], wl["l_x"], wl["min_size"]

    pos_pin = torch.from_numpy(pos_np).pin_memory()
    del pos_np
    pos = pos_pin.to(dev, non_blocking=True)
    ids = torch.empty(n, dtype=torch.int32, device=dev)
    sizes = torch.empty(n, dtype=torch.int32, device=dev)
    cap = max(1 << 20, n // 64)
    cat = torch.empty((cap, 2), dtype=torch.int32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.synchronize(dev)

    h = fof.fof_create(box, l_x, n)
    nc, r, nb = fof.fof_plan_info(h)
    cells = (nc ** 3)

    def step():
        fof.fof_link(h, pos, stream)
        return fof.fof_groups(h, ids, sizes, cat, cap, min_size, 1, stream)

    for _ in range(args.warmup):
        step()
    fof.fof_set_timing(h, True)
    fof.fof_reset_times(h)
    launches0 = fof.fof_kernel_launches(h)

    sampler = ClockSampler(dev.index)
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    res = None
    for _ in range(args.steps):
        res = step()
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    ms_total = max_over_ranks(ev0.elapsed_time(ev1), world, dev)
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    launches = fof.fof_kernel_launches(h) - launches0
    phases = fof.fof_phase_times(h)
    fof.fof_set_timing(h, False)
    code, ng, nk = res
    ms_step = ms_total / args.steps
    value = job_value(n, world, ms_step * 1e-3)

    # dominant kernel and its roofline
    peak, peak_kind = peaks()
    dom = max((k for k in phases if k in ALG_BYTES), key=lambda k: phases[k][0])
    dom_ms, dom_launches = phases[dom]
    per_launch_ms = dom_ms / max(1, args.steps)
    bp, bc = ALG_BYTES[dom]
    alg = bp * n + bc * cells
    achieved = alg / (per_launch_ms * 1e-3) / 1e9
    traffic = recorded_traffic(dom, wl["name"])
    path_alg = PATH_BYTES[0] * n + PATH_BYTES[1] * cells
    path_gbs = path_alg / (ms_step * 1e-3) / 1e9

    # end to end through the C ABI from pinned host buffers
    e2e = None
    if not args.no_e2e:
        ids_h = torch.empty(n, dtype=torch.int32).pin_memory()
        sizes_h = torch.empty(n, dtype=torch.int32).pin_memory()
        cat_h = torch.empty((cap, 2), dtype=torch.int32).pin_memory()
        fof.fof_run_host(h, pos_pin, ids_h, sizes_h, cat_h, cap, min_size, 1, stream)
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            _, _, nk_h = fof.fof_run_host(h, pos_pin, ids_h, sizes_h, cat_h, cap, min_size, 1, stream)
        torch.cuda.synchronize(dev)
        dt = max_over_ranks(time.perf_counter() - t0, world, dev)
        e2e = {"value": job_value(n * args.steps, world, dt), "unit": UNIT,
               "h2d_bytes_per_step": 12 * n,
               "d2h_bytes_per_step": 8 * n + 8 * min(nk_h[0], cap) + 64 + 16}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        c, dt = cpu_sample(args.cpu_k)
        cpu = {"value": c["n"] / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{c['name']}: n={c['n']}, box={c['box']}, a periodic box with the "
                         f"same density, blob recipe and l_x as the full workload"}

    fof.fof_destroy(h)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic",
            "config": {"workload": wl["name"], "n": n, "box": box, "l_x": l_x, "min_size": min_size,
                       "cells_per_axis": nc, "brick_cells": r, "l2": "inputs larger than L2",
                       "n_groups": ng[0], "n_catalogue": nk[0], "status": code},
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                         "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                         "traffic": traffic, "alg_bytes_per_launch": alg,
                         "ms_per_launch": per_launch_ms},
            "path_roofline": {"alg_bytes": path_alg, "achieved": path_gbs, "frac": path_gbs / peak},
            "phases_ms_per_step": {k: v[0] / args.steps for k, v in phases.items()},
            "e2e": e2e,
            "cpu_baseline": cpu,
            "gpu_launches": launches,
            "clocks": clocks,
            "gen_s": t_gen,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# batched and served forms against the plain per-box loop
# ---------------------------------------------------------------------------

def _clocks_start():
    c = ClockSampler(0)
    c.start()
    time.sleep(0.3)
    return c


def run_batch(args):
    """512 boxes (n log-uniform 16^3..160^3): one batch plan replayed as a CUDA
    graph vs a loop of per-box plans, both timed with CUDA events."""
    import numpy as np
    import torch
    from paper_2003_11468_gb300 import fof, synth
    fof.load()
    specs = synth.batch_512(args.boxes)
    t0 = time.perf_counter()
    poss = [synth.make_batch_box(sp) for sp in specs]
    t_gen = time.perf_counter() - t0
    ns = [sp["n"] for sp in specs]
    total = int(sum(ns))
    concat = torch.from_numpy(np.concatenate(poss)).cuda()
    offs = np.concatenate([[0], np.cumsum(ns)]).astype(np.int64)
    stream = torch.cuda.Stream()
    boxes, lxs = [sp["box"] for sp in specs], [sp["l_x"] for sp in specs]
    # plan options picked by the autotuner on this batch (untimed; FOF_TUNE_CACHE caches them)
    opt, tuned, t_tune = None, None, 0.0
    if not args.no_tune:
        from paper_2003_11468_gb300 import tune
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            opt, rep = tune.tune(boxes, lxs, ns, concat, repeats=1, min_size=20, stream=stream)
        t_tune = time.perf_counter() - t0
        tuned = {"options": rep["best"], "key": rep["key"], "cached": rep["cached"]}
    # batched: one plan, one graph
    h = fof.fof_batch_create(boxes, lxs, ns, opt)
    ids_b = torch.empty(total, dtype=torch.int32, device="cuda")
    sizes_b = torch.empty_like(ids_b)
    cat_b = torch.empty((total, 2), dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    fof.fof_graph_build(h, concat, ids_b, sizes_b, cat_b, total, 20, stream)
    for _ in range(args.warmup):
        fof.fof_graph_launch(h, stream)
        fof.fof_result(h, len(specs), stream)
    clocks = _clocks_start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        fof.fof_graph_launch(h, stream)
    e1.record(stream)
    code, ng, nk = fof.fof_result(h, len(specs), stream)
    ms_batch = e0.elapsed_time(e1) / args.steps
    # plain loop: a plan per box (created beforehand), link + groups per box
    plans = [fof.fof_create_ex(sp["box"], sp["l_x"], sp["n"], opt) for sp in specs]
    ids_p = torch.empty(total, dtype=torch.int32, device="cuda")
    sizes_p = torch.empty_like(ids_p)
    cat_p = torch.empty((total, 2), dtype=torch.int32, device="cuda")

    def loop():
        for i, hp in enumerate(plans):
            a, b = int(offs[i]), int(offs[i + 1])
            fof.fof_link(hp, concat[a:b], stream)
            fof.fof_groups(hp, ids_p[a:b], sizes_p[a:b], cat_p[a:b], b - a, 20, 1, stream)
    for _ in range(args.warmup):
        loop()
    e0.record(stream)
    for _ in range(args.steps):
        loop()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_plain = e0.elapsed_time(e1) / args.steps
    clk = clocks.stop()
    exact = bool(torch.equal(ids_b, ids_p)) and bool(torch.equal(sizes_b, sizes_p))
    for hp in plans:
        fof.fof_destroy(hp)
    fof.fof_destroy(h)
    line = {"metric": "particles grouped/s (batched, one CUDA graph)", "value": total / (ms_batch * 1e-3),
            "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_batch,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
            "data": "synthetic",
            "config": {"workload": f"batch of {len(specs)} clustered boxes", "particles": total,
                       "status": code, "tuned": tuned, "tune_s": t_tune},
            "plain_loop": {"value": total / (ms_plain * 1e-3), "unit": UNIT, "ms_per_step": ms_plain},
            "speedup_vs_plain": ms_plain / ms_batch, "identical_to_plain": exact,
            "gpu_launches": None, "clocks": clk, "gen_s": t_gen}
    print(json.dumps(line), flush=True)
    return 0


def run_served(args):
    """Poisson requests through the server vs the same requests one by one."""
    import numpy as np
    import torch
    from paper_2003_11468_gb300 import fof, synth
    from paper_2003_11468_gb300.server import Server
    fof.load()
    reqs = synth.served_requests(count=args.requests)
    # a pool of distinct inputs, reused by the requests (bounded generation)
    pool_n = sorted({int(np.exp(v)) for v in np.linspace(np.log(1e4), np.log(1e8), args.pool)})
    t0 = time.perf_counter()
    pool = {}
    for k, n in enumerate(pool_n):
        box = 100.0 * (n / 256 ** 3) ** (1.0 / 3.0)
        pos = synth.clustered_box(n, box, max(1, int(round(20000 * n / 256 ** 3))), seed=5_000_000 + k)
        pool[n] = (torch.from_numpy(pos).pin_memory(), box, synth.linking_length(n, box))
    t_gen = time.perf_counter() - t0
    keys = np.array(pool_n)
    jobs = []
    for r in reqs:
        n = int(keys[np.argmin(np.abs(np.log(keys) - np.log(r["n"])))])
        jobs.append((r["t_arrive"], n))
    total = sum(n for _, n in jobs)
    # plain: one request at a time, each with its own plan, results to host
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _, n in jobs:
        pos, box, l_x = pool[n]
        with fof.FoF(box, l_x, n) as f:
            ids, sizes, cat, _ = f.run(pos.cuda(non_blocking=True), min_size=20)
            ids.cpu(), sizes.cpu(), cat.cpu()
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t0
    # served: Poisson arrivals replayed in real time
    clocks = _clocks_start()
    nmax = max(pool_n)
    _, bmax, lmax = pool[nmax]
    with Server(memory_budget=args.budget_gb << 30, slots=args.slots, prealloc=(bmax, lmax, nmax)) as srv:
        futs = []
        start = time.perf_counter()
        for t_arr, n in jobs:
            wait = start + t_arr - time.perf_counter()
            if wait > 0:
                time.sleep(wait)
            pos, box, l_x = pool[n]
            futs.append(srv.submit(pos, box, l_x, 20))
        for f in futs:
            f.result()
        t_served = time.perf_counter() - start
    lat = np.array(srv.latencies)
    clk = clocks.stop()
    line = {"metric": "particles grouped/s (served, Poisson 200/s)", "value": total / t_served, "unit": UNIT,
            "n_gpus": 1, "steps": 1, "warmup": 0, "ms_per_step": t_served * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"{len(jobs)} Poisson requests, n log-uniform 1e4..1e8",
                       "particles": total, "budget_gb": args.budget_gb, "slots": args.slots},
            "latency_ms": {"p50": float(np.percentile(lat, 50) * 1e3),
                           "p99": float(np.percentile(lat, 99) * 1e3)},
            "plain_loop": {"value": total / t_plain, "unit": UNIT, "seconds": t_plain},
            "clocks": clk, "gen_s": t_gen}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-tune", action="store_true", help="batch workload: library default options")
    ap.add_argument("--workload", default="1024", choices=["1024", "1024s", "256", "32k", "batch", "served"])
    ap.add_argument("--boxes", type=int, default=512, help="batch workload: number of boxes")
    ap.add_argument("--requests", type=int, default=400, help="served workload: requests")
    ap.add_argument("--pool", type=int, default=24, help="served workload: distinct inputs")
    ap.add_argument("--slots", type=int, default=3)
    ap.add_argument("--budget-gb", type=int, default=120)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-k", type=int, default=8, help="CPU sample is a 1/k^3 volume box")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "served":
        return run_served(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
