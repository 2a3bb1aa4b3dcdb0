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
# (c), following the method's byte budget: read the positions (12), write the
# binned float4 (16) and the forest (4), one read of the binned float4 in the
# link sweep (16), read the forest at finalisation (4), write ids and sizes
# (8); 8 per cell for counts and starts.  The whole path: 60 per particle +
# 8 per cell.
ALG_BYTES = {
    "bin_count": (12, 0),      # read positions
    "bin_scatter": (0, 0),
    "brick_sort": (20, 8),     # write the binned float4 and parent[s] = s; cell counts + starts
    "team_self": (0, 0),
    "big_sort": (0, 0),
    "dense_self": (0, 0),
    "dense_pairs": (0, 0),
    "big_pairs": (0, 0),
    "link": (16, 0),           # one read of the binned float4
    "finalize": (4, 0),        # read the forest
    "outputs": (8, 0),         # write ids and sizes
    "catalogue": (0, 0),
    "scan_bricks": (0, 0),
}
PATH_BYTES = (60, 8)
# The bytes each phase of this implementation must move at least, given its
# two-pass binning and its arrays (reported beside the budget above).
ALG_BYTES_EXT = {
    "bin_count": (12, 0),      # read positions
    "bin_scatter": (28, 0),    # read positions, write brick-order float4
    "brick_sort": (44, 4),     # read float4, write float4 + parent/minorig/cnt, cell starts
    "link": (20, 4),           # read binned float4 + parent once, cell starts once
    "finalize": (8, 0),        # read parent + own index of non-roots
    "outputs": (20, 0),        # read parent, root data, own index; write ids, sizes
    "catalogue": (4, 0),       # read sizes
    "scan_bricks": (0, 0),
}


def workloads():
    from paper_2003_11468_gb300 import synth
    return {
        "1024": synth.clustered_1024,
        # 1/64 of the 1024^3 box at the same density, blob recipe and l_x:
        # the small case the per-kernel ncu captures run on; its grid is
        # fixed at 384^3 cells (3.33 l_x wide, 6 sub-cells per axis) to match
        # the 1024^3 box's 1520^3 (3.37 l_x, 6 sub-cells), where the default
        # choice for the smaller box would round down to 352^3 (3.64 l_x)
        "1024s": lambda: dict(synth.clustered_sample_of_1024(4), cells_per_axis=384),
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


def host_cpu_info() -> dict:
    """Core count, CPU model and affinity of this host (for the CPU baselines)."""
    info = {"nproc": os.cpu_count()}
    try:
        info["affinity"] = sorted(os.sched_getaffinity(0))
        aff = info["affinity"]
        info["affinity"] = f"{len(aff)} cpus: {aff[0]}-{aff[-1]}" if aff == list(range(aff[0], aff[-1] + 1)) \
            else ",".join(map(str, aff))
    except Exception:
        pass
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            with open("/proc/cpuinfo") as f:
                for line in f:
                    if line.lower().startswith(("model name", "cpu part")):
                        model = line.split(":", 1)[1].strip()
                        break
        except Exception:
            pass
    import platform
    info["cpu_model"] = model or platform.processor() or platform.machine()
    info["machine"] = platform.machine()
    return info


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
    host = host_cpu_info()
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        # what each step ran: a bounded sample of the workload (same density,
        # blob recipe and l_x), named here with its own size
        "config": {"workload": wl["name"], "sample": c["name"], "n": c["n"], "box": c["box"],
                   "l_x": c["l_x"], "min_size": c["min_size"],
                   "sample_of": {"n": wl["n"], "box": wl["box"]}},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{c['name']}: n={c['n']}, box={c['box']}, same density, "
                                   f"blob recipe and l_x as the full workload",
                         "host": host},
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

    if "cells_per_axis" in wl:
        opt = fof.fof_options()
        opt.cells_per_axis = wl["cells_per_axis"]
        h = fof.fof_create_ex(box, l_x, n, opt)
    else:
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
    ep, ec = ALG_BYTES_EXT.get(dom, (0, 0))
    alg_ext = ep * n + ec * cells
    traffic = recorded_traffic(dom, wl["name"])
    path_alg = PATH_BYTES[0] * n + PATH_BYTES[1] * cells
    path_gbs = path_alg / (ms_step * 1e-3) / 1e9

    # end to end through the C ABI from pinned host buffers
    e2e = None
    if not args.no_e2e:
        ids_h = torch.empty(n, dtype=torch.int32).pin_memory()
        sizes_h = torch.empty(n, dtype=torch.int32).pin_memory()
        cat_h = torch.empty((cap, 2), dtype=torch.int32).pin_memory()
        # every step copies its positions in from pinned host memory and its
        # ids, sizes and catalogue out; fof_run_host_many overlaps the copies
        # of one step with the compute of the next
        fof.fof_run_host_many(h, [pos_pin] * 2, [ids_h] * 2, [sizes_h] * 2, [cat_h] * 2, cap, min_size, 1,
                              stream)
        torch.cuda.synchronize(dev)
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        K = args.steps
        _, _, nk_h = fof.fof_run_host_many(h, [pos_pin] * K, [ids_h] * K, [sizes_h] * K, [cat_h] * K, cap,
                                           min_size, 1, stream)
        torch.cuda.synchronize(dev)
        dt = max_over_ranks(time.perf_counter() - t0, world, dev)
        e2e = {"value": job_value(n * K, world, dt), "unit": UNIT,
               "h2d_bytes_per_step": 12 * n,
               "d2h_bytes_per_step": 8 * n + 8 * min(nk_h[-1][0], cap) + 64 + 16,
               "api": "fof_run_host_many (copies of one step overlap the compute of the next)"}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        c, dt = cpu_sample(args.cpu_k)
        cpu = {"value": c["n"] / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{c['name']}: n={c['n']}, box={c['box']}, a periodic box with the "
                         f"same density, blob recipe and l_x as the full workload",
               "host": host_cpu_info()}

    fof.fof_destroy(h)
    # the batched and served forms against the plain per-box loop (one GPU)
    batched = served = None
    if world == 1 and wl["name"] == "fof-1024^3-clustered":
        del pos, ids, sizes, cat, pos_pin
        if e2e is not None:
            del ids_h, sizes_h, cat_h
        torch.cuda.empty_cache()
        if not args.no_batched:
            batched = batch_record(args)
        if not args.no_served:
            served = served_record(args)
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
                         "alg_bytes_ext": alg_ext, "frac_ext": alg_ext / (per_launch_ms * 1e-3) / 1e9 / peak,
                         "ms_per_launch": per_launch_ms},
            "path_roofline": {"alg_bytes": path_alg, "achieved": path_gbs, "frac": path_gbs / peak},
            "phases_ms_per_step": {k: v[0] / args.steps for k, v in phases.items()},
            "e2e": e2e,
            "cpu_baseline": cpu,
            "gpu_launches": launches,
            "clocks": clocks,
            "gen_s": t_gen,
            "batched": batched,
            "served": served,
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


def batch_record(args) -> dict:
    """The batched form: 512 boxes (n log-uniform 16^3..160^3) in one batch
    plan replayed as a CUDA graph, against a loop of per-box plans (created
    before timing), both timed with CUDA events on the same stream."""
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
    del poss
    offs = np.concatenate([[0], np.cumsum(ns)]).astype(np.int64)
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()                           # inputs written before the library's stream reads them
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
    h = fof.fof_batch_create(boxes, lxs, ns, opt)
    ids_b = torch.empty(total, dtype=torch.int32, device="cuda")
    sizes_b = torch.empty_like(ids_b)
    cat_b = torch.empty((total, 2), dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    fof.fof_graph_build(h, concat, ids_b, sizes_b, cat_b, total, 20, stream)
    for _ in range(args.warmup):
        fof.fof_graph_launch(h, stream)
        fof.fof_result(h, len(specs), stream)
    launches0 = fof.fof_kernel_launches(h)
    clocks = _clocks_start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        fof.fof_graph_launch(h, stream)
    e1.record(stream)
    code, ng, nk = fof.fof_result(h, len(specs), stream)
    ms_batch = e0.elapsed_time(e1) / args.steps
    launches = (fof.fof_kernel_launches(h) - launches0) // max(1, args.steps)
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
    del concat, ids_b, sizes_b, cat_b, ids_p, sizes_p, cat_p
    torch.cuda.empty_cache()
    return {"metric": "particles grouped/s (batched, one CUDA graph)",
            "value": total / (ms_batch * 1e-3), "unit": UNIT, "ms_per_step": ms_batch,
            "steps": args.steps, "warmup": args.warmup,
            "config": {"workload": f"batch of {len(specs)} clustered boxes, n log-uniform 16^3..160^3",
                       "particles": total, "status": code, "tuned": tuned, "tune_s": t_tune},
            "plain_loop": {"value": total / (ms_plain * 1e-3), "unit": UNIT, "ms_per_step": ms_plain,
                           "how": "per-box plans created before timing; fof_link + fof_groups per box"},
            "speedup_vs_plain": ms_plain / ms_batch, "identical": exact,
            "gpu_launches_per_step": launches, "clocks": clk, "gen_s": t_gen}


def _serve(srv, pool, inputs, jobs, replay: bool):
    """Submit the jobs (at their arrival times when replay, else at once) and
    wait for all; returns (seconds, latencies).  Only the latency of each
    result is kept: results are dropped as soon as they arrive, so the host
    never holds more than the requests in flight."""
    done = threading.Semaphore(0)
    lat, errs = [], []
    lock = threading.Lock()

    def on_done(f):
        try:
            v = f.result().latency_s
            with lock:
                lat.append(v)
        except Exception as e:      # reported after the run
            with lock:
                errs.append(e)
        done.release()

    start = time.perf_counter()
    for t_arr, k in jobs:
        if replay:
            wait = start + t_arr - time.perf_counter()
            if wait > 0:
                time.sleep(wait)
        srv.submit(inputs[k], pool[k]["box"], pool[k]["l_x"], 20).add_done_callback(on_done)
    for _ in jobs:
        done.acquire()
    dt = time.perf_counter() - start
    if errs:
        raise errs[0]
    return dt, lat


def served_record(args) -> dict:
    """The served form against the plain loop, on the same requests.

    Requests: Poisson arrivals (mean 200/s), sizes log-uniform on [1e4, 1e8];
    each request takes the input of nearest log-size from a pool of distinct
    inputs (generation is bounded; every input is a real box of that size).
    Every form copies each request's positions from pinned host memory and
    its ids and sizes back to host memory.
      * plain loop: one request at a time, back to back, a plan per distinct
        size created before timing;
      * served, all at once: every request submitted at t = 0 -- the server's
        busy throughput, comparable with the plain loop;
      * served, Poisson replay: requests submitted at their arrival times --
        latency from arrival to result (p50/p99); its throughput is bounded
        by the arrival rate.
    Throughputs are repeated (args.served_repeats) and given as median,
    mean and standard deviation."""
    import numpy as np
    import torch
    from paper_2003_11468_gb300 import fof, synth
    from paper_2003_11468_gb300.server import Server
    fof.load()
    pool = synth.served_pool(args.pool)
    t0 = time.perf_counter()
    inputs = [torch.from_numpy(synth.make_served(sp)).pin_memory() for sp in pool]
    t_gen = time.perf_counter() - t0
    reqs = synth.served_requests(count=args.requests)
    logs = np.log(np.array([sp["n"] for sp in pool], dtype=np.float64))
    jobs = [(r["t_arrive"], int(np.argmin(np.abs(logs - np.log(r["n"]))))) for r in reqs]
    total = sum(pool[k]["n"] for _, k in jobs)

    def stats(v):
        return {"median": statistics.median(v), "mean": statistics.fmean(v),
                "std": statistics.pstdev(v) if len(v) > 1 else 0.0, "runs": v}

    # plain loop: plans and buffers for every distinct size, made before timing
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream()
    plain = []
    for sp in pool:
        n = sp["n"]
        plain.append(dict(h=fof.fof_create(sp["box"], sp["l_x"], n),
                          pos=torch.empty((n, 3), dtype=torch.float32, device=dev),
                          ids=torch.empty(n, dtype=torch.int32, device=dev),
                          sizes=torch.empty(n, dtype=torch.int32, device=dev),
                          cat=torch.empty((n, 2), dtype=torch.int32, device=dev),
                          ids_h=torch.empty(n, dtype=torch.int32).pin_memory(),
                          sizes_h=torch.empty(n, dtype=torch.int32).pin_memory()))

    def plain_pass():
        for _, k in jobs:
            P, sp = plain[k], pool[k]
            with torch.cuda.stream(stream):
                P["pos"].copy_(inputs[k], non_blocking=True)
                fof.fof_link(P["h"], P["pos"], stream)
                _, _, nk = fof.fof_groups(P["h"], P["ids"], P["sizes"], P["cat"], sp["n"], 20, 1, stream)
                P["ids_h"].copy_(P["ids"], non_blocking=True)
                P["sizes_h"].copy_(P["sizes"], non_blocking=True)
                P["cat"][: nk[0]].cpu()
            stream.synchronize()

    clocks = _clocks_start()
    plain_pass()                                   # warm-up
    t_plain = []
    for _ in range(args.served_repeats):
        t0 = time.perf_counter()
        plain_pass()
        t_plain.append(total / (time.perf_counter() - t0))
    big = max(range(len(pool)), key=lambda k: pool[k]["n"])
    prealloc = (pool[big]["box"], pool[big]["l_x"], pool[big]["n"])
    at_once, lat, t_poisson, identical = [], None, None, True
    with Server(memory_budget=args.budget_gb << 30, slots=args.slots, prealloc=prealloc) as srv:
        # warm-up, and the exactness check against the plain loop's outputs
        futs = [srv.submit(inputs[k], sp["box"], sp["l_x"], 20) for k, sp in enumerate(pool)]
        for k, f in enumerate(futs):
            r = f.result()
            identical &= bool(np.array_equal(r.ids, plain[k]["ids_h"].numpy())) and \
                bool(np.array_equal(r.sizes, plain[k]["sizes_h"].numpy()))
        del futs, r
        for _ in range(args.served_repeats):
            dt, _ = _serve(srv, pool, inputs, jobs, replay=False)
            at_once.append(total / dt)
        dt, lat = _serve(srv, pool, inputs, jobs, replay=True)
        t_poisson = total / dt
        lat = np.array(lat)
        held_gb = srv.held_bytes() / 2 ** 30
    clk = clocks.stop()
    for P in plain:
        fof.fof_destroy(P["h"])
    del plain, inputs
    torch.cuda.empty_cache()
    sa, sp_ = stats(at_once), stats(t_plain)
    return {"metric": "particles grouped/s (served, continuous batching)",
            "value": sa["median"], "unit": UNIT,
            "config": {"workload": f"{len(jobs)} Poisson requests (200/s), n log-uniform 1e4..1e8, "
                                   f"inputs from a pool of {len(pool)} distinct sizes",
                       "particles": total, "budget_gb": args.budget_gb, "slots": args.slots,
                       "repeats": args.served_repeats},
            "served_all_at_once": sa,
            "plain_loop": dict(sp_, how="one request at a time; plans and buffers made before timing; "
                                        "H2D of positions and D2H of ids/sizes/catalogue per request"),
            "speedup_vs_plain": sa["median"] / sp_["median"],
            "poisson_replay": {"value": t_poisson, "unit": UNIT,
                               "latency_ms": {"p50": float(np.percentile(lat, 50) * 1e3),
                                              "p99": float(np.percentile(lat, 99) * 1e3)}},
            "identical": identical, "server_held_gb": held_gb, "clocks": clk, "gen_s": t_gen}


def run_batch(args):
    line = batch_record(args)
    line.update({"n_gpus": 1, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                 "dtype": "f32+f64", "data": "synthetic"})
    print(json.dumps(line), flush=True)
    return 0


def run_served(args):
    line = served_record(args)
    line.update({"n_gpus": 1, "steps": args.served_repeats, "warmup": 1, "higher_is_better": True,
                 "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic"})
    print(json.dumps(line), flush=True)
    return 0


def run_ablation(args):
    """The paper's union-find alternatives (fof.h variant fields) timed on one
    workload: each variant runs the same input, its ids are checked equal to
    the default's (or, for the strict tie rule, reported as differing), and
    the per-phase device times are reported.  One JSON line."""
    import numpy as np
    import torch
    from paper_2003_11468_gb300 import fof
    fof.load()
    wl = workloads()[args.workload]()
    pos = torch.from_numpy(wl["make"]()).cuda()
    n, box, l_x = wl["n"], wl["box"], wl["l_x"]
    ids = torch.empty(n, dtype=torch.int32, device="cuda")
    sizes = torch.empty_like(ids)
    torch.cuda.synchronize()                           # inputs written before the library's stream reads them
    ref = None
    variants = [
        ("default: halving on paths of depth >= 2, hook onto the smaller root, warp-aggregated sizes", {}),
        ("control: the default through the variant-capable kernels", {"debug_flags": 2}),
        ("find: halving at every depth", {"find_variant": 1}),
        ("find: full compression", {"find_variant": 2}),
        ("find: no compression", {"find_variant": 3}),
        ("union: randomised linking (Jayanti-Tarjan)", {"link_order": 1}),
        ("sizes: per-block hash table", {"size_count": 1}),
        ("tie rule: distance < l_x", {"tie_rule": 1}),
    ]
    out = []
    clocks = _clocks_start()
    for name, fields in variants:
        opt = fof.fof_options()
        for k, v in fields.items():
            setattr(opt, k, v)
        h = fof.fof_create_ex(box, l_x, n, opt)
        stream = torch.cuda.Stream()
        for _ in range(args.warmup):
            fof.fof_link(h, pos, stream)
            fof.fof_groups(h, ids, sizes, None, 0, 20, 1, stream)
        fof.fof_set_timing(h, True)
        fof.fof_reset_times(h)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            fof.fof_link(h, pos, stream)
            _, ng, _ = fof.fof_groups(h, ids, sizes, None, 0, 20, 1, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ph = fof.fof_phase_times(h)
        fof.fof_destroy(h)
        got = ids.cpu().numpy()
        if ref is None:
            ref = got.copy()
        same = bool(np.array_equal(got, ref))
        out.append({"variant": name, "options": fields, "ms_per_step": e0.elapsed_time(e1) / args.steps,
                    "phases_ms": {k: v[0] / args.steps for k, v in ph.items() if v[0] > 0},
                    "ids_equal_default": same, "n_groups": ng[0]})
    line = {"metric": "ms per step by union-find variant", "workload": wl["name"], "n": n,
            "steps": args.steps, "warmup": args.warmup, "variants": out, "clocks": clocks.stop()}
    print(json.dumps(line), flush=True)
    return 0


def run_relink(args):
    """fof_relink against fof_link on the same workload after the particles
    move: unmoved (path 0), moved toward their cell centres (no cell change,
    path 0), and displaced by a small random step (typically path 2 on a
    large box: some particle always leaves its brick).  Device times with
    CUDA events; ids checked equal to fof_link's."""
    import numpy as np
    import torch
    from paper_2003_11468_gb300 import fof
    fof.load()
    wl = workloads()[args.workload]()
    n, box, l_x = wl["n"], wl["box"], wl["l_x"]
    pos0 = torch.from_numpy(wl["make"]()).cuda()
    geo = fof.fof_box_geometry(box, l_x, n)
    q, nf, inv = geo.sub_cells, geo.fine_per_axis, float(np.float32(geo.inv_fine))
    step = 0.01 * l_x
    boxf = float(np.float32(box))
    gen = torch.Generator(device="cuda").manual_seed(7)

    def cells(p):
        f = torch.clamp((p * torch.tensor(inv, dtype=torch.float32, device=p.device)).to(torch.int32),
                        max=nf - 1)
        return torch.div(f, q, rounding_mode="floor")

    def moved(kind):
        out = torch.empty_like(pos0)
        chunk = 1 << 25
        for i in range(0, n, chunk):
            p = pos0[i:i + chunk]
            if kind == "near":
                c = cells(p)
                centre = ((c.to(torch.float64) + 0.5) * q / inv).to(torch.float32)
                m = p + 0.3 * (centre - p)
                keep = (cells(m) == c).all(dim=1, keepdim=True)
                out[i:i + chunk] = torch.where(keep, m, p)
            else:
                r = torch.randn(p.shape, device="cuda", generator=gen, dtype=torch.float32)
                m = torch.remainder(p.double() + step * r.double(), box).float()
                out[i:i + chunk] = torch.where(m >= boxf, torch.zeros_like(m), m)
        return out

    ids = torch.empty(n, dtype=torch.int32, device="cuda")
    ids_ref = torch.empty_like(ids)
    sizes = torch.empty_like(ids)
    stream = torch.cuda.Stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    h = fof.fof_create(box, l_x, n)
    torch.cuda.synchronize()
    res = []
    clocks = _clocks_start()
    for name, kind in (("unmoved", None), ("toward cell centres", "near"), (f"random step {step:.3g}", "jit")):
        p = pos0 if kind is None else moved(kind)
        torch.cuda.synchronize()                       # inputs written before the library's stream reads them
        fof.fof_link(h, p, stream)
        fof.fof_groups(h, ids_ref, sizes, None, 0, 20, 1, stream)
        t_link, t_relink, paths = [], [], []
        same = True
        for _ in range(max(1, args.steps // 2)):
            fof.fof_link(h, pos0, stream)                  # the previous binning
            torch.cuda.synchronize()
            e0.record(stream)
            fof.fof_link(h, p, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            t_link.append(e0.elapsed_time(e1))
            fof.fof_link(h, pos0, stream)
            torch.cuda.synchronize()
            e0.record(stream)
            paths.append(fof.fof_relink(h, p, stream))
            e1.record(stream)
            torch.cuda.synchronize()
            t_relink.append(e0.elapsed_time(e1))
            fof.fof_groups(h, ids, sizes, None, 0, 20, 1, stream)
            same &= bool(torch.equal(ids, ids_ref))
        res.append({"case": name, "path": paths[-1], "fof_link_ms": statistics.median(t_link),
                    "fof_relink_ms": statistics.median(t_relink), "ids_equal": same})
        del p
        torch.cuda.empty_cache()
    fof.fof_destroy(h)
    print(json.dumps({"metric": "fof_relink vs fof_link (ms, binning + linking)", "workload": wl["name"],
                      "n": n, "cases": res, "clocks": clocks.stop()}), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-tune", action="store_true", help="batch workload: library default options")
    ap.add_argument("--workload", default="1024", choices=["1024", "1024s", "256", "32k", "batch", "served"])
    ap.add_argument("--ablation", action="store_true", help="time the union-find variants on --workload")
    ap.add_argument("--relink", action="store_true", help="time fof_relink against fof_link on --workload")
    ap.add_argument("--boxes", type=int, default=512, help="batch workload: number of boxes")
    ap.add_argument("--requests", type=int, default=2000, help="served workload: requests")
    ap.add_argument("--served-repeats", type=int, default=3, help="served workload: timed repeats")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched sub-record")
    ap.add_argument("--no-served", action="store_true", help="skip the served sub-record")
    ap.add_argument("--pool", type=int, default=24, help="served workload: distinct inputs")
    ap.add_argument("--slots", type=int, default=3)
    ap.add_argument("--budget-gb", type=int, default=120)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-k", type=int, default=8, help="CPU sample is a 1/k^3 volume box")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.ablation:
        return run_ablation(args)
    if args.relink:
        return run_relink(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "served":
        return run_served(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
