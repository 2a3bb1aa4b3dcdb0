"""The bench's multi-rank host logic on two gloo ranks (CPU).

With N GPUs every rank groups its own box of the same recipe (weak
scaling, no collective on the data path); the step time is the slowest
rank's, and the whole-job value counts every rank's particles.  The
reference arm runs on rank 0 only.
"""
import importlib.util
import json
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench = _bench()
        from paper_2003_11468_gb300 import synth
        import oracle
        w, r, _ = bench.dist_setup()
        seed = bench.rank_seed(7, r)
        # each rank its own independent small box of one recipe
        n, box = 3000, 12.0
        pos = synth.clustered_box(n, box, 6, seed=seed)
        ids, sizes = oracle.groups(pos, box, synth.linking_length(n, box))
        local_s = 0.010 + 0.005 * r                 # the ranks finish at different times
        slowest = bench.max_over_ranks(local_s, w)
        value = bench.job_value(n, w, slowest)
        # the reference arm: only rank 0 works
        class A:
            workload, warmup, steps, cpu_k, gpus = "32k", 0, 1, 64, w
        ref_rc = bench.run_reference(A()) if r != 0 else None
        with open(os.path.join(out_dir, f"rank{r}.json"), "w") as f:
            json.dump({"world": w, "seed": seed, "slowest": slowest, "value": value,
                       "first_pos": pos[0].tolist(), "n_groups": int((sizes > 0).sum()),
                       "ref_rc": ref_rc}, f)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn")
    r0 = json.load(open(tmp_path / "rank0.json"))
    r1 = json.load(open(tmp_path / "rank1.json"))
    assert r0["world"] == r1["world"] == 2
    assert r0["seed"] != r1["seed"] and r0["first_pos"] != r1["first_pos"]   # independent boxes
    assert r0["slowest"] == r1["slowest"] == pytest.approx(0.015)           # max over ranks
    assert r0["value"] == r1["value"] == pytest.approx(2 * 3000 / 0.015)    # all ranks' particles
    assert r1["ref_rc"] == 0                                                # rank 1 skips the oracle arm
    assert r0["n_groups"] > 0 and r1["n_groups"] > 0


def test_single_rank_helpers():
    bench = _bench()
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_value(1000, 1, 0.5) == 2000.0
    assert bench.rank_seed(3, 0) == 3 and bench.rank_seed(3, 2) != bench.rank_seed(3, 1)
