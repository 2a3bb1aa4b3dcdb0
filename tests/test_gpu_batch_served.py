"""Batched and served forms: every box / request gets exactly its solo result.

Batched: independent boxes of uneven sizes, box sides and linking lengths in
one plan (one set of launches, optionally one CUDA graph).  Served: requests
arriving over time through the continuous-batching server.
"""
import time

import numpy as np
import pytest

import oracle
from paper_2003_11468_gb300 import synth

pytestmark = pytest.mark.gpu


def _boxes(count, seed, n_lo=200, n_hi=60000):
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        n = int(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi))))
        box = float(rng.uniform(5.0, 40.0))
        l_x = synth.linking_length(n, box, float(rng.uniform(0.15, 0.35)))
        pos = synth.clustered_box(n, box, max(1, n // 200), seed=seed * 1000 + b)
        out.append((pos, box, l_x))
    return out


def _solo(fof, pos, box, l_x, min_size):
    import torch
    n = pos.shape[0]
    with fof.FoF(box, l_x, n) as f:
        ids, sizes, cat, ng = f.run(torch.from_numpy(pos).cuda(), min_size=min_size)
        return ids.cpu().numpy(), sizes.cpu().numpy(), cat.cpu().numpy(), ng


def test_batch_matches_oracle_per_box(cuda_lib):
    import torch
    fof = cuda_lib
    boxes = _boxes(24, seed=1)
    boxes.insert(5, (np.zeros((0, 3), np.float32), 10.0, 0.3))      # an empty box
    boxes.insert(9, (np.array([[1.0, 2.0, 3.0]], np.float32), 10.0, 0.3))
    ns = [p.shape[0] for p, _, _ in boxes]
    concat = torch.from_numpy(np.concatenate([p for p, _, _ in boxes])).cuda()
    fb = fof.FoFBatch([b for _, b, _ in boxes], [l for _, _, l in boxes], ns)
    try:
        ids, sizes, cat, ng, nk = fb.run(concat, min_size=5)
    finally:
        fb.close()
    ids, sizes, cat = ids.cpu().numpy(), sizes.cpu().numpy(), cat.cpu().numpy()
    off = np.concatenate([[0], np.cumsum(ns)])
    koff = np.concatenate([[0], np.cumsum(nk)])
    for i, (pos, box, l_x) in enumerate(boxes):
        wid, wsz = oracle.groups(pos, box, l_x)
        assert np.array_equal(ids[off[i]:off[i + 1]], wid), i
        assert np.array_equal(sizes[off[i]:off[i + 1]], wsz), i
        assert np.array_equal(cat[koff[i]:koff[i + 1]], oracle.catalogue(wsz, 5)), i
        assert ng[i] == int((wsz > 0).sum())


def test_batch_equals_solo_and_graph_replays(cuda_lib):
    import torch
    fof = cuda_lib
    boxes = _boxes(40, seed=2, n_lo=1000, n_hi=120000)
    ns = [p.shape[0] for p, _, _ in boxes]
    total = sum(ns)
    concat = torch.from_numpy(np.concatenate([p for p, _, _ in boxes])).cuda()
    h = fof.fof_batch_create([b for _, b, _ in boxes], [l for _, _, l in boxes], ns)
    s = torch.cuda.Stream()
    try:
        ids = torch.empty(total, dtype=torch.int32, device="cuda")
        sizes = torch.empty(total, dtype=torch.int32, device="cuda")
        cat = torch.empty((total, 2), dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        fof.fof_graph_build(h, concat, ids, sizes, cat, total, 20, s)
        results = []
        for _ in range(2):
            ids.fill_(-1)
            torch.cuda.synchronize()
            fof.fof_graph_launch(h, s)
            code, ng, nk = fof.fof_result(h, len(boxes), s)
            assert code == 0
            results.append((ids.cpu().numpy().copy(), sizes.cpu().numpy().copy()))
        assert np.array_equal(results[0][0], results[1][0])
    finally:
        fof.fof_destroy(h)
    off = np.concatenate([[0], np.cumsum(ns)])
    for i, (pos, box, l_x) in enumerate(boxes):
        sid, ssz, _, sng = _solo(fof, pos, box, l_x, 20)
        assert np.array_equal(results[0][0][off[i]:off[i + 1]], sid), i
        assert np.array_equal(results[0][1][off[i]:off[i + 1]], ssz), i
        assert ng[i] == sng


def test_server_results_equal_solo_in_the_mix(cuda_lib):
    import torch
    fof = cuda_lib
    from paper_2003_11468_gb300.server import Server
    boxes = _boxes(30, seed=3, n_lo=500, n_hi=150000)
    solo = [_solo(fof, p, b, l, 10) for p, b, l in boxes]
    futs = []
    with Server(memory_budget=2 << 30, slots=3, max_batch_boxes=8) as srv:
        for k, (p, b, l) in enumerate(boxes):
            futs.append(srv.submit(torch.from_numpy(p).pin_memory(), b, l, 10))
            if k % 5 == 0:
                time.sleep(0.002)                   # arrivals spread over time
        res = [f.result(timeout=120) for f in futs]
    lat = list(srv.latencies)            # complete once close() joined the scheduler
    for r, (sid, ssz, scat, sng) in zip(res, solo):
        assert np.array_equal(r.ids, sid)
        assert np.array_equal(r.sizes, ssz)
        assert np.array_equal(r.catalogue, scat)
        assert r.n_groups == sng
    assert len(lat) == len(boxes) and min(lat) > 0


def test_server_admission_and_oversize(cuda_lib):
    import torch
    fof = cuda_lib
    from paper_2003_11468_gb300.server import Server
    boxes = _boxes(6, seed=4, n_lo=20000, n_hi=40000)
    need = max(fof.fof_batch_workspace_bytes([b], [l], [p.shape[0]]) + 28 * p.shape[0]
               for p, b, l in boxes)
    # a budget that admits one request at a time: results must not change
    with Server(memory_budget=int(need * 1.5), slots=4) as srv:
        futs = [srv.submit(torch.from_numpy(p).pin_memory(), b, l, 3) for p, b, l in boxes]
        res = [f.result(timeout=120) for f in futs]
        big = srv.submit(torch.zeros((400000, 3), dtype=torch.float32).pin_memory(), 100.0, 0.5, 3)
        with pytest.raises(MemoryError):
            big.result(timeout=60)
    for r, (p, b, l) in zip(res, boxes):
        wid, wsz = oracle.groups(p, b, l)
        assert np.array_equal(r.ids, wid) and np.array_equal(r.sizes, wsz)


def test_server_budget_covers_retained_buffers(cuda_lib):
    """The budget bounds what the slots keep, idle or busy: after a large
    request the slots' retained buffers plus later small batches stay within
    it, and the process's reserved device memory grows by no more than the
    budget."""
    import torch
    fof = cuda_lib
    from paper_2003_11468_gb300.server import Server
    big = _boxes(1, seed=5, n_lo=400000, n_hi=400001)[0]
    small = _boxes(12, seed=6, n_lo=20000, n_hi=60000)
    need_big = fof.fof_batch_workspace_bytes([big[1]], [big[2]], [big[0].shape[0]]) + 28 * big[0].shape[0]
    budget = int(need_big * 1.6)                 # room for one big slot, not two
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    base = torch.cuda.memory_reserved()
    with Server(memory_budget=budget, slots=3) as srv:
        r0 = srv.submit(torch.from_numpy(big[0]).pin_memory(), big[1], big[2], 5).result(timeout=120)
        futs = [srv.submit(torch.from_numpy(p).pin_memory(), b, l, 5) for p, b, l in small]
        res = [f.result(timeout=120) for f in futs]
        r1 = srv.submit(torch.from_numpy(big[0]).pin_memory(), big[1], big[2], 5).result(timeout=120)
        assert srv.held_bytes() <= budget
        torch.cuda.synchronize()
        assert torch.cuda.memory_reserved() - base <= budget + (64 << 20)
    assert np.array_equal(r0.ids, r1.ids)
    for r, (p, b, l) in zip(res, small):
        wid, wsz = oracle.groups(p, b, l)
        assert np.array_equal(r.ids, wid) and np.array_equal(r.sizes, wsz)
