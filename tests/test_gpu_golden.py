"""Full-size parity: SHA-256 of the GPU outputs against the oracle's.

The records in tests/golden/fullsize/ were written by
tests/golden/make_fullsize_goldens.py, which runs only the seeded generators
and the CPU oracle.  Each test regenerates the same inputs, checks their
hash first (a mismatch there is a generator difference between machines,
not a group-finder error), runs the CUDA path in the configuration the
benchmark times, and compares the hashes of ids, sizes and the catalogue,
which compares every element bit for bit, plus the group counts.

Covers every workload at its own size: 32^3 uniform, 256^3 clustered,
1024^3 clustered (plain plan), the 512 boxes of the batched form (one batch
plan replayed as a CUDA graph) and the served workload's input pool (all
requests through the continuous-batching server at once).
"""
import hashlib
import json
import os

import numpy as np
import pytest

from paper_2003_11468_gb300 import synth

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "fullsize")


def _records(name):
    path = os.path.join(GOLD, name + ".json")
    if not os.path.exists(path):
        pytest.fail(f"golden record {path} is missing")
    with open(path) as f:
        return json.load(f)["records"]


def _sha(a) -> str:
    if hasattr(a, "cpu"):
        a = a.cpu().numpy()
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def _check(rec, ids, sizes, cat, n_groups, n_cat):
    where = rec["name"]
    assert n_groups == rec["n_groups"], where
    assert n_cat == rec["n_catalogue"], where
    assert _sha(ids) == rec["ids_sha256"], f"{where}: ids differ from the oracle"
    assert _sha(sizes) == rec["sizes_sha256"], f"{where}: sizes differ from the oracle"
    assert _sha(cat) == rec["catalogue_sha256"], f"{where}: catalogue differs from the oracle"


def _input_ok(rec, pos):
    assert _sha(pos) == rec["input_sha256"], (
        f"{rec['name']}: the generator produced different input bits on this machine")


def _plain(fof, pos_np, rec):
    """One plan with the library defaults (the benchmark's configuration)."""
    import torch
    n = rec["n"]
    pos = torch.from_numpy(pos_np).cuda()
    ids = torch.empty(n, dtype=torch.int32, device="cuda")
    sizes = torch.empty(n, dtype=torch.int32, device="cuda")
    cap = max(1, rec["n_catalogue"])
    cat = torch.empty((cap, 2), dtype=torch.int32, device="cuda")
    h = fof.fof_create(rec["box"], rec["l_x"], n)
    try:
        fof.fof_link(h, pos)
        _, ng, nk = fof.fof_groups(h, ids, sizes, cat, cap, rec["min_size"])
    finally:
        fof.fof_destroy(h)
    del pos
    return ids, sizes, cat[: nk[0]], ng[0], nk[0]


@pytest.mark.parametrize("which", ["fof-32^3-uniform", "fof-256^3-clustered"])
def test_small_configs_hash(cuda_lib, which):
    rec = {r["name"]: r for r in _records("small")}[which]
    c = synth.uniform_32k() if which.endswith("uniform") else synth.clustered_256()
    pos = c["make"]()
    _input_ok(rec, pos)
    _check(rec, *_plain(cuda_lib, pos, rec))


def test_clustered_1024_hash(cuda_lib):
    import torch
    rec = _records("clustered_1024")[0]
    pos = synth.clustered_1024()["make"]()
    _input_ok(rec, pos)
    out = _plain(cuda_lib, pos, rec)
    del pos
    _check(rec, *out)
    del out
    torch.cuda.empty_cache()


def test_batch_512_hash(cuda_lib):
    """The 512-box batch in one plan with the library defaults, replayed as a CUDA graph."""
    import torch
    fof = cuda_lib
    recs = _records("batch_512")
    specs = synth.batch_512()
    assert len(recs) == len(specs)
    poss = [synth.make_batch_box(sp) for sp in specs]
    for rec, pos in zip(recs, poss):
        _input_ok(rec, pos)
    ns = [sp["n"] for sp in specs]
    total = sum(ns)
    concat = torch.from_numpy(np.concatenate(poss)).cuda()
    del poss
    ids = torch.empty(total, dtype=torch.int32, device="cuda")
    sizes = torch.empty(total, dtype=torch.int32, device="cuda")
    cap = sum(r["n_catalogue"] for r in recs) + 1
    cat = torch.empty((cap, 2), dtype=torch.int32, device="cuda")
    h = fof.fof_batch_create([sp["box"] for sp in specs], [sp["l_x"] for sp in specs], ns)
    s = torch.cuda.Stream()
    try:
        torch.cuda.synchronize()
        fof.fof_graph_build(h, concat, ids, sizes, cat, cap, 20, s)
        for _ in range(2):                      # a replay reproduces the result
            ids.fill_(-1)
            torch.cuda.synchronize()
            fof.fof_graph_launch(h, s)
            _, ng, nk = fof.fof_result(h, len(specs), s)
    finally:
        fof.fof_destroy(h)
    ids, sizes, cat = ids.cpu().numpy(), sizes.cpu().numpy(), cat.cpu().numpy()
    off = np.concatenate([[0], np.cumsum(ns)])
    koff = np.concatenate([[0], np.cumsum(nk)])
    for b, rec in enumerate(recs):
        _check(rec, ids[off[b]:off[b + 1]], sizes[off[b]:off[b + 1]], cat[koff[b]:koff[b + 1]],
               ng[b], nk[b])


def test_served_pool_hash(cuda_lib):
    """Every input of the served workload's pool, submitted at once to the server."""
    import torch
    from paper_2003_11468_gb300.server import Server
    recs = _records("served_pool")
    pool = synth.served_pool()
    assert len(recs) == len(pool)
    inputs = []
    for rec, sp in zip(recs, pool):
        pos = synth.make_served(sp)
        _input_ok(rec, pos)
        inputs.append(torch.from_numpy(pos).pin_memory())
    with Server(memory_budget=120 << 30, slots=3) as srv:
        futs = [srv.submit(p, sp["box"], sp["l_x"], sp["min_size"]) for p, sp in zip(inputs, pool)]
        res = [f.result(timeout=600) for f in futs]
    for rec, r in zip(recs, res):
        _check(rec, r.ids, r.sizes, r.catalogue, r.n_groups, r.catalogue.shape[0])
