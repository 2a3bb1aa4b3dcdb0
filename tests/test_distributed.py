"""The distributed group finder (paper Sec. 3.3) on gloo ranks (CPU).

A periodic box is cut into x-slabs, one per rank; each rank finds the
groups of its own particles plus ghosts, the boundary links are all-gathered
and merged with the library's union-find (fof_merge_links, host code).  On
CPU the local step is the oracle (injected), so these tests check the
exchange, the global ids, the links and the merge; the GPU local step is
covered by test_distributed_gpu_local_step (two ranks on one GPU, each with
its own independent kernels).  The
result must equal the oracle run on the whole box in the ranks' global order.
"""
import json
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _box(case):
    """Positions, box side and l_x of a test case (the same on every rank)."""
    sys.path.insert(0, ROOT)
    from paper_2003_11468_gb300 import synth
    if case == "clustered":
        n, box = 6000, 10.0
        pos = synth.clustered_box(n, box, 25, seed=4242)
        return pos, box, synth.linking_length(n, box, 0.35)
    # a filament along x through every slab, wrapping around the box, plus
    # noise: one group spans all ranks and closes through the periodic edge
    box, l_x = 8.0, 0.1
    t = np.arange(0.0, box, 0.07)
    line = np.stack([t, 4.0 + 0.02 * np.sin(t), np.full_like(t, 3.0)], axis=1)
    rng = np.random.default_rng(5)
    noise = rng.random((900, 3)) * box
    pos = np.concatenate([noise, line]).astype(np.float32)
    pos[pos >= np.float32(box)] = 0.0
    return pos, box, l_x


def _global_order(pos, box, world):
    from paper_2003_11468_gb300 import distributed
    r = distributed.slab_of(pos[:, 0], box, world)
    return np.argsort(r, kind="stable")


def _rank_main(rank, world, port, out_dir, case, gpu=False):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_2003_11468_gb300 import distributed
        pos, box, l_x = _box(case)
        order = _global_order(pos, box, world)
        mine = pos[order][distributed.slab_of(pos[order][:, 0], box, world) == rank]

        def local(p, b, l):
            return oracle.groups(p, b, l)[0]
        gid0, labels, cat = distributed.distributed_groups(mine, box, l_x, min_size=3,
                                                           local_fof=None if gpu else local)
        np.save(os.path.join(out_dir, f"labels{rank}.npy"), labels)
        np.save(os.path.join(out_dir, f"cat{rank}.npy"), cat)
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"gid0": gid0, "n": int(mine.shape[0])}, f)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _check(tmp_path, world, case):
    sys.path.insert(0, ROOT)
    import oracle
    pos, box, l_x = _box(case)
    order = _global_order(pos, box, world)
    want_ids, want_sizes = oracle.groups(pos[order], box, l_x)
    got = []
    cats = []
    off = 0
    for r in range(world):
        meta = json.load(open(tmp_path / f"rank{r}.json"))
        assert meta["gid0"] == off                       # exclusive scan of the counts
        off += meta["n"]
        got.append(np.load(tmp_path / f"labels{r}.npy"))
        cats.append(np.load(tmp_path / f"cat{r}.npy"))
    got = np.concatenate(got)
    assert np.array_equal(got, want_ids.astype(np.int64))
    cat = np.concatenate([c for c in cats if c.size]) if any(c.size for c in cats) else np.zeros((0, 2))
    cat = cat[np.argsort(cat[:, 0])] if cat.size else cat
    assert np.array_equal(cat, oracle.catalogue(want_sizes, 3).astype(np.int64))
    # the case is not trivial: some group spans ranks
    gs = want_ids
    owner = np.repeat(np.arange(world), np.diff(np.searchsorted(
        np.arange(pos.shape[0]), [0] + [json.load(open(tmp_path / f"rank{r}.json"))["gid0"]
                                        for r in range(1, world)] + [pos.shape[0]])))
    spans = {g for g in np.unique(gs) if np.unique(owner[gs == g]).size > 1}
    assert spans
    if case == "filament":
        assert any(np.unique(owner[gs == g]).size == world for g in spans)


@pytest.mark.parametrize("world,case", [(2, "clustered"), (3, "clustered"), (4, "filament")])
def test_distributed_equals_whole_box(tmp_path, world, case):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(world, port, str(tmp_path), case), nprocs=world,
                       start_method="spawn")
    _check(tmp_path, world, case)


@pytest.mark.gpu
@pytest.mark.parametrize("case", ["clustered", "filament"])
def test_distributed_gpu_local_step(tmp_path, case):
    """Two ranks on the one GPU, each running the library on its slab plus
    ghosts (their kernels are independent; only the host merge exchanges
    data, over gloo)."""
    import torch
    import torch.multiprocessing as mp
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path), case, True), nprocs=2,
                       start_method="spawn")
    _check(tmp_path, 2, case)


def test_merge_links_pins():
    """fof_merge_links against a plain connected-components computation:
    smallest id per set, indirect links, union by weight, absent ids."""
    sys.path.insert(0, ROOT)
    import networkx as nx
    from paper_2003_11468_gb300 import fof
    rng = np.random.default_rng(3)
    ids = rng.choice(10 ** 12, size=400, replace=False).astype(np.int64)
    a = rng.choice(ids, 300)
    b = rng.choice(ids, 300)
    g = nx.Graph()
    g.add_nodes_from(ids.tolist())
    g.add_edges_from(zip(a.tolist(), b.tolist()))
    comp = {}
    for c in nx.connected_components(g):
        m = min(c)
        for v in c:
            comp[v] = (m, len(c))
    q = np.concatenate([ids, np.array([7, -5], dtype=np.int64)])
    lab, w = fof.fof_merge_links(a, b, q, weight_ids=ids, weights=np.ones(400, np.int64),
                                 want_weights=True)
    for k, v in enumerate(q.tolist()):
        if v in comp:
            assert lab[k] == comp[v][0] and w[k] == comp[v][1]
        else:
            assert lab[k] == v and w[k] == 0
    # a chain of links given in reverse order still reaches the smallest id
    chain = np.arange(100, 0, -1, dtype=np.int64)
    assert (fof.fof_merge_links(chain[:-1], chain[1:], chain) == 1).all()
    assert fof.fof_merge_links(np.zeros(0, np.int64), np.zeros(0, np.int64), np.array([9])).tolist() == [9]
