"""Autotuner: candidate grid, option mapping, cache (CPU); on the GPU the
tuned plan must give the oracle's partition and a second call must hit the
cache."""
import json

import numpy as np
import pytest

from paper_2003_11468_gb300 import tune


def test_candidate_grid_and_options():
    c = tune.candidates()
    assert len(c) == 3 * 3 * 3
    assert len({json.dumps(x, sort_keys=True) for x in c}) == len(c)
    o = tune.options_from({"occupancy": 0.25, "dense_min": 192, "team_min": 6, "brick_cells": 8})
    assert (o.occupancy, o.dense_min, o.team_min, o.brick_cells) == (0.25, 192, 6, 8)
    assert o.cells_per_axis == 0 and o.retry_cap == 0           # library defaults kept
    assert tune.options_from(None) is None


def test_shape_key_groups_equal_shapes():
    k1 = tune.shape_key([100.0], [0.2 * 100 / 256], [256 ** 3])
    k2 = tune.shape_key([50.0], [0.2 * 50 / 256], [256 ** 3])     # same n and l_x / separation
    k3 = tune.shape_key([100.0], [0.3 * 100 / 256], [256 ** 3])
    assert k1 == k2 != k3
    assert k1.startswith("boxes1_n2^24_b0.20")
    kb = tune.shape_key([10.0, 20.0], [0.1, 0.2], [1000, 8000])
    assert kb.startswith("boxes2_")


def test_cache_round_trip(tmp_path):
    p = tmp_path / "sub" / "tune.json"
    c = tune.TuneCache(str(p))
    assert c.get("k") is None
    c.put("k", {"occupancy": 0.35})
    c.put("j", {"dense_min": 256})
    c2 = tune.TuneCache(str(p))
    assert c2.get("k") == {"occupancy": 0.35} and c2.get("j") == {"dense_min": 256}
    mem = tune.TuneCache("")                                     # no file: memory only
    mem.put("k", {"team_min": 4})
    assert mem.get("k") == {"team_min": 4}


@pytest.mark.gpu
def test_tuned_plan_is_exact_and_cached(cuda_lib, tmp_path):
    import torch
    import oracle
    from paper_2003_11468_gb300 import synth
    fof = cuda_lib
    n, box = 150000, 30.0
    l_x = synth.linking_length(n, box)
    pos = synth.clustered_box(n, box, 60, seed=77)
    pd = torch.from_numpy(pos).cuda()
    grid = {"occupancy": (0.35, 0.7), "dense_min": (128,), "team_min": (4, 8)}
    path = str(tmp_path / "tune.json")
    opt, rep = tune.tune([box], [l_x], [n], pd, grid=grid, cache=path)
    assert not rep["cached"] and len(rep["ms"]) == 4 and rep["best"] in tune.candidates(grid)
    with fof.FoF(box, l_x, n, opt) as f:
        ids, sizes, cat, ng = f.run(pd, min_size=20)
    wid, wsz = oracle.groups(pos, box, l_x)
    assert np.array_equal(ids.cpu().numpy(), wid) and np.array_equal(sizes.cpu().numpy(), wsz)
    opt2, rep2 = tune.tune([box], [l_x], [n], pd, grid=grid, cache=path)
    assert rep2["cached"] and rep2["best"] == rep["best"]
    # a batch of two boxes tunes through the batch plan
    p2 = synth.clustered_box(40000, 12.0, 20, seed=78)
    cat2 = torch.from_numpy(np.concatenate([pos, p2])).cuda()
    optb, repb = tune.tune([box, 12.0], [l_x, synth.linking_length(40000, 12.0)], [n, 40000], cat2,
                           grid={"occupancy": (0.35, 0.5)})
    assert repb["key"].startswith("boxes2_") and len(repb["ms"]) == 2
