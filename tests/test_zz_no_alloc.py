"""fof_run_noalloc: the allocation-free entry point for callers that cannot
allocate device memory (an application that owns all GPU memory, or a loop
that must not call cudaMalloc).  It must give exactly what the plan-based
entry points give, call after call, although every call reuses the same
fixed scratch array.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2003_11468_gb300 import synth

pytestmark = pytest.mark.gpu


def _with_plan(fof, pos_dev, box, l_x, min_size, cap):
    import torch
    n = pos_dev.shape[0]
    ids = torch.empty(n, dtype=torch.int32, device="cuda")
    sizes = torch.empty(n, dtype=torch.int32, device="cuda")
    cat = torch.empty((cap, 2), dtype=torch.int32, device="cuda")
    h = fof.fof_create(box, l_x, n)
    try:
        fof.fof_link(h, pos_dev)
        code, ng, nk = fof.fof_groups(h, ids, sizes, cat, cap, min_size)
    finally:
        fof.fof_destroy(h)
    return code, ids.cpu().numpy(), sizes.cpu().numpy(), cat.cpu().numpy()[: nk[0]], ng[0], nk[0]


def _no_alloc(fof, pos_dev, box, l_x, min_size, cap):
    import torch
    n = pos_dev.shape[0]
    ids = torch.full((n,), -3, dtype=torch.int32, device="cuda")
    sizes = torch.full((n,), -3, dtype=torch.int32, device="cuda")
    cat = torch.full((cap, 2), -3, dtype=torch.int32, device="cuda")
    code, ng, nk = fof.fof_run_noalloc(box, l_x, n, pos_dev, ids, sizes, cat, cap, min_size,
                                       torch.cuda.current_stream())
    return code, ids.cpu().numpy(), sizes.cpu().numpy(), cat.cpu().numpy()[:nk], ng, nk


def test_no_alloc_matches_plan_path_twice(cuda_lib):
    import torch
    fof = cuda_lib
    cases = [
        (synth.clustered_box(200000, 40.0, 150, seed=901), 40.0, synth.linking_length(200000, 40.0), 20),
        (synth.uniform_box(50000, 3.0, seed=902), 3.0, synth.linking_length(50000, 3.0, 0.4), 2),
    ]
    # two calls in a row, different geometries: leftovers of the first call
    # in the shared scratch must not leak into the second
    for pos, box, l_x, min_size in cases:
        dpos = torch.from_numpy(pos).cuda()
        cap = pos.shape[0]
        want = _with_plan(fof, dpos, box, l_x, min_size, cap)
        got = _no_alloc(fof, dpos, box, l_x, min_size, cap)
        assert got[0] == want[0] == 0
        for g, w in zip(got[1:4], want[1:4]):
            assert np.array_equal(g, w)
        assert got[4:] == want[4:]


def test_no_alloc_rejects_oversize(cuda_lib):
    fof = cuda_lib
    with pytest.raises(fof.FoFError) as ei:
        fof.fof_run_noalloc(100.0, 0.05, 5_000_000, None, None, None, None, 0, 1)
    assert ei.value.code == fof.FOF_ERR_TOO_LARGE
