"""Parity at the full workload sizes, in the launch configuration bench.py times.

* 256^3 clustered box: the whole oracle runs, every output is compared.
* 1024^3 clustered box: the oracle cannot label 1.07e9 particles in a test,
  so (a) sampled particles have their whole group recomputed by the oracle's
  breadth-first search on a periodic sub-cube around them (grown until the
  group lies at least 1.05 l_x inside it, so no outside particle can link
  to it), and every member's id, the label and the size are compared; and
  (b) properties that hold at any size are checked on all outputs.
"""
import numpy as np
import pytest

import oracle
from paper_2003_11468_gb300 import synth

pytestmark = pytest.mark.gpu


def _gpu_run(fof, pos_dev, c, cap):
    import torch
    n = c["n"]
    ids = torch.empty(n, dtype=torch.int32, device="cuda")
    sizes = torch.empty(n, dtype=torch.int32, device="cuda")
    cat = torch.empty((cap, 2), dtype=torch.int32, device="cuda")
    h = fof.fof_create(c["box"], c["l_x"], n)       # the bench's plan: all defaults
    try:
        fof.fof_link(h, pos_dev)
        code, ng, nk = fof.fof_groups(h, ids, sizes, cat, cap, c["min_size"])
    finally:
        fof.fof_destroy(h)
    return ids, sizes, cat[: nk[0]], ng[0]


def test_clustered_256_full(cuda_lib):
    import torch
    c = synth.clustered_256()
    pos = c["make"]()
    ids, sizes, cat, ng = _gpu_run(cuda_lib, torch.from_numpy(pos).cuda(), c, c["n"])
    wid, wsz = oracle.groups(pos, c["box"], c["l_x"])
    wcat = oracle.catalogue(wsz, c["min_size"])
    got = ids.cpu().numpy()
    bad = np.nonzero(got != wid)[0]
    assert bad.size == 0, f"{bad.size} ids differ"
    assert np.array_equal(sizes.cpu().numpy(), wsz)
    assert np.array_equal(cat.cpu().numpy(), wcat)
    assert ng == int((wsz > 0).sum())


def _component_in_cube(pos_dev, pos_np, box, l_x, i, w0=0.5):
    """Oracle group of particle i from a periodic sub-cube around it.

    The cube is selected with float32 offsets (rounding ~1e-5 of the box
    side); the group must sit 1.05 l_x inside the cube, a margin far above
    that rounding, so every particle within l_x of a member is in the cube.
    """
    import torch
    c = pos_dev[i].clone()
    w = w0
    while True:
        d = pos_dev - c
        d.add_(0.5 * box).remainder_(box).sub_(0.5 * box).abs_()
        dmax = d.amax(dim=1)
        del d
        sel = torch.nonzero(dmax <= w).squeeze(1)
        sel_np = sel.cpu().numpy()
        start = int(np.searchsorted(sel_np, i))
        assert sel_np[start] == i
        _, members = oracle.component(pos_np[sel_np], box, l_x, start)
        gm = sel_np[members]
        depth = dmax[sel[torch.from_numpy(members).cuda().long()]].max().item()
        del dmax
        if depth <= w - 1.05 * l_x or w >= 0.5 * box:
            return int(gm.min()), gm
        w *= 2.0


def test_clustered_1024_sampled(cuda_lib):
    import torch
    c = synth.clustered_1024()
    pos = c["make"]()
    n = c["n"]
    pos_dev = torch.from_numpy(pos).cuda()
    cap = 1 << 24
    ids, sizes, cat, ng = _gpu_run(cuda_lib, pos_dev, c, cap)

    # (b) properties at full size
    idx = torch.arange(n, device="cuda", dtype=torch.int32)
    assert bool((ids <= idx).all())
    assert bool((ids[ids.long()] == ids).all())
    assert int(sizes.sum(dtype=torch.int64)) == n
    labels = torch.nonzero(sizes > 0).squeeze(1)
    assert labels.numel() == ng
    assert bool((ids[labels] == labels.int()).all())
    counts = torch.bincount(ids.long(), minlength=n)
    assert bool((counts.int() == sizes).all())
    want_cat = torch.nonzero(sizes >= c["min_size"]).squeeze(1)
    assert cat.shape[0] == want_cat.numel()
    assert bool((cat[:, 0].long() == want_cat).all())
    assert bool((cat[:, 1] == sizes[want_cat]).all())
    del idx, counts

    # (a) sampled groups recomputed by the oracle
    rng = np.random.default_rng(1024)
    samples = list(rng.integers(0, n, size=16))
    big = torch.argsort(cat[:, 1], descending=True)[:2]
    samples += [int(cat[k, 0]) for k in big.tolist()]
    ids_np = ids.cpu().numpy()
    sizes_np = sizes.cpu().numpy()
    for i in samples:
        lab, members = _component_in_cube(pos_dev, pos, c["box"], c["l_x"], int(i))
        assert ids_np[i] == lab
        assert sizes_np[lab] == members.size
        assert (ids_np[members] == lab).all()
