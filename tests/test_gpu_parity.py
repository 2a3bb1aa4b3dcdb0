"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

The partition is exact, so ids, sizes, the catalogue and the group count
must match the oracle bit for bit on the same seeded inputs.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2003_11468_gb300 import synth

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


def run_gpu(fof, pos, box, l_x, min_size=1, opt=None, cap=None, repeat=1):
    torch = _torch()
    n = pos.shape[0]
    dpos = torch.from_numpy(np.ascontiguousarray(pos, dtype=np.float32)).cuda()
    h = fof.fof_create_ex(box, l_x, n, opt)
    try:
        out = []
        for _ in range(repeat):
            ids = torch.full((n,), -7, dtype=torch.int32, device="cuda")
            sizes = torch.full((n,), -7, dtype=torch.int32, device="cuda")
            c = n if cap is None else cap
            cat = torch.full((max(c, 1), 2), -7, dtype=torch.int32, device="cuda")
            fof.fof_link(h, dpos, torch.cuda.current_stream())
            code, ng, nk = fof.fof_groups(h, ids, sizes, cat, c, min_size, 1,
                                          torch.cuda.current_stream(), allow_capacity=True)
            out.append((code, ids.cpu().numpy(), sizes.cpu().numpy(),
                        cat.cpu().numpy()[: min(nk[0], c)], ng[0], nk[0]))
        return out
    finally:
        fof.fof_destroy(h)


def assert_parity(fof, pos, box, l_x, min_size=1, opt=None, repeat=1, want=None):
    if want is None:
        want = oracle.groups(pos, box, l_x)
    wid, wsz = want
    wcat = oracle.catalogue(wsz, min_size)
    for code, ids, sizes, cat, ng, nk in run_gpu(fof, pos, box, l_x, min_size, opt, repeat=repeat):
        assert code == 0
        bad = np.nonzero(ids != wid)[0]
        assert bad.size == 0, f"{bad.size} ids differ, first {bad[:5]} got {ids[bad[:5]]} want {wid[bad[:5]]}"
        assert np.array_equal(sizes, wsz)
        assert nk == wcat.shape[0]
        assert np.array_equal(cat, wcat)
        assert ng == int((wsz > 0).sum())


# --------------------------------------------------------------------------
# the small configurations
# --------------------------------------------------------------------------

def test_uniform_32k_repeated(cuda_lib):
    c = synth.uniform_32k()
    pos = c["make"]()
    assert_parity(cuda_lib, pos, c["box"], c["l_x"], c["min_size"], repeat=3)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_clustered_small(cuda_lib, seed):
    n, box = 60000 + 7919 * seed, 30.0 + 5 * seed
    pos = synth.clustered_box(n, box, 60 + 20 * seed, seed=300 + seed)
    l_x = synth.linking_length(n, box)
    assert_parity(cuda_lib, pos, box, l_x, 20, repeat=2)


@pytest.mark.parametrize("b", [0.1, 0.35, 0.7, 1.2])
def test_linking_lengths(cuda_lib, b):
    n, box = 40000, 10.0
    pos = synth.clustered_box(n, box, 50, seed=41)
    l_x = min(synth.linking_length(n, box, b), 0.49 * box)
    assert_parity(cuda_lib, pos, box, l_x, 2)


# the plan options are pure performance knobs: results must not change
OPTS = [
    dict(cells_per_axis=1), dict(cells_per_axis=2), dict(cells_per_axis=3),
    dict(cells_per_axis=7, brick_cells=1), dict(cells_per_axis=16, brick_cells=16),
    dict(cells_per_axis=24, brick_cells=8), dict(brick_cells=2), dict(occupancy=0.3),
    dict(occupancy=8.0), dict(dense_min=1), dict(dense_min=1 << 30), dict(dense_min=4),
]


@pytest.mark.parametrize("k", range(len(OPTS)))
def test_plan_options_do_not_change_results(cuda_lib, k):
    n, box = 30000, 12.0
    pos = synth.clustered_box(n, box, 40, seed=55)
    l_x = synth.linking_length(n, box, 0.3)
    want = oracle.groups(pos, box, l_x)
    opt = cuda_lib.fof_options()
    for key, v in OPTS[k].items():
        setattr(opt, key, v)
    assert_parity(cuda_lib, pos, box, l_x, 3, opt=opt, want=want)


# --------------------------------------------------------------------------
# closed forms and edge cases
# --------------------------------------------------------------------------

def _lattice(k):
    m = 2 ** k
    g = (np.arange(m, dtype=np.float64) / m).astype(np.float32)
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)


@pytest.mark.parametrize("k", [2, 3, 4, 5])
def test_lattice(cuda_lib, k):
    pos = _lattice(k)
    n = pos.shape[0]
    d = 2.0 ** -k
    (code, ids, sizes, cat, ng, nk), = run_gpu(cuda_lib, pos, 1.0, d, 1)
    assert (ids == 0).all() and sizes[0] == n and ng == 1
    (code, ids, sizes, cat, ng, nk), = run_gpu(cuda_lib, pos, 1.0, float(np.nextafter(d, 0)), 1)
    assert (ids == np.arange(n)).all() and (sizes == 1).all() and ng == n


def test_periodic_chain(cuda_lib):
    from conftest import read_rows
    for r in read_rows("chain_wrap.txt"):
        removed = [] if r[0] == "-" else [int(v) for v in r[0].split(",")]
        keep = [k for k in range(16) if k not in removed]
        pos = np.array([[k / 16.0, 0.5, 0.5] for k in keep], dtype=np.float32)
        want = np.array([int(v) for v in r[1:]], dtype=np.int32)
        (code, ids, sizes, cat, ng, nk), = run_gpu(cuda_lib, pos, 1.0, 1.0 / 16.0)
        assert np.array_equal(ids, want), (r, ids)


def test_tie_pairs(cuda_lib):
    from conftest import read_rows
    for r in read_rows("tie_pairs.txt"):
        box = float(r[0])
        a = [float(v) for v in r[1:4]]
        b = [float(v) for v in r[4:7]]
        l_x, want, exact = float(r[7]), int(r[8]), int(r[9])
        if not l_x < box / 2:
            continue
        pos = np.array([a, b], dtype=np.float32)
        (code, ids, *_), = run_gpu(cuda_lib, pos, box, l_x)
        assert (ids[1] == 0) == bool(want), r
        if exact:
            (code, ids, *_), = run_gpu(cuda_lib, pos, box, float(np.nextafter(l_x, 0)))
            assert ids[1] == 1, r


def test_degenerate(cuda_lib):
    # n = 0
    (code, ids, sizes, cat, ng, nk), = run_gpu(cuda_lib, np.zeros((0, 3), np.float32), 1.0, 0.1)
    assert code == 0 and ids.size == 0 and ng == 0 and nk == 0
    # n = 1
    (code, ids, sizes, cat, ng, nk), = run_gpu(cuda_lib, np.array([[0.3, 0.2, 0.1]], np.float32), 1.0, 0.1)
    assert ids.tolist() == [0] and sizes.tolist() == [1] and ng == 1
    # everything at one point: one group, and the dense path has one huge cell
    same = np.tile(np.array([[0.7, 0.7, 0.7]], dtype=np.float32), (5000, 1))
    assert_parity(cuda_lib, same, 1.0, 1e-6, 2)
    # 0 and L - ulp link through the wrap, on every axis
    u = np.float32(1) - np.float32(2 ** -24)
    edge = np.array([[0, 0.5, 0.5], [0.5, 0.5, 0.5], [u, 0.5, 0.5], [0.5, 0, 0.25], [0.5, u, 0.25],
                     [0.25, 0.25, 0], [0.25, 0.25, u]], dtype=np.float32)
    assert_parity(cuda_lib, edge, 1.0, 1e-6)


def test_cell_boundaries_exact(cuda_lib):
    """Particles exactly on cell boundaries and pairs exactly l_x apart across them."""
    box, nc = 1.0, 16
    l_x = 1.0 / 32
    g = np.arange(0, 64, dtype=np.float64) / 64        # multiples of 1/64 hit cell edges
    rng = np.random.default_rng(5)
    pos = g[rng.integers(0, 64, size=(3000, 3))].astype(np.float32)
    opt = cuda_lib.fof_options()
    opt.cells_per_axis = 31
    assert_parity(cuda_lib, pos, box, l_x, 2)
    assert_parity(cuda_lib, pos, box, l_x, 2, opt=opt)


def test_near_threshold_pairs(cuda_lib):
    """Pairs whose double-precision distance sits within a few ulps of l_x:
    the float32 pre-test must hand every one of them to the exact test."""
    rng = np.random.default_rng(11)
    box = 100.0
    l_x = 0.0195312
    m = 4000
    a = rng.random((m, 3)) * box
    d = rng.normal(size=(m, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    scale = l_x * (1 + rng.integers(-40, 41, size=m) * 2.0 ** -24)
    b = a + d * scale[:, None]
    pos = np.empty((2 * m, 3), dtype=np.float32)
    pos[0::2] = (a % box).astype(np.float32)
    pos[1::2] = (b % box).astype(np.float32)
    pos[pos >= np.float32(box)] = 0
    # spread pairs far apart so each pair is its own problem
    want = oracle.groups(pos, box, l_x)
    linked = (want[0][1::2] == want[0][0::2]).mean()
    assert 0.2 < linked < 0.8       # both sides of the threshold are exercised
    assert_parity(cuda_lib, pos, box, l_x, 2, want=want)


def test_permutation_invariance(cuda_lib):
    n, box = 50000, 15.0
    pos = synth.clustered_box(n, box, 80, seed=61)
    l_x = synth.linking_length(n, box)
    perm = np.random.default_rng(2).permutation(n)
    (_, ids, sizes, _, ng, _), = run_gpu(cuda_lib, pos, box, l_x)
    (_, ids_p, sizes_p, _, ng_p, _), = run_gpu(cuda_lib, pos[perm], box, l_x)
    assert ng == ng_p
    # group of particle perm[k] in the original == group of k in the permuted
    a, b = ids[perm], ids_p
    pairs = set(zip(a.tolist(), b.tolist()))
    assert len(pairs) == len(set(a.tolist())) == len(set(b.tolist()))


# --------------------------------------------------------------------------
# errors
# --------------------------------------------------------------------------

def test_range_errors(cuda_lib):
    torch = _torch()
    fof = cuda_lib
    base = synth.uniform_box(1000, 1.0, 3)
    for bad in (np.nan, -1e-7, 1.0, 1.5, np.inf):
        pos = base.copy()
        pos[417, 1] = bad
        dpos = torch.from_numpy(pos).cuda()
        h = fof.fof_create(1.0, 0.02, 1000)
        try:
            ids = torch.empty(1000, dtype=torch.int32, device="cuda")
            sizes = torch.empty(1000, dtype=torch.int32, device="cuda")
            fof.fof_link(h, dpos)
            with pytest.raises(fof.FoFError) as ei:
                fof.fof_groups(h, ids, sizes, None, 0, 1)
            assert ei.value.code == fof.FOF_ERR_RANGE
            # the handle stays usable with valid input
            fof.fof_link(h, torch.from_numpy(base).cuda())
            code, ng, nk = fof.fof_groups(h, ids, sizes, None, 0, 1)
            assert code == 0
        finally:
            fof.fof_destroy(h)


def test_state_and_capacity(cuda_lib):
    torch = _torch()
    fof = cuda_lib
    c = synth.uniform_32k()
    pos = c["make"]()
    wid, wsz = oracle.groups(pos, c["box"], c["l_x"])
    wcat = oracle.catalogue(wsz, 2)
    h = fof.fof_create(c["box"], c["l_x"], c["n"])
    try:
        ids = torch.empty(c["n"], dtype=torch.int32, device="cuda")
        sizes = torch.empty(c["n"], dtype=torch.int32, device="cuda")
        with pytest.raises(fof.FoFError) as ei:
            fof.fof_groups(h, ids, sizes, None, 0, 2)
        assert ei.value.code == fof.FOF_ERR_STATE
        fof.fof_link(h, torch.from_numpy(pos).cuda())
        cap = 100
        cat = torch.full((cap, 2), -1, dtype=torch.int32, device="cuda")
        code, ng, nk = fof.fof_groups(h, ids, sizes, cat, cap, 2, allow_capacity=True)
        assert code == fof.FOF_ERR_CAPACITY and nk[0] == wcat.shape[0] > cap
        assert np.array_equal(cat.cpu().numpy(), wcat[:cap])
        assert np.array_equal(ids.cpu().numpy(), wid)
    finally:
        fof.fof_destroy(h)


def test_retry_cap_exhaustion_reports_timeout(cuda_lib):
    """With FOF_DEBUG_UNION_NO_RETRY every Union gives up before its first
    CAS, as a union that exhausted its retry cap does.  The 32^3 uniform box
    has hundreds of linked pairs between sparse cells, so unions are certain
    to be attempted: the library must report FOF_ERR_TIMEOUT, never a
    partition.  The same plan options without the flag give the exact
    answer."""
    import oracle
    torch = _torch()
    fof = cuda_lib
    c = synth.uniform_32k()
    pos = c["make"]()
    n = c["n"]
    wid, _ = oracle.groups(pos, c["box"], c["l_x"])
    assert (wid != np.arange(n)).any()            # some pairs are linked
    dev = torch.from_numpy(pos).cuda()
    ids = torch.empty(n, dtype=torch.int32, device="cuda")
    sizes = torch.empty(n, dtype=torch.int32, device="cuda")
    for flag in (fof.FOF_DEBUG_UNION_NO_RETRY, 0):
        opt = fof.fof_options()
        opt.debug_flags = flag
        h = fof.fof_create_ex(c["box"], c["l_x"], n, opt)
        try:
            fof.fof_link(h, dev)
            if flag:
                with pytest.raises(fof.FoFError) as e:
                    fof.fof_groups(h, ids, sizes, None, 0, 1)
                assert e.value.code == fof.FOF_ERR_TIMEOUT
            else:
                fof.fof_groups(h, ids, sizes, None, 0, 1)
                assert np.array_equal(ids.cpu().numpy(), wid)
        finally:
            fof.fof_destroy(h)


# --------------------------------------------------------------------------
# other entry points
# --------------------------------------------------------------------------

def test_run_host_matches_device_path(cuda_lib):
    torch = _torch()
    fof = cuda_lib
    n, box = 70000, 25.0
    pos = synth.clustered_box(n, box, 90, seed=71)
    l_x = synth.linking_length(n, box)
    wid, wsz = oracle.groups(pos, box, l_x)
    wcat = oracle.catalogue(wsz, 20)
    h = fof.fof_create(box, l_x, n)
    try:
        ph = torch.from_numpy(pos).pin_memory()
        ids = torch.empty(n, dtype=torch.int32).pin_memory()
        sizes = torch.empty(n, dtype=torch.int32).pin_memory()
        cat = torch.empty((n, 2), dtype=torch.int32).pin_memory()
        for _ in range(2):
            code, ng, nk = fof.fof_run_host(h, ph, ids, sizes, cat, n, 20)
            assert code == 0
            assert np.array_equal(ids.numpy(), wid) and np.array_equal(sizes.numpy(), wsz)
            assert np.array_equal(cat.numpy()[: nk[0]], wcat)
    finally:
        fof.fof_destroy(h)


def test_graph_replay(cuda_lib):
    torch = _torch()
    fof = cuda_lib
    n, box = 50000, 20.0
    pos = synth.clustered_box(n, box, 70, seed=81)
    l_x = synth.linking_length(n, box)
    wid, wsz = oracle.groups(pos, box, l_x)
    s = torch.cuda.Stream()
    h = fof.fof_create(box, l_x, n)
    try:
        dpos = torch.from_numpy(pos).cuda()
        ids = torch.empty(n, dtype=torch.int32, device="cuda")
        sizes = torch.empty(n, dtype=torch.int32, device="cuda")
        cat = torch.empty((n, 2), dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        fof.fof_graph_build(h, dpos, ids, sizes, cat, n, 20, s)
        for _ in range(3):
            ids.fill_(-1)
            torch.cuda.synchronize()
            fof.fof_graph_launch(h, s)
            code, ng, nk = fof.fof_result(h, 1, s)
            assert code == 0
            assert np.array_equal(ids.cpu().numpy(), wid) and np.array_equal(sizes.cpu().numpy(), wsz)
    finally:
        fof.fof_destroy(h)


def test_phase_timing_and_launch_count(cuda_lib):
    torch = _torch()
    fof = cuda_lib
    c = synth.uniform_32k()
    pos = torch.from_numpy(c["make"]()).cuda()
    h = fof.fof_create(c["box"], c["l_x"], c["n"])
    try:
        fof.fof_set_timing(h, True)
        ids = torch.empty(c["n"], dtype=torch.int32, device="cuda")
        sizes = torch.empty(c["n"], dtype=torch.int32, device="cuda")
        for _ in range(2):
            fof.fof_link(h, pos)
            fof.fof_groups(h, ids, sizes, None, 0, 2)
        t = fof.fof_phase_times(h)
        assert set(t) >= {"bin_count", "link", "finalize", "outputs", "catalogue"}
        assert all(ms >= 0 for ms, _ in t.values()) and t["link"][0] > 0
        per_run = sum(k for _, k in t.values()) // 2
        assert fof.fof_kernel_launches(h) == 2 * per_run
    finally:
        fof.fof_destroy(h)


# --------------------------------------------------------------------------
# team cells in z order: block pairs pruned by their z gap, neighbour streams
# cut to a z-prefix (cells sorted by k_team_self, searched in k_link)
# --------------------------------------------------------------------------

def _layered_cells(seed, nc=8, box=8.0, n_bg=3000, n_cells=40):
    rng = np.random.default_rng(seed)
    h = box / nc
    parts = [rng.uniform(0.0, box, size=(n_bg, 3))]
    cells = rng.integers(0, nc, size=(n_cells, 3))
    cells[:8, 2] = nc - 1                      # some at the top row: wrap to z = 0
    for c in cells:
        m = int(rng.integers(20, 240))          # both sides of the 32-particle sort threshold
        layers = rng.choice([0.03, 0.3, 0.6, 0.97], size=int(rng.integers(2, 5)), replace=False)
        lay = layers[rng.integers(0, len(layers), size=m)]
        p = np.empty((m, 3))
        p[:, 0] = (c[0] + rng.uniform(0.0, 1.0, m)) * h
        p[:, 1] = (c[1] + rng.uniform(0.0, 1.0, m)) * h
        p[:, 2] = (c[2] + np.clip(lay + rng.normal(0.0, 0.01, m), 0.0, 0.999)) * h
        parts.append(p)
    pos = np.concatenate(parts) % box
    pos = pos.astype(np.float32)
    pos[pos >= np.float32(box)] = 0.0
    return pos[rng.permutation(pos.shape[0])]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_zsorted_team_cells(cuda_lib, seed):
    box, l_x = 8.0, 0.3
    pos = _layered_cells(seed)
    want = oracle.groups(pos, box, l_x)
    opt = cuda_lib.fof_options()
    opt.cells_per_axis = 8
    opt.dense_min = 1 << 30                    # no sub-cells: every large cell is a team cell
    assert_parity(cuda_lib, pos, box, l_x, 5, opt=opt, repeat=2, want=want)
    assert_parity(cuda_lib, pos, box, l_x, 5, want=want)      # default cell grid


@pytest.mark.parametrize("seed", range(3))
def test_tie_rule_option(cuda_lib, seed):
    """FOF_TIE_LT (distance < l_x, the naive listing of Sec. 3.1) against the
    oracle's strict rule, on grid points where many pairs are exactly l_x
    apart; the default rule on the same input for contrast."""
    torch = _torch()
    fof = cuda_lib
    rng = np.random.default_rng(900 + seed)
    n = 20000
    g = 2.0 ** -5
    pos = (rng.integers(0, 32, size=(n, 3)) * g).astype(np.float32)
    dev = torch.from_numpy(pos).cuda()
    for strict in (True, False):
        opt = fof.fof_options()
        opt.tie_rule = fof.FOF_TIE_LT if strict else fof.FOF_TIE_LE
        with fof.FoF(1.0, g, n, opt) as f:
            ids, sizes, _, _ = f.run(dev)
        wid, wsz = oracle.groups(pos, 1.0, g, strict=strict)
        assert np.array_equal(ids.cpu().numpy(), wid), strict
        assert np.array_equal(sizes.cpu().numpy(), wsz), strict


@pytest.mark.parametrize("find,link,size", [
    (0, 0, 1), (1, 0, 0), (2, 0, 0), (3, 0, 0),
    (0, 1, 0), (1, 1, 1), (2, 1, 0), (3, 1, 1),
])
def test_union_find_variants(cuda_lib, find, link, size):
    """Every union-find variant of fof.h (compression of Find, Sec. 3.4.3;
    randomised linking, Sec. 3.2; hash-table size count, Sec. 3.4.1) gives
    exactly the oracle's partition, sizes and catalogue on a clustered box
    with dense, team and sparse cells."""
    torch = _torch()
    fof = cuda_lib
    n, box = 300000, 30.0
    pos = synth.clustered_box(n, box, 120, seed=700 + 10 * find + 3 * link + size)
    l_x = synth.linking_length(n, box, 0.25)
    opt = fof.fof_options()
    opt.find_variant, opt.link_order, opt.size_count = find, link, size
    with fof.FoF(box, l_x, n, opt) as f:
        ids, sizes, cat, ng = f.run(torch.from_numpy(pos).cuda(), min_size=10)
    wid, wsz = oracle.groups(pos, box, l_x)
    assert np.array_equal(ids.cpu().numpy(), wid)
    assert np.array_equal(sizes.cpu().numpy(), wsz)
    assert np.array_equal(cat.cpu().numpy(), oracle.catalogue(wsz, 10))
    assert ng == int((wsz > 0).sum())


def test_relink_paths(cuda_lib):
    """fof_relink on moved particles: every path gives the oracle's answer for
    the new positions.  Unmoved particles take path 0 (cells re-used),
    particles moved toward their cell's centre path 1 or 0 (no brick change
    possible), large moves path 2 (full re-binning)."""
    torch = _torch()
    fof = cuda_lib
    n, box = 200000, 25.0
    pos = synth.clustered_box(n, box, 90, seed=811)
    l_x = synth.linking_length(n, box, 0.3)
    geo = fof.fof_box_geometry(box, l_x, n)
    q, inv = geo.sub_cells, np.float32(geo.inv_fine)

    def cells(p):
        f = np.minimum((p * inv).astype(np.int32), geo.fine_per_axis - 1)
        return f // q

    # toward the cell centre by 30%: no particle crosses a cell face
    c = cells(pos)
    centre = ((c.astype(np.float64) + 0.5) * q / float(inv)).astype(np.float32)
    near = (pos + np.float32(0.3) * (centre - pos)).astype(np.float32)
    stay = (cells(near) == c).all(axis=1)
    near[~stay] = pos[~stay]
    rng = np.random.default_rng(3)
    far = np.mod(pos + rng.normal(0, 0.4, pos.shape), box).astype(np.float32)
    far[far >= np.float32(box)] = 0.0
    ids = torch.empty(n, dtype=torch.int32, device="cuda")
    sizes = torch.empty(n, dtype=torch.int32, device="cuda")
    h = fof.fof_create(box, l_x, n)
    try:
        fof.fof_link(h, torch.from_numpy(pos).cuda())
        fof.fof_groups(h, ids, sizes, None, 0, 1)
        for p, allowed in ((pos, (0,)), (near, (0, 1)), (far, (2,)), (far, (0,)), (pos, (1, 2))):
            dev = torch.from_numpy(np.ascontiguousarray(p)).cuda()
            path = fof.fof_relink(h, dev)
            assert path in allowed
            fof.fof_groups(h, ids, sizes, None, 0, 1)
            wid, wsz = oracle.groups(p, box, l_x)
            assert np.array_equal(ids.cpu().numpy(), wid), path
            assert np.array_equal(sizes.cpu().numpy(), wsz), path
    finally:
        fof.fof_destroy(h)


def _big_cell_box(seed):
    """One cell of side 6.5 l_x holding 50,000 particles in 8 tight blobs (a
    2x2x2 lattice 3.25 l_x apart, so most stay separate groups), inside a
    10^3-cell box with a sparse background and a blob straddling the big
    cell's +x face."""
    rng = np.random.default_rng(seed)
    l_x, h, nc = 0.1, 0.65, 10
    box = h * nc
    lo = np.array([h, h, h])
    g = np.array([[i, j, k] for i in (0.25, 0.75) for j in (0.25, 0.75) for k in (0.25, 0.75)])
    cent = lo + g * h
    inside = cent[rng.integers(0, 8, 50000)] + rng.normal(0, 0.2 * l_x, (50000, 3))
    inside = np.clip(inside, lo, lo + h * (1 - 1e-6))
    edge = np.array([2 * h, 1.5 * h, 1.5 * h]) + rng.normal(0, 0.4 * l_x, (3000, 3))
    bg = rng.random((20000, 3)) * box
    pos = np.mod(np.concatenate([inside, edge, bg]), box).astype(np.float32)
    pos[pos >= np.float32(box)] = 0.0
    return pos, box, l_x, nc


def test_big_cell_sub_cell_path(cuda_lib):
    """A cell of 50,000 particles (above the shared-memory dense range) is
    linked by the big-cell kernels in sub-cell order: exact against the
    oracle, and in well under a second (no pair-by-pair O(m^2) work)."""
    import time
    torch = _torch()
    fof = cuda_lib
    pos, box, l_x, nc = _big_cell_box(31)
    n = pos.shape[0]
    opt = fof.fof_options()
    opt.cells_per_axis = nc
    opt.brick_cells = 2
    geo = fof.fof_box_geometry(box, l_x, n, opt)
    assert geo.cells_per_axis == nc and geo.sub_cells > 1
    dev = torch.from_numpy(pos).cuda()
    with fof.FoF(box, l_x, n, opt) as f:
        f.run(dev)                                    # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ids, sizes, cat, ng = f.run(dev, min_size=20)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
    wid, wsz = oracle.groups(pos, box, l_x)
    assert np.array_equal(ids.cpu().numpy(), wid)
    assert np.array_equal(sizes.cpu().numpy(), wsz)
    assert np.array_equal(cat.cpu().numpy(), oracle.catalogue(wsz, 20))
    assert dt < 1.0, dt


@pytest.mark.parametrize("n,width", [(20000, 2.6), (8000, 2.9)])
def test_box_without_splittable_cells(cuda_lib, n, width):
    """A box fewer than 3 linking lengths wide has at most 2 cells per axis
    and cannot be split into sub-cells: every pair is tested (O(n^2) work
    spread over the warps); exact and bounded in time."""
    import time
    torch = _torch()
    fof = cuda_lib
    l_x = 0.05
    box = width * l_x
    rng = np.random.default_rng(n)
    pos = (rng.random((n, 3)) * box).astype(np.float32)
    pos[pos >= np.float32(box)] = 0.0
    geo = fof.fof_box_geometry(box, l_x, n)
    assert geo.sub_cells == 1 and geo.cells_per_axis < 3
    dev = torch.from_numpy(pos).cuda()
    with fof.FoF(box, l_x, n) as f:
        f.run(dev)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ids, sizes, _, _ = f.run(dev)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
    wid, wsz = oracle.groups(pos, box, l_x)
    assert np.array_equal(ids.cpu().numpy(), wid)
    assert np.array_equal(sizes.cpu().numpy(), wsz)
    assert dt < 1.0, dt


def test_run_host_many_pipelined(cuda_lib):
    """fof_run_host_many: several host inputs of one plan, copies overlapped
    with compute on separate streams; every step's ids, sizes, catalogue and
    counts equal the oracle's for that step's input."""
    torch = _torch()
    fof = cuda_lib
    n, box = 120000, 20.0
    l_x = synth.linking_length(n, box)
    inputs = [synth.clustered_box(n, box, 40 + 10 * k, seed=950 + k) for k in range(4)]
    pos_h = [torch.from_numpy(p).pin_memory() for p in inputs]
    ids_h = [torch.empty(n, dtype=torch.int32).pin_memory() for _ in inputs]
    sizes_h = [torch.empty(n, dtype=torch.int32).pin_memory() for _ in inputs]
    cap = 5000
    cat_h = [torch.empty((cap, 2), dtype=torch.int32).pin_memory() for _ in inputs]
    stream = torch.cuda.Stream()
    h = fof.fof_create(box, l_x, n)
    try:
        for _ in range(2):                     # the second call re-uses the staging
            code, ng, nk = fof.fof_run_host_many(h, pos_h, ids_h, sizes_h, cat_h, cap, 10, 1, stream)
            assert code == 0
            for k, p in enumerate(inputs):
                wid, wsz = oracle.groups(p, box, l_x)
                wcat = oracle.catalogue(wsz, 10)
                assert np.array_equal(ids_h[k].numpy(), wid), k
                assert np.array_equal(sizes_h[k].numpy(), wsz), k
                assert nk[k][0] == wcat.shape[0] and ng[k][0] == int((wsz > 0).sum())
                assert np.array_equal(cat_h[k].numpy()[: nk[k][0]], wcat)
                ids_h[k].fill_(-1)
    finally:
        fof.fof_destroy(h)
