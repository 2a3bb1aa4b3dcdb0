"""Host-side geometry of the CUDA path, checked by float32 emulation.

The kernels index cells in float32: fine = min(nf-1, (int)(x * inv_fine)),
cell = fine // q, and pre-test pairs with a float32 squared distance against
[t_lo, t_hi].  The library derives these constants with proven margins
(fof_box_geometry).  Here numpy's IEEE float32 arithmetic replays the
kernels' index and pre-test formulas on adversarial pairs and the oracle's
exact predicate decides which pairs are linked.  No GPU is needed.
"""
import numpy as np
import pytest

import oracle
from paper_2003_11468_gb300 import fof, synth

f32 = np.float32

CASES = [
    (1.0, 0.2 / 32, 32 ** 3),
    (100.0, 0.2 * 100 / 256, 256 ** 3),
    (100.0, 0.2 * 100 / 1024, 1024 ** 3),
    (3.0, 0.0371, 5000),
    (77.7, 0.9, 100000),
    (12.5, 0.2 * 100 / 1024, 128 ** 3),
    (1.0, 0.3, 1000),            # 3 cells per axis
]


def _fine(x, gm):
    g = (x.astype(f32) * f32(gm.inv_fine)).astype(np.int64)
    return np.clip(g, 0, gm.fine_per_axis - 1)


def _pairs(rng, box, l_x, m, lo, hi):
    a = (rng.random((m, 3)) * box).astype(f32)
    d = rng.normal(size=(m, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = l_x * rng.uniform(lo, hi, size=m)
    b = np.mod(a.astype(np.float64) + d * r[:, None], box).astype(f32)
    b[b >= f32(box)] = 0
    return a, b


def _pairs_on_cell_edges(rng, box, gm, l_x, m):
    """a on fine-cell boundaries (as float32 sees them), b near l_x away."""
    nf = gm.fine_per_axis
    k = rng.integers(0, nf, size=(m, 3))
    a = (k.astype(np.float64) * (box / nf)).astype(f32)
    a[a >= f32(box)] = 0
    d = rng.normal(size=(m, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = l_x * rng.uniform(0.99, 1.0, size=m)
    b = np.mod(a.astype(np.float64) + d * r[:, None], box).astype(f32)
    b[b >= f32(box)] = 0
    return a, b


def _pdist(ga, gb, n):
    d = np.abs(ga - gb)
    return np.minimum(d, n - d)


@pytest.mark.parametrize("case", range(len(CASES)))
def test_linked_pairs_stay_in_the_stencil(case):
    box, l_x, n = CASES[case]
    gm = fof.fof_box_geometry(box, l_x, n)
    assert box / gm.cells_per_axis >= l_x
    rng = np.random.default_rng(case)
    a1, b1 = _pairs(rng, box, l_x, 200000, 0.95, 1.0005)
    a2, b2 = _pairs_on_cell_edges(rng, box, gm, l_x, 200000)
    a, b = np.concatenate([a1, a2]), np.concatenate([b1, b2])
    link = oracle.linked_many(a, b, box, l_x)
    assert link.sum() > 1000
    ga, gb = _fine(a[link], gm), _fine(b[link], gm)
    q = gm.sub_cells
    if q > 1:
        assert _pdist(ga, gb, gm.fine_per_axis).max() <= 2
    assert _pdist(ga // q, gb // q, gm.cells_per_axis).max() <= 1


@pytest.mark.parametrize("case", range(len(CASES)))
def test_fine_cells_are_cliques(case):
    box, l_x, n = CASES[case]
    gm = fof.fof_box_geometry(box, l_x, n)
    if gm.sub_cells == 1:
        # larger cells at a higher occupancy are split
        opt = fof.fof_options()
        opt.occupancy = 4.0
        gm = fof.fof_box_geometry(box, l_x, n, opt)
    if gm.sub_cells == 1:
        pytest.skip("cells are not split for this box")
    rng = np.random.default_rng(100 + case)
    hf = box / gm.fine_per_axis
    m = 300000
    k = rng.integers(0, gm.fine_per_axis, size=(m, 3)).astype(np.float64)
    # corners of the fine cell and random points, stretched slightly beyond it
    ua = rng.choice([0.0, 1e-7, 0.5, 1 - 1e-6, 1.0], size=(m, 3))
    ub = np.where(rng.random((m, 3)) < 0.5, 1.0 - ua, rng.random((m, 3)))
    a = ((k + ua) * hf).astype(f32)
    b = ((k + ub) * hf).astype(f32)
    a[a >= f32(box)] = 0
    b[b >= f32(box)] = 0
    same = (_fine(a, gm) == _fine(b, gm)).all(axis=1)
    assert same.sum() > 5000
    assert oracle.linked_many(a[same], b[same], box, l_x).all()


def _d2_f32(a, b, box):
    Lf = f32(box)
    d = np.abs(a - b)                       # float32 subtraction, rounded
    m = np.minimum(d, Lf - d)
    mx, my, mz = m[:, 0], m[:, 1], m[:, 2]
    xx = mx * mx
    t = (my.astype(np.float64) * my + xx).astype(f32)     # fma, one rounding
    return (mz.astype(np.float64) * mz + t).astype(f32)


@pytest.mark.parametrize("case", range(len(CASES)))
def test_float32_pretest_never_contradicts_exact(case):
    box, l_x, n = CASES[case]
    gm = fof.fof_box_geometry(box, l_x, n)
    assert gm.t_lo <= l_x * l_x <= gm.t_hi
    rng = np.random.default_rng(200 + case)
    a1, b1 = _pairs(rng, box, l_x, 300000, 0.99, 1.01)
    a2, b2 = _pairs(rng, box, l_x, 100000, 0.0, 3.0)
    a, b = np.concatenate([a1, a2]), np.concatenate([b1, b2])
    link = oracle.linked_many(a, b, box, l_x)
    sf = _d2_f32(a, b, box)
    assert not link[sf > f32(gm.t_hi)].any()
    assert link[sf < f32(gm.t_lo)].all()
    # the uncertainty band is narrow: few pairs spread over [0, 3 l_x] fall in it
    wide = sf[a1.shape[0]:]
    band = (wide >= f32(gm.t_lo)) & (wide <= f32(gm.t_hi))
    assert band.mean() < 0.01


@pytest.mark.parametrize("case", range(len(CASES)))
def test_bounding_box_gap_keeps_every_partner(case):
    """The team filter drops a candidate when its float32 gap to the box of
    the team's particles exceeds bb_reach2; replay it with one-particle boxes
    (the tightest case) and periodic shifts by float32(L)."""
    box, l_x, n = CASES[case]
    gm = fof.fof_box_geometry(box, l_x, n)
    rng = np.random.default_rng(300 + case)
    a, b = _pairs(rng, box, l_x, 300000, 0.98, 1.0001)
    # put a near the low faces so the partner often sits across the wrap
    a = (a.astype(np.float64) * 0.01).astype(f32)
    d = rng.normal(size=a.shape)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    b = np.mod(a.astype(np.float64) + d * (l_x * rng.uniform(0.98, 1.0001, size=(a.shape[0], 1))), box)
    b = b.astype(f32)
    b[b >= f32(box)] = 0
    link = oracle.linked_many(a, b, box, l_x)
    a, b = a[link], b[link]
    Lf = f32(box)
    # the shift that brings b next to a (as the kernel's cell offsets do)
    shift = np.where(b - a > Lf / 2, -Lf, np.where(a - b > Lf / 2, Lf, f32(0))).astype(f32)
    x = (b + shift).astype(f32)
    gap = np.abs(x - a).astype(f32)
    g2 = (gap[:, 0] * gap[:, 0] + gap[:, 1] * gap[:, 1] + gap[:, 2] * gap[:, 2]).astype(f32)
    assert link.sum() > 1000
    assert (g2 <= f32(gm.bb_reach2)).all()


def test_valid_coordinate_limit():
    for box, l_x, n in CASES:
        gm = fof.fof_box_geometry(box, l_x, n)
        assert float(gm.xmax) < box
        assert float(np.nextafter(f32(gm.xmax), f32(np.inf))) >= box
