"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these checks re-uses the oracle's own formula: they compare it with
closed forms (exact ties, lattices, periodic chains), with the brute-force
all-pairs union-find of the paper's naive listing (Sec. 3.1), with an
independent connected-components routine, and with invariants that any
correct partition satisfies.
"""
import functools
import math

import numpy as np
import pytest

import oracle
from conftest import read_rows
from paper_2003_11468_gb300 import synth


# --------------------------------------------------------------------------
# the predicate
# --------------------------------------------------------------------------

def test_tie_pairs_golden():
    rows = read_rows("tie_pairs.txt")
    assert len(rows) >= 8
    for r in rows:
        box = float(r[0])
        a = np.array([float(v) for v in r[1:4]], dtype=np.float32)
        b = np.array([float(v) for v in r[4:7]], dtype=np.float32)
        l_x, want, exact = float(r[7]), int(r[8]), int(r[9])
        assert oracle.linked(a, b, box, l_x) == bool(want), r
        assert oracle.linked(b, a, box, l_x) == bool(want), r      # symmetric
        if exact:
            below = float(np.nextafter(l_x, 0.0))
            assert not oracle.linked(a, b, box, below), r
            above = float(np.nextafter(l_x, 1.0))
            assert oracle.linked(a, b, box, above), r


def test_each_axis_counts():
    """A dropped or mis-indexed axis would link points that differ on it."""
    box, l_x = 1.0, 0.0625
    base = np.array([0.5, 0.5, 0.5], dtype=np.float32)
    for ax in range(3):
        far = base.copy()
        far[ax] += np.float32(0.25)
        assert not oracle.linked(base, far, box, l_x)
        near = base.copy()
        near[ax] += np.float32(0.0625)
        assert oracle.linked(base, near, box, l_x)
    # the sum runs over all three squares: 3-4-12 gives 13
    s = np.float32(2.0 ** -8)
    a = np.array([0.25, 0.25, 0.25], dtype=np.float32)
    b = a + np.array([3 * s, 4 * s, 12 * s], dtype=np.float32)
    assert oracle.linked(a, b, 1.0, 13 * 2.0 ** -8)
    assert not oracle.linked(a, b, 1.0, float(np.nextafter(13 * 2.0 ** -8, 0)))
    assert not oracle.linked(a, b, 1.0, 12.99 * 2.0 ** -8)


# --------------------------------------------------------------------------
# closed forms
# --------------------------------------------------------------------------

def _lattice(k):
    m = 2 ** k
    g = (np.arange(m, dtype=np.float64) / m).astype(np.float32)
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)


def test_lattice_closed_form():
    for r in read_rows("lattice.txt"):
        k, n = int(r[0]), int(r[1])
        pos = _lattice(k)
        assert pos.shape[0] == n
        d = 2.0 ** -k
        ids, sizes = oracle.groups(pos, 1.0, d)
        assert (ids == 0).all() and sizes[0] == n and sizes[1:].sum() == 0
        ids, sizes = oracle.groups(pos, 1.0, float(np.nextafter(d, 0.0)))
        assert (ids == np.arange(n)).all() and (sizes == 1).all()


def test_lattice_brute_matches_closed_form():
    pos = _lattice(3)
    assert (oracle.brute(pos, 1.0, 0.125) == 0).all()
    assert (oracle.brute(pos, 1.0, float(np.nextafter(0.125, 0))) == np.arange(512)).all()


def test_periodic_chain_golden():
    for r in read_rows("chain_wrap.txt"):
        removed = [] if r[0] == "-" else [int(v) for v in r[0].split(",")]
        keep = [k for k in range(16) if k not in removed]
        pos = np.array([[k / 16.0, 0.5, 0.5] for k in keep], dtype=np.float32)
        want = np.array([int(v) for v in r[1:]], dtype=np.int32)
        ids, sizes = oracle.groups(pos, 1.0, 1.0 / 16.0)
        assert (ids == want).all(), (r, ids)
        assert (oracle.brute(pos, 1.0, 1.0 / 16.0) == want).all()
        labels, counts = np.unique(want, return_counts=True)
        assert (sizes[labels] == counts).all() and sizes.sum() == len(keep)


def test_degenerate_sizes():
    e = np.zeros((0, 3), dtype=np.float32)
    ids, sizes = oracle.groups(e, 1.0, 0.1)
    assert ids.size == 0 and sizes.size == 0
    one = np.array([[0.3, 0.2, 0.1]], dtype=np.float32)
    ids, sizes = oracle.groups(one, 1.0, 0.1)
    assert ids.tolist() == [0] and sizes.tolist() == [1]
    same = np.tile(np.array([[0.7, 0.7, 0.7]], dtype=np.float32), (50, 1))
    ids, sizes = oracle.groups(same, 1.0, 1e-6)
    assert (ids == 0).all() and sizes[0] == 50
    # x = 0 and x = L - ulp are neighbours through the wrap
    edge = np.array([[0.0, 0.5, 0.5], [0.5, 0.5, 0.5], [np.float32(1) - np.float32(2 ** -24), 0.5, 0.5]],
                    dtype=np.float32)
    ids, sizes = oracle.groups(edge, 1.0, 1e-6)
    assert ids.tolist() == [0, 1, 0] and sizes.tolist() == [2, 1, 0]


# --------------------------------------------------------------------------
# brute force and an independent connected-components routine
# --------------------------------------------------------------------------

@functools.lru_cache(maxsize=1)
def _cases():
    out = []
    for seed in range(6):
        n = [1, 2, 37, 300, 900, 2000][seed]
        box = [1.0, 3.0, 10.0, 100.0, 7.5, 64.0][seed]
        for b in (0.2, 0.5, 1.0):
            l_x = min(synth.linking_length(max(n, 1), box, b), 0.49 * box)
            out.append((synth.uniform_box(n, box, seed=100 + seed), box, l_x))
            out.append((synth.clustered_box(n, box, max(1, n // 100), seed=200 + seed), box, l_x))
    return out


@pytest.mark.parametrize("case", range(36))
def test_bfs_equals_brute_force(case):
    pos, box, l_x = _cases()[case]
    ids, sizes = oracle.groups(pos, box, l_x)
    assert (ids == oracle.brute(pos, box, l_x)).all()


def test_components_match_scipy_on_enumerated_edges():
    """Edges listed pair by pair, components by scipy's graph routine."""
    sp = pytest.importorskip("scipy.sparse")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    for pos, box, l_x in _cases()[::3]:
        n = pos.shape[0]
        if n < 2 or n > 400:
            continue
        rows, cols = [], []
        for i in range(n):
            for j in range(i + 1, n):
                if oracle.linked(pos[i], pos[j], box, l_x):
                    rows.append(i)
                    cols.append(j)
        g = sp.coo_matrix((np.ones(len(rows)), (rows, cols)), shape=(n, n))
        _, lab = csgraph.connected_components(g, directed=False)
        ids, _ = oracle.groups(pos, box, l_x)
        # same partition: first member of each scipy component is its minimum
        first = {}
        for i in range(n):
            first.setdefault(lab[i], i)
        assert all(ids[i] == first[lab[i]] for i in range(n))


# --------------------------------------------------------------------------
# invariants
# --------------------------------------------------------------------------

def _check_invariants(ids, sizes, n):
    idx = np.arange(n)
    assert (ids <= idx).all()
    assert (ids[ids] == ids).all()
    assert sizes.sum() == n
    labels, counts = np.unique(ids, return_counts=True)
    assert (sizes[labels] == counts).all()
    mask = np.zeros(n, bool)
    mask[labels] = True
    assert (sizes[~mask] == 0).all()


def test_invariants_clustered():
    pos = synth.clustered_box(20000, 20.0, 40, seed=9)
    l_x = synth.linking_length(20000, 20.0)
    ids, sizes = oracle.groups(pos, 20.0, l_x)
    _check_invariants(ids, sizes, 20000)
    # every sampled linked pair shares a label
    rng = np.random.default_rng(0)
    for i in rng.integers(0, 20000, 200):
        d = pos - pos[i]
        d = np.where(d > 10.0, d - 20.0, np.where(d < -10.0, d + 20.0, d))
        near = np.nonzero((d.astype(np.float64) ** 2).sum(1) <= 0.9 * l_x * l_x)[0]
        assert (ids[near] == ids[i]).all()


def test_permutation_invariance():
    n, box = 5000, 10.0
    pos = synth.clustered_box(n, box, 20, seed=11)
    l_x = synth.linking_length(n, box)
    ids, _ = oracle.groups(pos, box, l_x)
    perm = np.random.default_rng(1).permutation(n)
    ids_p, _ = oracle.groups(pos[perm], box, l_x)
    # ids_p labels positions in the permuted order: same partition
    a = ids[perm]
    b = ids_p
    pairs = set(zip(a.tolist(), b.tolist()))
    assert len(pairs) == len(set(a.tolist())) == len(set(b.tolist()))
    # the label is the minimum index of the group in its own order
    inv = np.empty(n, dtype=np.int64)
    inv[perm] = np.arange(n)
    for lab in np.unique(b)[:200]:
        members = np.nonzero(b == lab)[0]
        assert members.min() == lab


def test_translation_invariance_exact_shift():
    # coordinates on a 2^-16 grid in the unit box; shifts on the same grid
    # are exact in float32, so distances are unchanged
    rng = np.random.default_rng(3)
    n = 4000
    q = rng.integers(0, 2 ** 16, size=(n, 3))
    pos = (q / 2.0 ** 16).astype(np.float32)
    l_x = 0.2 / n ** (1 / 3) * 2
    ids, sizes = oracle.groups(pos, 1.0, l_x)
    for shift in ([0.5, 0.25, 0.125], [0.75, 0.0, 0.9375]):
        s = np.asarray(shift)
        pos2 = (((q / 2.0 ** 16) + s) % 1.0).astype(np.float32)
        ids2, sizes2 = oracle.groups(pos2, 1.0, l_x)
        assert (ids2 == ids).all() and (sizes2 == sizes).all()


def test_uniform_isolated_fraction():
    """Poisson statistics: P(no neighbour within l_x) = exp(-n 4/3 pi l_x^3)."""
    c = synth.uniform_32k()
    pos = c["make"]()
    ids, sizes = oracle.groups(pos, c["box"], c["l_x"])
    iso = (sizes[ids] == 1).mean()
    want = math.exp(-c["n"] * 4.0 / 3.0 * math.pi * c["l_x"] ** 3)
    assert abs(iso - want) < 0.005
    _check_invariants(ids, sizes, c["n"])


def test_component_matches_groups():
    n, box = 8000, 10.0
    pos = synth.clustered_box(n, box, 30, seed=13)
    l_x = synth.linking_length(n, box)
    ids, sizes = oracle.groups(pos, box, l_x)
    for i in [0, 1, 17, 4000, 7999]:
        lab, members = oracle.component(pos, box, l_x, i)
        assert lab == ids[i]
        assert (members == np.nonzero(ids == ids[i])[0]).all()
        assert sizes[lab] == members.size


def test_catalogue_filter():
    sizes = np.array([3, 0, 0, 1, 25, 0, 20, 19, 0], dtype=np.int32)
    cat = oracle.catalogue(sizes, 20)
    assert cat.tolist() == [[4, 25], [6, 20]]
    cat = oracle.catalogue(sizes, 0)
    assert cat[:, 0].tolist() == [0, 3, 4, 6, 7]
    assert oracle.catalogue(sizes, 26).shape == (0, 2)


# --------------------------------------------------------------------------
# the strict tie rule (distance < l_x, the naive listing of Sec. 3.1) and the
# array form of the predicate
# --------------------------------------------------------------------------

def test_strict_rule_on_tie_pairs():
    """At distance exactly l_x the strict rule does not link; just above the
    tie (the next double above l_x) it does, like the default rule."""
    for r in read_rows("tie_pairs.txt"):
        box = float(r[0])
        a = np.array([float(v) for v in r[1:4]], dtype=np.float32)
        b = np.array([float(v) for v in r[4:7]], dtype=np.float32)
        l_x, want, exact = float(r[7]), int(r[8]), int(r[9])
        if exact:
            assert not oracle.linked(a, b, box, l_x, strict=True), r
            assert oracle.linked(a, b, box, float(np.nextafter(l_x, 1.0)), strict=True), r
        elif not want:
            assert not oracle.linked(a, b, box, l_x, strict=True), r


def test_strict_rule_lattice_closed_form():
    """A lattice of spacing d: with l_x = d the strict rule leaves every point
    alone (each neighbour is exactly d away), the default rule joins all."""
    pos = _lattice(3)
    d = 2.0 ** -3
    ids, sizes = oracle.groups(pos, 1.0, d, strict=True)
    assert np.array_equal(ids, np.arange(pos.shape[0])) and (sizes == 1).all()
    ids, _ = oracle.groups(pos, 1.0, float(np.nextafter(d, 1.0)), strict=True)
    assert (ids == 0).all()


@pytest.mark.parametrize("seed", range(6))
def test_strict_rule_groups_equal_brute(seed):
    """Cell list + BFS under the strict rule equals the all-pairs loop."""
    rng = np.random.default_rng(500 + seed)
    n = int(rng.integers(50, 600))
    # points on a coarse grid so that many pairs sit exactly at l_x
    g = 2.0 ** -4
    pos = (rng.integers(0, 16, size=(n, 3)) * g).astype(np.float32)
    ids, _ = oracle.groups(pos, 1.0, g, strict=True)
    assert np.array_equal(ids, oracle.brute(pos, 1.0, g, strict=True))
    ids_le, _ = oracle.groups(pos, 1.0, g)
    assert np.array_equal(ids_le, oracle.brute(pos, 1.0, g))
    # on this grid the two rules differ: exact ties join only under <=
    assert not np.array_equal(ids, ids_le)


def test_linked_many_equals_linked_on_adversarial_pairs():
    """The array form of the predicate against the single-pair form, on pairs
    at exact ties, one float step inside and outside l_x, across the periodic
    wrap on every axis, and random pairs."""
    rng = np.random.default_rng(11)
    box, l_x = 1.0, 0.03125
    a = []
    b = []
    for r in read_rows("tie_pairs.txt"):
        if float(r[0]) == box and float(r[7]) == l_x:
            a.append([float(v) for v in r[1:4]])
            b.append([float(v) for v in r[4:7]])
    base = rng.random((400, 3)).astype(np.float32)
    dirs = rng.normal(size=(400, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    for scale in (1.0 - 2.0 ** -22, 1.0, 1.0 + 2.0 ** -22, 0.5, 2.0):
        far = np.mod(base + (dirs * l_x * scale), box).astype(np.float32)
        far[far >= np.float32(box)] = 0.0
        a.extend(base.tolist())
        b.extend(far.tolist())
    # wrap: points near 0 against points near the box side on one axis
    for ax in range(3):
        p = rng.random((50, 3)).astype(np.float32)
        q = p.copy()
        p[:, ax] = rng.random(50).astype(np.float32) * np.float32(l_x / 2)
        q[:, ax] = np.float32(box) - rng.random(50).astype(np.float32) * np.float32(l_x / 2)
        q[q >= np.float32(box)] = 0.0
        a.extend(p.tolist())
        b.extend(q.tolist())
    A = np.array(a, dtype=np.float32)
    B = np.array(b, dtype=np.float32)
    many = oracle.linked_many(A, B, box, l_x)
    single = np.array([oracle.linked(A[k], B[k], box, l_x) for k in range(A.shape[0])])
    assert np.array_equal(many, single)
    assert many.any() and not many.all()
