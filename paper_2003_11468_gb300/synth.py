"""Seeded synthetic particle sets for the Friends-of-Friends workloads.

This module only draws positions.  It holds none of the group finder's
arithmetic (no distances, no cells, no linking), so both the CUDA path and
the CPU oracle can take their inputs from it without sharing method code.

Workloads stand in for the EAGLE z=0.1 snapshot the paper measures on
(Sec. 4.1: 4.25e8 particles, about 2e5 groups of more than 20 members), which
is not available here:

* ``uniform_box``: positions uniform in the periodic cube [0, L)^3.
* ``clustered_box``: a fraction f of the particles sits in K Plummer blobs,
  the rest is uniform.  Blob masses follow dN/dM ~ M^-1.9 on [1, 1e4]
  (inverse-CDF draw), are scaled to integer member counts that sum exactly
  to round(f n) (largest remainder), each blob has a Plummer scale radius
  a_k = 0.05 s m_k^(1/3) with s = L / n^(1/3) the mean separation (central
  overdensity about 1.9e3 for every blob), radii r = a / sqrt(u^(-2/3) - 1)
  redrawn when r > 10 a, isotropic directions, and periodic wrapping.

Positions are drawn in float64, wrapped into [0, L), cast to float32, and a
float32 value equal to L (possible only through the cast) is replaced by 0,
which is the same point of the periodic box.

Particle order is the generation order: blob members come blob by blob
(in random order inside each blob), followed by the uniform background in
random spatial order.

Large sets are drawn in fixed-size chunks, each chunk from its own child of
the seed's ``SeedSequence``, on a thread pool.  The chunking does not depend
on the thread count, so a seed always gives the same array.

Machine independence: every value is computed with IEEE-754 basic
operations only (+, -, *, /, sqrt, floor, ldexp/frexp), which numpy rounds
the same way on every CPU.  The logarithms, exponentials and cube roots the
recipe needs are evaluated by the short series below instead of the C
library or numpy's vectorised transcendental functions, whose last-bit
rounding differs between machines (x86-64 with AVX-512 and aarch64 give
different bits); isotropic directions come from Marsaglia's (1972)
rejection method instead of sin/cos.  Sums of many terms use math.fsum
(correctly rounded).  So a seed gives the same float32 array everywhere,
which lets stored hashes of oracle outputs be checked on another machine.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

CHUNK = 1 << 21          # particles per independently seeded chunk
MASS_SLOPE = -1.9        # dN/dM ~ M^MASS_SLOPE
MASS_RANGE = (1.0, 1.0e4)
PLUMMER_A0 = 0.05        # a_k = PLUMMER_A0 * s * m_k^(1/3)
PLUMMER_RMAX = 10.0      # radii beyond PLUMMER_RMAX * a are redrawn


# --------------------------------------------------------------------------
# machine-independent elementary functions (float64, basic operations only)
# --------------------------------------------------------------------------

_LN2_HI = 6.93147180369123816490e-01   # high part of ln 2 (trailing zero bits)
_LN2_LO = 1.90821492927058770002e-10   # ln 2 - _LN2_HI
_INV_LN2 = 1.44269504088896338700e+00
_SQRT_HALF = 0.70710678118654752440
# Taylor coefficients 1/k! (k = 0..14) of exp on |r| <= ln2/2
_EXP_C = [1.0 / math.factorial(k) for k in range(15)]
# atanh series coefficients 1/(2k+1) (k = 0..14) for log(m) = 2 atanh(s)
_LOG_C = [1.0 / (2 * k + 1) for k in range(15)]


def det_exp(y):
    """exp(y) for float64 arrays (relative error ~1e-15), the same bits on every machine.

    Argument reduction y = k ln2 + r with |r| <= ln2/2 (ln2 split in two
    parts), a degree-14 Taylor polynomial for exp(r) in Horner form, and an
    exact scaling by 2^k."""
    y = np.asarray(y, dtype=np.float64)
    k = np.floor(y * _INV_LN2 + 0.5)
    r = (y - k * _LN2_HI) - k * _LN2_LO
    p = np.full_like(r, _EXP_C[-1])
    for c in reversed(_EXP_C[:-1]):
        p = p * r + c
    return np.ldexp(p, k.astype(np.int64))


def det_log(x):
    """Natural logarithm of positive float64 arrays, the same bits on every machine.

    x = m 2^e with m in [sqrt(1/2), sqrt(2)) (exact), log m = 2 atanh(s) with
    s = (m - 1) / (m + 1), |s| < 0.172, summed as an odd series to s^29."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)
    low = m < _SQRT_HALF
    m = np.where(low, m * 2.0, m)
    e = (e - low.astype(np.int64)).astype(np.float64)
    s = (m - 1.0) / (m + 1.0)
    z = s * s
    p = np.full_like(z, _LOG_C[-1])
    for c in reversed(_LOG_C[:-1]):
        p = p * z + c
    return e * _LN2_HI + (e * _LN2_LO + 2.0 * s * p)


def det_pow(x, a: float):
    """x^a for positive float64 arrays (exp(a log x)), machine independent."""
    return det_exp(a * det_log(x))


def det_cbrt(x):
    """Cube root of non-negative float64 arrays (0 -> 0), machine independent."""
    x = np.asarray(x, dtype=np.float64)
    out = det_pow(np.where(x > 0.0, x, 1.0), 1.0 / 3.0)
    return np.where(x > 0.0, out, 0.0)


def _scalar(f, v: float) -> float:
    return float(f(np.array([v], dtype=np.float64))[0])


def _iso_directions(rng: np.random.Generator, m: int) -> np.ndarray:
    """m isotropic unit vectors by Marsaglia's (1972) method: (u, v) uniform
    in the unit disc (rejection from the square), then
    (2u sqrt(1-t), 2v sqrt(1-t), 1 - 2t) with t = u^2 + v^2."""
    u = np.empty(m)
    v = np.empty(m)
    todo = np.arange(m)
    while todo.size:
        a = 2.0 * rng.random(todo.size) - 1.0
        b = 2.0 * rng.random(todo.size) - 1.0
        t = a * a + b * b
        ok = t < 1.0
        u[todo[ok]] = a[ok]
        v[todo[ok]] = b[ok]
        todo = todo[~ok]
    t = u * u + v * v
    w = np.sqrt(1.0 - t)
    d = np.empty((m, 3))
    d[:, 0] = 2.0 * u * w
    d[:, 1] = 2.0 * v * w
    d[:, 2] = 1.0 - 2.0 * t
    return d


def _threads() -> int:
    return max(1, min(32, os.cpu_count() or 1))


def _finish(x: np.ndarray, box: float) -> np.ndarray:
    """float64 -> wrapped float32 in [0, box)."""
    x = np.mod(x, box)
    out = x.astype(np.float32)
    out[out >= np.float32(box)] = np.float32(0.0)
    return out


def _uniform_chunk(seed_seq, m: int, box: float) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed_seq))
    return _finish(rng.random((m, 3)) * box, box)


def uniform_box(n: int, box: float, seed: int) -> np.ndarray:
    """n positions uniform in [0, box)^3, float32, shape (n, 3)."""
    out = np.empty((n, 3), dtype=np.float32)
    _fill_uniform(out, box, np.random.SeedSequence(seed))
    return out


def _fill_uniform(out: np.ndarray, box: float, ss: np.random.SeedSequence) -> None:
    n = out.shape[0]
    nch = (n + CHUNK - 1) // CHUNK
    kids = ss.spawn(nch) if nch else []

    def work(c):
        lo = c * CHUNK
        hi = min(n, lo + CHUNK)
        out[lo:hi] = _uniform_chunk(kids[c], hi - lo, box)

    if nch <= 1:
        for c in range(nch):
            work(c)
    else:
        with ThreadPoolExecutor(_threads()) as ex:
            list(ex.map(work, range(nch)))


def blob_counts(n_clustered: int, n_blobs: int, rng: np.random.Generator) -> np.ndarray:
    """Integer member counts of the blobs, power-law masses, exact total."""
    if n_blobs <= 0 or n_clustered <= 0:
        return np.zeros(max(n_blobs, 0), dtype=np.int64)
    g = 1.0 + MASS_SLOPE                      # exponent of the CDF
    lo, hi = _scalar(lambda a: det_pow(a, g), MASS_RANGE[0]), _scalar(lambda a: det_pow(a, g), MASS_RANGE[1])
    u = rng.random(n_blobs)
    mass = det_pow(lo + u * (hi - lo), 1.0 / g)
    share = mass * (n_clustered / math.fsum(mass.tolist()))
    counts = np.floor(share).astype(np.int64)
    rest = int(n_clustered - counts.sum())
    if rest > 0:
        order = np.argsort(-(share - counts), kind="stable")
        counts[order[:rest]] += 1
    return counts


def _blob_chunk(seed_seq, centres, counts, radii, box: float) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed_seq))
    m = int(counts.sum())
    a = np.repeat(radii, counts)
    c = np.repeat(centres, counts, axis=0)
    r = np.empty(m)
    todo = np.arange(m)
    while todo.size:
        u = 1.0 - rng.random(todo.size)          # (0, 1]
        with np.errstate(divide="ignore", invalid="ignore"):
            rr = a[todo] / np.sqrt(det_pow(u, -2.0 / 3.0) - 1.0)
        ok = rr <= PLUMMER_RMAX * a[todo]
        r[todo[ok]] = rr[ok]
        todo = todo[~ok]
    d = _iso_directions(rng, m)
    x = c + r[:, None] * d
    return _finish(x, box)


def clustered_box(n: int, box: float, n_blobs: int, seed: int,
                  frac: float = 0.5) -> np.ndarray:
    """Plummer-blob mixture: round(frac*n) particles in n_blobs blobs, rest uniform."""
    ss = np.random.SeedSequence(seed)
    ss_blob, ss_uni, ss_par = ss.spawn(3)
    par = np.random.Generator(np.random.PCG64(ss_par))
    n_cl = int(round(frac * n)) if n_blobs > 0 else 0
    counts = blob_counts(n_cl, n_blobs, par)
    centres = par.random((max(n_blobs, 0), 3)) * box
    s = box / _scalar(det_cbrt, float(n)) if n > 0 else 0.0
    radii = PLUMMER_A0 * s * det_cbrt(counts.astype(np.float64))

    out = np.empty((n, 3), dtype=np.float32)
    # chunks of whole blobs, about CHUNK particles each
    starts = np.concatenate([[0], np.cumsum(counts)])
    bounds = [0]
    acc = 0
    for k in range(len(counts)):
        acc += counts[k]
        if acc >= CHUNK:
            bounds.append(k + 1)
            acc = 0
    if bounds[-1] != len(counts):
        bounds.append(len(counts))
    kids = ss_blob.spawn(max(1, len(bounds) - 1))

    def work(c):
        b0, b1 = bounds[c], bounds[c + 1]
        lo, hi = int(starts[b0]), int(starts[b1])
        if hi > lo:
            out[lo:hi] = _blob_chunk(kids[c], centres[b0:b1], counts[b0:b1],
                                     radii[b0:b1], box)

    nch = len(bounds) - 1
    if nch <= 1:
        for c in range(nch):
            work(c)
    else:
        with ThreadPoolExecutor(_threads()) as ex:
            list(ex.map(work, range(nch)))
    _fill_uniform(out[n_cl:], box, ss_uni)
    return out


def linking_length(n: int, box: float, b: float = 0.2) -> float:
    """l_x = b times the mean inter-particle separation L / n^(1/3), in float64."""
    return b * box / _scalar(det_cbrt, float(n))


# --------------------------------------------------------------------------
# Named workloads: dict(name, n, box, l_x, min_size, seed, make(seed=...)).
# --------------------------------------------------------------------------

def uniform_32k():
    """32^3 particles uniform in the unit box, l_x = 0.2/32, min size 2."""
    n, box = 32 ** 3, 1.0
    return dict(name="fof-32^3-uniform", n=n, box=box,
                l_x=0.2 * box / 32, min_size=2, seed=1,
                make=lambda seed=1: uniform_box(n, box, seed=seed))


def clustered_256():
    """256^3 particles, box 100, 20,000 blobs, l_x = 0.2*100/256, min size 20."""
    n, box = 256 ** 3, 100.0
    return dict(name="fof-256^3-clustered", n=n, box=box,
                l_x=0.2 * box / 256, min_size=20, seed=2,
                make=lambda seed=2: clustered_box(n, box, 20000, seed=seed))


def clustered_1024():
    """1024^3 particles, box 100, 500,000 blobs, l_x = 0.2*100/1024, min size 20."""
    n, box = 1024 ** 3, 100.0
    return dict(name="fof-1024^3-clustered", n=n, box=box,
                l_x=0.2 * box / 1024, min_size=20, seed=3,
                make=lambda seed=3: clustered_box(n, box, 500000, seed=seed))


def clustered_sample_of_1024(k: int = 4):
    """A periodic 1/k^3-volume box with the 1024^3 recipe's density and l_x.

    n = (1024/k)^3, L = 100/k, 500000/k^3 blobs (rounded), same l_x as the
    1024^3 box.  Used to time the CPU oracle on a bounded sample.
    """
    side = 1024 // k
    n, box = side ** 3, 100.0 / k
    blobs = max(1, int(round(500000 / k ** 3)))
    return dict(name=f"fof-{side}^3-clustered-sample", n=n, box=box,
                l_x=0.2 * 100.0 / 1024, min_size=20, seed=3000 + k,
                make=lambda seed=3000 + k: clustered_box(n, box, blobs, seed=seed))


def batch_512(count: int = 512, seed0: int = 4000):
    """Independent boxes: n log-uniform on [16^3, 160^3], L uniform on [50, 150].

    Each box b draws (n_b, L_b) from seed seed0 + b; K_b = max(1, round(20000
    n_b / 256^3)) blobs, 50% clustered, l_x = 0.2 L_b / n_b^(1/3), min size 20.
    """
    boxes = []
    for b in range(count):
        rng = np.random.Generator(np.random.PCG64(seed0 + b))
        lo, hi = _scalar(det_log, 16.0 ** 3), _scalar(det_log, 160.0 ** 3)
        n = int(round(_scalar(det_exp, lo + (hi - lo) * rng.random())))
        box = 50.0 + 100.0 * rng.random()
        k = max(1, int(round(20000 * n / 256 ** 3)))
        boxes.append(dict(n=n, box=box, l_x=linking_length(n, box), min_size=20,
                          blobs=k, seed=seed0 + b))
    return boxes


def make_batch_box(spec) -> np.ndarray:
    return clustered_box(spec["n"], spec["box"], spec["blobs"], seed=spec["seed"] + 10 ** 6)


def served_box_side(n: int) -> float:
    """Box side of a served request of n particles at the 256^3 workload's density."""
    return 100.0 * _scalar(det_cbrt, n / 256 ** 3)


def served_pool(count: int = 24, n_lo: float = 1e4, n_hi: float = 1e8):
    """Distinct request inputs reused by the served workload (bounded generation).

    Sizes log-spaced on [n_lo, n_hi] (duplicates after rounding dropped), each
    a clustered box at the 256^3 density: L = served_box_side(n), K = max(1,
    round(20000 n / 256^3)) blobs, l_x = 0.2 L / n^(1/3), min size 20; pool
    entry k is drawn from seed 5,000,000 + k.  A request takes the entry of
    nearest log-size."""
    llo, lhi = _scalar(det_log, n_lo), _scalar(det_log, n_hi)
    sizes = []
    for k in range(count):
        v = llo + (lhi - llo) * (k / (count - 1) if count > 1 else 0.0)
        n = int(_scalar(det_exp, v) + 0.5)
        if n not in sizes:
            sizes.append(n)
    pool = []
    for k, n in enumerate(sorted(sizes)):
        box = served_box_side(n)
        pool.append(dict(k=k, n=n, box=box, l_x=linking_length(n, box), min_size=20,
                         blobs=max(1, int(round(20000 * n / 256 ** 3))), seed=5_000_000 + k))
    return pool


def make_served(spec) -> np.ndarray:
    return clustered_box(spec["n"], spec["box"], spec["blobs"], seed=spec["seed"])


def served_requests(count: int = 2000, rate: float = 200.0, seed: int = 5,
                    n_lo: float = 1e4, n_hi: float = 1e8):
    """Poisson arrivals (mean `rate` per second), sizes log-uniform in [n_lo, n_hi].

    Each request k has a clustered box with the 256^3 workload's density:
    L = 100 (n / 256^3)^(1/3), K = max(1, round(20000 n / 256^3)), min size 20.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = -det_log(1.0 - rng.random(count)) / rate      # exponential, mean 1/rate
    t = np.cumsum(gaps)
    llo, lhi = _scalar(det_log, n_lo), _scalar(det_log, n_hi)
    ln = llo + (lhi - llo) * rng.random(count)
    reqs = []
    for k in range(count):
        n = int(round(_scalar(det_exp, float(ln[k]))))
        box = served_box_side(n)
        reqs.append(dict(k=k, t_arrive=float(t[k]), n=n, box=box,
                         l_x=linking_length(n, box), min_size=20,
                         blobs=max(1, int(round(20000 * n / 256 ** 3))),
                         seed=5_000_000 + k))
    return reqs
