"""Autotuner for the plan options of one box or a batch of boxes.

The options choose the search structure only: the cell occupancy (which sets
cells per axis, hence the cell side, never below l_x), the size from which a
cell is split into sub-cells and linked by a thread block (dense_min), and the
size from which a cell's particles are linked by a warp team (team_min).  Cells
are a search structure for the pairs within l_x (Sec. 3.1 matches them to the
linking length); every choice yields the same partition, so the tuner may pick
by speed alone.

`tune` times each candidate on the caller's own input with CUDA events (link +
groups on one stream, after one untimed run), checks that every candidate gave
identical ids and sizes, and returns the fastest.  Results are cached by the
problem's shape (particle count per box, linking length in units of the mean
separation, box count) in a JSON file: the path given, else the environment
variable FOF_TUNE_CACHE, else no cache.
"""
from __future__ import annotations

import itertools
import json
import math
import os
import tempfile

from . import fof

# candidate values; every combination is timed
DEFAULT_GRID = {
    "occupancy": (0.25, 0.35, 0.5),
    "dense_min": (192, 256, 384),
    "team_min": (4, 8, 10),
}


def candidates(grid: dict | None = None) -> list[dict]:
    g = DEFAULT_GRID if grid is None else grid
    keys = sorted(g)
    return [dict(zip(keys, vals)) for vals in itertools.product(*(g[k] for k in keys))]


def options_from(d: dict | None) -> fof.fof_options | None:
    """fof_options with the given fields set (unset fields keep the library default)."""
    if d is None:
        return None
    o = fof.fof_options()
    if "occupancy" in d:
        o.occupancy = float(d["occupancy"])
    if "dense_min" in d:
        o.dense_min = int(d["dense_min"])
    if "team_min" in d:
        o.team_min = int(d["team_min"])
    if "brick_cells" in d:
        o.brick_cells = int(d["brick_cells"])
    return o


def shape_key(boxes, lxs, ns) -> str:
    """Cache key: box count, log2 of the mean particles per box, and l_x in
    units of the mean interparticle separation (both rounded)."""
    nb = len(ns)
    tot = max(1, int(sum(ns)))
    mean_n = tot / max(nb, 1)
    # particle-weighted mean of l_x / (L / n^(1/3))
    b = sum(l / (L / max(n, 1) ** (1.0 / 3.0)) * n for L, l, n in zip(boxes, lxs, ns)) / tot
    return f"boxes{nb}_n2^{round(math.log2(max(mean_n, 1)))}_b{b:.2f}"


class TuneCache:
    """JSON file {shape key: option dict}; written atomically."""

    def __init__(self, path: str | None = None):
        self.path = path if path is not None else os.environ.get("FOF_TUNE_CACHE")
        self.data = {}
        if self.path and os.path.exists(self.path):
            with open(self.path) as f:
                self.data = json.load(f)

    def get(self, key: str) -> dict | None:
        return self.data.get(key)

    def put(self, key: str, value: dict) -> None:
        self.data[key] = value
        if not self.path:
            return
        d = os.path.dirname(os.path.abspath(self.path))
        os.makedirs(d, exist_ok=True)
        fd, tmp = tempfile.mkstemp(dir=d, prefix=".tune.")
        with os.fdopen(fd, "w") as f:
            json.dump(self.data, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


def _time_candidate(boxes, lxs, ns, pos, opt, repeats, min_size, stream, out):
    import torch
    ids, sizes = out
    if len(ns) == 1:
        h = fof.fof_create_ex(boxes[0], lxs[0], ns[0], opt)
    else:
        h = fof.fof_batch_create(boxes, lxs, ns, opt)
    try:
        fof.fof_link(h, pos, stream)
        fof.fof_groups(h, ids, sizes, None, 0, min_size, len(ns), stream)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(repeats):
            fof.fof_link(h, pos, stream)
            fof.fof_groups_async(h, ids, sizes, None, 0, min_size, stream)
        e1.record(stream)
        e1.synchronize()
        code, _, _ = fof.fof_result(h, len(ns), stream)
        if code != 0:
            raise fof.FoFError(code, "tune")
        return e0.elapsed_time(e1) / repeats
    finally:
        fof.fof_destroy(h)


def tune(boxes, lxs, ns, pos, grid: dict | None = None, repeats: int = 2, min_size: int = 20,
         cache: TuneCache | str | None = None, stream=None, retune: bool = False):
    """Pick plan options for these boxes by timing the candidates on `pos`.

    boxes, lxs, ns: per-box side, linking length and particle count (one box
    or a batch, as for fof_create / fof_batch_create).  pos: the device
    positions (concatenated for a batch).  Returns (fof_options, report) where
    report = {"key", "best", "ms": {candidate: ms}, "cached"}.  Raises
    RuntimeError if two candidates disagree (they compute one partition).
    """
    import torch
    boxes, lxs, ns = [float(x) for x in boxes], [float(x) for x in lxs], [int(x) for x in ns]
    if not isinstance(cache, TuneCache):
        cache = TuneCache(cache)
    key = shape_key(boxes, lxs, ns)
    hit = None if retune else cache.get(key)
    if hit is not None:
        return options_from(hit), {"key": key, "best": hit, "ms": {}, "cached": True}
    total = int(sum(ns))
    dev = pos.device
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    ids = torch.empty(max(total, 1), dtype=torch.int32, device=dev)
    sizes = torch.empty_like(ids)
    ref = None
    times = {}
    best, best_ms = None, float("inf")
    for cand in candidates(grid):
        ms = _time_candidate(boxes, lxs, ns, pos, options_from(cand), repeats, min_size, s, (ids, sizes))
        s.synchronize()
        if ref is None:
            ref = (ids.clone(), sizes.clone())
        elif not (torch.equal(ref[0], ids) and torch.equal(ref[1], sizes)):
            raise RuntimeError(f"tune: candidate {cand} changed the partition")
        times[json.dumps(cand, sort_keys=True)] = ms
        if ms < best_ms:
            best, best_ms = cand, ms
    cache.put(key, best)
    return options_from(best), {"key": key, "best": best, "ms": times, "cached": False}
