"""Groups of one periodic box spread over several GPUs (paper Sec. 3.3).

The box is cut into slabs along x, one per rank (one process per GPU).  Each
rank holds the particles of its slab and runs the four steps of the paper's
distributed Union-Find (Sec. 3.3, Fig. "Distributed Union-Find"):

1. local groups: the ghost particles within l_x of the slab (sent by the
   ranks that own them) are appended to the rank's own particles and the
   GPU group finder runs on the union, in the same periodic box;
2. globally unique ids: particle ids are offset by an exclusive scan of the
   ranks' particle counts (the paper's MPI_Scan); a local group is named by
   the smallest global id among its members;
3. links: for every ghost and every own particle that is a ghost elsewhere,
   the pair (its local group's id, its global id) -- only groups that reach
   within l_x of a slab boundary take part;
4. merge: the link lists of all ranks are all-gathered (all-gather of
   variable-length lists) and every rank runs the union-find over the whole
   list (fof_merge_links, union by size, smallest id kept), which follows
   indirect links through third ranks; each rank then relabels its own
   particles.  Group sizes of spanning groups are summed over the ranks.

Every true edge of the particle graph is seen by the rank that owns one of
its ends (the other end is its own particle or a ghost), so the merged
components are exactly the groups of the whole box, labelled by their
smallest global particle id.

Communication uses torch.distributed (NCCL between GPUs, gloo on CPU);
remote particles are copied into the receiving rank's memory, never read in
place.  The merge itself is host code in the library (fof_merge_links).
"""
from __future__ import annotations

import numpy as np

from . import fof

# Ghost band: particles whose periodic x-distance to a slab is at most
# l_x * (1 + GHOST_MARGIN) are sent to it.  Any superset of the particles
# within l_x is correct (extra ghosts only add true edges); the margin
# covers the float32 coordinates and the double slab bounds many times over.
GHOST_MARGIN = 1e-3


def slab_bounds(box: float, world: int, rank: int):
    """[lo, hi) in x of rank's slab."""
    return box * rank / world, box * (rank + 1) / world


def slab_of(x, box: float, world: int):
    """Slab (rank) of each x coordinate."""
    r = np.floor(np.asarray(x, dtype=np.float64) * world / box).astype(np.int64)
    return np.clip(r, 0, world - 1)


def _periodic_gap(x, lo: float, hi: float, box: float):
    """Periodic distance in x from each coordinate to the interval [lo, hi)."""
    x = np.asarray(x, dtype=np.float64)
    inside = (x >= lo) & (x < hi)
    d_lo = np.mod(lo - x, box)          # distance going up to lo
    d_hi = np.mod(x - hi, box)          # distance going down to hi
    gap = np.minimum(d_lo, d_hi)
    return np.where(inside, 0.0, gap)


def _gpu_local(pos, box, l_x):
    """Step 1 on this rank's GPU: min-local-index labels of own + ghosts."""
    import torch
    n = pos.shape[0]
    if n == 0:
        return np.zeros(0, dtype=np.int32)
    with fof.FoF(box, l_x, n) as f:
        ids, _, _, _ = f.run(torch.from_numpy(np.ascontiguousarray(pos)).cuda())
        return ids.cpu().numpy()


def _allgather_var(arr: np.ndarray, group=None, device=None):
    """All-gather of variable-length 1-D int64/float arrays (an all-gatherv)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    t = torch.from_numpy(np.ascontiguousarray(arr))
    if device is not None:
        t = t.to(device)
    n = torch.tensor([t.numel()], dtype=torch.int64, device=t.device)
    ns = [torch.zeros_like(n) for _ in range(world)]
    dist.all_gather(ns, n, group=group)
    ns = [int(v.item()) for v in ns]
    m = max(ns) if ns else 0
    pad = torch.zeros(m, dtype=t.dtype, device=t.device)
    pad[: t.numel()] = t
    outs = [torch.zeros_like(pad) for _ in range(world)]
    dist.all_gather(outs, pad, group=group)
    return [o[:k].cpu().numpy() for o, k in zip(outs, ns)]


def distributed_groups(pos_own, box: float, l_x: float, min_size: int = 1, group=None,
                       local_fof=None, device=None):
    """Groups of a box whose particles are spread over the ranks by x-slab.

    pos_own: float32 [n_r, 3], the particles of this rank's slab (x in
    [box r / G, box (r + 1) / G)), in their global order; rank r's particles
    get global ids offset by the particles of ranks < r.
    Returns (gid0, labels, catalogue): the first global id of this rank,
    int64 labels (smallest global id of each own particle's group), and the
    (label, size) rows, ascending label, of the groups of at least min_size
    whose label particle this rank owns.
    local_fof(pos, box, l_x) -> min-index labels (default: this rank's GPU).
    device: where collectives stage their tensors (a CUDA device for NCCL).
    """
    import torch.distributed as dist
    local_fof = local_fof or _gpu_local
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    pos_own = np.ascontiguousarray(pos_own, dtype=np.float32).reshape(-1, 3)
    n_own = pos_own.shape[0]
    lo, hi = slab_bounds(box, world, rank)
    if n_own and not np.all(slab_of(pos_own[:, 0], box, world) == rank):
        raise ValueError("a particle lies outside this rank's slab")
    if not l_x < 0.5 * box:
        raise ValueError("l_x must be below box / 2")

    # step 2: global ids from an exclusive scan of the particle counts
    counts = [int(c[0]) for c in _allgather_var(np.array([n_own], dtype=np.int64), group, device)]
    gid0 = int(sum(counts[:rank]))
    gid_own = gid0 + np.arange(n_own, dtype=np.int64)

    # ghost exchange: every particle within l_x of this rank's slab edges
    reach = l_x * (1.0 + GHOST_MARGIN)
    inner = np.minimum(pos_own[:, 0].astype(np.float64) - lo, hi - pos_own[:, 0].astype(np.float64))
    send = np.nonzero(inner <= reach)[0] if world > 1 else np.zeros(0, dtype=np.int64)
    all_pos = _allgather_var(pos_own[send].reshape(-1).view(np.float32).astype(np.float64), group, device)
    all_gid = _allgather_var(gid_own[send], group, device)
    ghost_pos, ghost_gid = [], []
    for r in range(world):
        if r == rank:
            continue
        p = all_pos[r].astype(np.float32).reshape(-1, 3)
        keep = _periodic_gap(p[:, 0], lo, hi, box) <= reach
        ghost_pos.append(p[keep])
        ghost_gid.append(all_gid[r][keep])
    ghost_pos = np.concatenate(ghost_pos) if ghost_pos else np.zeros((0, 3), np.float32)
    ghost_gid = np.concatenate(ghost_gid) if ghost_gid else np.zeros(0, np.int64)

    # step 1: local groups of own + ghosts
    pos_loc = np.concatenate([pos_own, ghost_pos]) if ghost_pos.size else pos_own
    gid_loc = np.concatenate([gid_own, ghost_gid])
    ids_loc = np.asarray(local_fof(pos_loc, box, l_x), dtype=np.int64)
    # a local group's id: the smallest global id among its members
    gmin = np.full(pos_loc.shape[0], np.iinfo(np.int64).max, dtype=np.int64)
    np.minimum.at(gmin, ids_loc, gid_loc)
    glab = gmin[ids_loc]

    # step 3: links of the groups that touch a slab boundary
    touch = np.concatenate([send, n_own + np.arange(ghost_gid.shape[0])])
    la = glab[touch]
    lb = gid_loc[touch]
    # step 4: all-gather the link lists, union-find over all of them
    ga = np.concatenate(_allgather_var(la, group, device))
    gb = np.concatenate(_allgather_var(lb, group, device))
    own_lab = glab[:n_own]
    uniq, inv, cnt = np.unique(own_lab, return_inverse=True, return_counts=True)
    final_u = fof.fof_merge_links(ga, gb, uniq)
    labels = final_u[inv]

    # sizes: own particles per final label, summed over ranks for the labels
    # of spanning groups (those whose final label differs from a local one
    # or that appear in a link)
    fl, fcnt = np.unique(labels, return_counts=True)
    spanning = np.isin(fl, np.concatenate([ga, gb])) if ga.size else np.zeros(fl.shape, bool)
    part_l = _allgather_var(fl[spanning], group, device)
    part_c = _allgather_var(fcnt[spanning], group, device)
    tot = {}
    for lab_r, cnt_r in zip(part_l, part_c):
        for a_, c_ in zip(lab_r.tolist(), cnt_r.tolist()):
            tot[a_] = tot.get(a_, 0) + c_
    sizes = np.array([tot[a_] if s_ else c_ for a_, c_, s_ in zip(fl.tolist(), fcnt.tolist(), spanning.tolist())],
                     dtype=np.int64)
    owned = (fl >= gid0) & (fl < gid0 + n_own)
    keep = owned & (sizes >= max(min_size, 1))
    catalogue = np.stack([fl[keep], sizes[keep]], axis=1) if keep.any() else np.zeros((0, 2), np.int64)
    return gid0, labels, catalogue
