// Self- and pair-cell linking (the paper's "self" and "pair" tasks over
// cells, Sec. 3.1, Fig. 1), on the binned particle order.
//
// A warp takes 32 consecutive binned particles (one per lane).  For every
// particle the cell itself and its 13 forward neighbours (half of the
// periodic 26-neighbourhood) are searched, so each unordered cell pair is
// visited once; inside the own cell only partners with a larger slot are
// tested.
//
// Cells with at least team_min particles are linked by the warp as a
// team: the lanes that belong to the cell keep their current root, the
// candidates of the neighbour cells are loaded 32 at a time (coalesced
// float4) and filtered by the team's bounding box, the survivors are
// gathered in shared memory, and for up to 32 of them at once their roots
// are taken and
//   * the whole buffer is skipped when all roots on both sides agree,
//   * a pair is skipped when the member's root equals the candidate's,
// which is exact because groups only ever merge: two particles whose roots
// were once equal stay in one group.  Sparse particles search on their own.
//
// Cells that the dense kernels link (subdivided cells, fof_dense.cu) are
// skipped here, as own cells and as neighbours: every pair that involves
// one of them belongs to a dense task.  Where the box has sub-cells, a
// linked pair is at most 2 fine cells apart on each axis, so a particle
// only visits the forward neighbours across faces it lies within 2 fine
// cells of (exact pruning of the stencil).
//
// Linked pairs are merged with the CAS union of fof_internal.cuh.
#include "fof_internal.cuh"

namespace fofgpu {

namespace {

struct Cell {
    int cx, cy, cz;
};

// cell_key with the Morton spreading of the in-brick coordinates (< 16)
// read from a shared-memory table instead of computed
__device__ __forceinline__ int64_t cell_key_tab(const BoxDev& b, int cx, int cy, int cz, const uint32_t* tab)
{
    const int m = b.r - 1;
    const int64_t r3 = (int64_t)b.r * b.r * b.r;
    return b.cell0 + brick_local(b, cx, cy, cz) * r3 + (tab[cx & m] | (tab[cy & m] << 1) | (tab[cz & m] << 2));
}

__device__ __forceinline__ int64_t nbr_key_tab(const BoxDev& b, const Cell& c, int k, const uint32_t* tab)
{
    int dx, dy, dz;
    fwd_offset(k, dx, dy, dz);
    return cell_key_tab(b, wrap_cell(c.cx + dx, b.nc), wrap_cell(c.cy + dy, b.nc), wrap_cell(c.cz + dz, b.nc),
                        tab);
}

__device__ __forceinline__ int64_t nbr_key(const BoxDev& b, const Cell& c, int k)
{
    int dx, dy, dz;
    fwd_offset(k, dx, dy, dz);
    return cell_key(b, wrap_cell(c.cx + dx, b.nc), wrap_cell(c.cy + dy, b.nc),
                    wrap_cell(c.cz + dz, b.nc));
}

// Neighbour k duplicates the own cell or an earlier neighbour (only when
// fewer than 3 cells per axis).
__device__ __forceinline__ bool nbr_duplicate(const BoxDev& b, const Cell& c, int k, int64_t self)
{
    if (b.nc >= 3)
        return false;
    int64_t key = nbr_key(b, c, k);
    if (key == self)
        return true;
    for (int q = 0; q < k; ++q)
        if (nbr_key(b, c, q) == key)
            return true;
    return false;
}

// The forward neighbours particle p can reach.  With sub-cells (q > 1) a
// linked pair is at most 2 fine cells apart on each axis, so p needs the
// neighbour across a face only when it sits within 2 fine cells of that
// face; without sub-cells every neighbour is kept.  Bit k = fwd_offset(k).
__device__ __forceinline__ unsigned reach_mask(const float4& p, const BoxDev& b, const Cell& c)
{
    if (b.q == 1)
        return 0x1fffu;
    const int q = b.q;
    const int lx = fine_coord(p.x, b) - c.cx * q;
    const int ly = fine_coord(p.y, b) - c.cy * q;
    const int lz = fine_coord(p.z, b) - c.cz * q;
    const unsigned hx = lx >= q - 2, hy = ly >= q - 2, hz = lz >= q - 2;
    const unsigned wx = lx <= 1, wy = ly <= 1;
    // per axis, bit d+1 set when offset d in {-1, 0, +1} is reachable
    const unsigned xm = wx | 2u | (hx << 2);
    const unsigned ym = wy | 2u | (hy << 2);
    // k = 0..8: dz = +1, k = 3 (dy+1) + (dx+1); k = 9..11: dz = 0, dy = +1;
    // k = 12: dz = dy = 0, dx = +1  (the order of fwd_offset)
    unsigned m9 = ((ym & 1u) ? xm : 0u) | ((ym & 2u) ? xm << 3 : 0u) | ((ym & 4u) ? xm << 6 : 0u);
    return (hz ? m9 : 0u) | (hy ? xm << 9 : 0u) | (hx << 12);
}

// 16-byte asynchronous copy global -> shared (cp.async), its commit and
// the wait for all of the thread's copies
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_all;" ::: "memory");
}

__device__ __forceinline__ float4 shfl4(float4 v, int src)
{
    v.x = __shfl_sync(kFull, v.x, src);
    v.y = __shfl_sync(kFull, v.y, src);
    v.z = __shfl_sync(kFull, v.z, src);
    return v;
}

// Bounding box of the team's particles.
struct TeamBox {
    float lx, ly, lz, hx, hy, hz;
};

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Inclusive warp prefix sum.
__device__ __forceinline__ int warp_incl(int v, int lane)
{
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += y;
    }
    return v;
}

// Last lane l with start(l) <= t, where `start` is a non-decreasing per-lane
// value with start(0) == 0 <= t (a binary search over the lanes; lanes
// with an empty range share their successor's start and are never chosen).
__device__ __forceinline__ int owner_lane(int start, int t)
{
    int lo = 0;
#pragma unroll
    for (int step = 16; step; step >>= 1) {      // lo + step <= 31 throughout
        const int probe = __shfl_sync(kFull, start, lo + step);
        if (probe <= t) lo += step;
    }
    return lo;
}

// The index of the r-th (0-based) set bit of m (r < popc(m)).
__device__ __forceinline__ int nth_bit(unsigned m, int r)
{
    for (; r > 0; --r) m &= m - 1u;
    return __ffs(m) - 1;
}

// Per-warp staging of the team path: the team's members and one chunk of
// compacted candidates, in shared memory.
struct TeamStage {
    float4 mpos[32];    // member a = lane lo + a of the team: x, y, z, w = reach mask bits
    float4 cpos[32];    // candidate b of the chunk: x, y, z, w = neighbour index (13 = own cell)
    int mroot[32];      // a root of member a (possibly stale: equal roots prove one group)
    int croot[32];      // root snapshot of candidate b
    int cslot[32];      // slot of candidate b
    unsigned lmask[32]; // candidates of the chunk member a is linked to
    TeamBox box;        // the team's bounding box (kept here, not in registers)
    float4 shift[16];   // periodic shift of stream entry k's positions (k < 13)
};

constexpr int kLinkThreads = 256;
constexpr int kLinkWarps = kLinkThreads / 32;
constexpr int kOwnCell = 13;     // stream index of a team's own cell (cells above kTeamSelfMax)

// The buffered candidates S.cpos/cslot[0..c) of a team against its m
// members: their roots; nothing more when all roots (members and
// candidates) agree, which is exact because groups only merge; otherwise
// the m x c pairs are tested lane-parallel (one pair per lane and step),
// skipping pairs whose roots already agree, linked pairs set bits in the
// member's link mask, and each member merges with the distinct candidate
// roots it links to.
template <bool kVar>
__device__ __forceinline__ void team_flush(TeamStage& S, int* __restrict__ parent, const BoxDev& b, int lane,
                                           int m, int first, int c, const UfArgs& uf)
{
    __syncwarp();
    int rj = -1;
    if (lane < c) {
        rj = ufind<kVar>(parent, S.cslot[lane], uf);
        S.croot[lane] = rj;
    }
    const int ref = S.mroot[0];
    const int mr = lane < m ? S.mroot[lane] : ref;
    if (__all_sync(kFull, mr == ref && (lane >= c || rj == ref)))
        return;
    __syncwarp();
    // pair t2 = a * c + bb, advanced by 32 per step without a division
    const int P = m * c;
    int a = lane / c;
    int bb = lane - a * c;
    const int qa = kWarp / c, qb = kWarp - qa * c;
    for (int t2 = lane; t2 < P; t2 += kWarp) {
        const float4 pm = S.mpos[a];
        const float4 qc = S.cpos[bb];
        const int kc = __float_as_int(qc.w);
        bool need = kc == kOwnCell ? S.cslot[bb] > first + a : ((__float_as_int(pm.w) >> kc) & 1);
        need = need && S.mroot[a] != S.croot[bb];
        if (need && linked(pm, qc, b))
            atomicOr(&S.lmask[a], 1u << bb);
        bb += qb;
        a += qa;
        if (bb >= c) {
            bb -= c;
            ++a;
        }
    }
    __syncwarp();
    if (lane < m) {
        unsigned links = S.lmask[lane];
        if (links) {
            int ri = S.mroot[lane];
            int last = -1;
            while (links) {
                const int u = __ffs(links) - 1;
                links &= links - 1u;
                const int rt = S.croot[u];
                if (rt != ri && rt != last) {
                    ri = uunion<kVar>(parent, ri, rt, uf);
                    last = rt;
                }
            }
            S.mroot[lane] = ri;
            S.lmask[lane] = 0u;
        }
    }
    __syncwarp();
}

// One team cell: its members (lanes lo .. lo+m-1 of the warp, contiguous
// slots first .. first+m-1) against every particle they can reach in the
// forward neighbour cells, as ONE stream of candidates, 32 per chunk.
// Lane k < 13 holds neighbour k's first slot and count (0 when the team does
// not reach it or the dense kernels own it); lane 13 the rest of the own
// cell when the cell is larger than kTeamSelfMax (k_team_self links the own
// pairs of smaller cells).  Candidates outside the team's bounding box + l_x
// are dropped; the survivors of successive chunks are gathered in shared
// memory (most are dropped, so a team usually fills one buffer of 32) and
// handed to team_flush when the buffer is full and at the end, so that the
// roots, pair tests and unions of several chunks take one round.
template <bool kVar>
__device__ __forceinline__ void team_cell(TeamStage& S, int* __restrict__ parent,
                                          const float4* __restrict__ sorted, const BoxDev& b, int lane,
                                          int lo, int m, int first, int j0k, int cntk,
                                          const TeamBox& tb, bool filter, const UfArgs& uf)
{
    const int start_k = warp_incl(cntk, lane) - cntk;
    const int total = __shfl_sync(kFull, start_k + cntk, 31);
    int nb = 0;                                 // candidates in the buffer
    // one pass past the end of the stream flushes the rest (team_flush is
    // inlined once)
    for (int cb = 0; cb < total + kWarp; cb += kWarp) {
        const int t = cb + lane;
        bool jv = t < total;
        int k = 0;                              // last stream entry starting at or before t
#pragma unroll
        for (int step = 8; step; step >>= 1) {
            const int probe = k + step <= 13 ? k + step : 13;
            const int sm = __shfl_sync(kFull, start_k, probe);
            if (k + step <= 13 && sm <= t) k += step;
        }
        int j = __shfl_sync(kFull, j0k, k) + (t - __shfl_sync(kFull, start_k, k));
        float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
        if (jv) {
            FOF_DCHECK_SLOT(j, b, uf.err);
            q = sorted[j];
            if (filter && k < kOwnCell) {
                const float4 sh = S.shift[k];
                const float xx = q.x + sh.x, yy = q.y + sh.y, zz = q.z + sh.z;
                const float gx = fmaxf(0.f, fmaxf(tb.lx - xx, xx - tb.hx));
                const float gy = fmaxf(0.f, fmaxf(tb.ly - yy, yy - tb.hy));
                const float gz = fmaxf(0.f, fmaxf(tb.lz - zz, zz - tb.hz));
                jv = gx * gx + gy * gy + gz * gz <= b.bb_reach2;
            }
        }
        const unsigned cand = __ballot_sync(kFull, jv);
        const int c = __popc(cand);
        if (nb + c > kWarp || (cb >= total && nb > 0)) {
            team_flush<kVar>(S, parent, b, lane, m, first, nb, uf);
            nb = 0;
        }
        if (jv) {
            const int r = nb + __popc(cand & lanemask_lt());
            S.cpos[r] = make_float4(q.x, q.y, q.z, __int_as_float(k));
            S.cslot[r] = j;
        }
        nb += c;
    }
}

template <bool kVar>
__global__ void __launch_bounds__(kLinkThreads) k_link(Geometry g, const float4* __restrict__ sorted,
                                                       const int* __restrict__ cell_start, int* parent,
                                                       int dense_min, UfArgs uf)
{
    __shared__ TeamStage stage[kLinkWarps];
    __shared__ uint32_t spread_tab[16];
    if (threadIdx.x < 16)
        spread_tab[threadIdx.x] = spread3(threadIdx.x);
    __syncthreads();
    // each lane's binned record of the warp's next window, copied ahead
    // (cp.async) while the current window is linked; two buffers
    __shared__ float4 ahead[kLinkWarps][2][kWarp];
    const int lane = threadIdx.x & 31;
    TeamStage& S = stage[threadIdx.x >> 5];
    float4* pf = &ahead[threadIdx.x >> 5][0][0];
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    if (lane < 32)
        S.lmask[lane] = 0u;
    __syncwarp();
    if (warp * kWarp + lane < g.total_n)
        cp_async16(pf + lane, sorted + warp * kWarp + lane);
    cp_async_commit();

    int par = 0;
    for (int64_t base = warp * kWarp; base < g.total_n; base += nwarps * kWarp, par ^= 1) {
        const int64_t s = base + lane;
        const bool valid = s < g.total_n;
        float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
        int bi = 0;
        Cell c{0, 0, 0};
        int64_t self = -1;
        int c0 = 0, c1 = 0;
        cp_async_wait_all();                    // this lane's copy of slot s
        if (valid)
            p = pf[par * kWarp + lane];
        // the other buffer was read one window ago: refill it
        if (s + nwarps * kWarp < g.total_n)
            cp_async16(pf + (par ^ 1) * kWarp + lane, sorted + s + nwarps * kWarp);
        cp_async_commit();
        if (valid) {
            bi = box_of(g.box_p0, g.nbox, s);
            const BoxDev& b = g.boxes[bi];
            c.cx = cell_coord(p.x, b);
            c.cy = cell_coord(p.y, b);
            c.cz = cell_coord(p.z, b);
            self = cell_key_tab(b, c.cx, c.cy, c.cz, spread_tab);
            c0 = cell_start[self];
            c1 = cell_start[self + 1];
        }
        const bool sub = valid && is_sub(c1 - c0, g.boxes[bi], dense_min);
        const bool team = valid && !sub && (c1 - c0) >= g.boxes[bi].team_min;
        unsigned tmask = __ballot_sync(kFull, team);

        // ---- team cells: the warp links each cell's members as a team ----
        while (tmask) {
            const int lead = __ffs(tmask) - 1;
            const int64_t key = __shfl_sync(kFull, self, lead);
            const bool mine = team && self == key;
            const unsigned peers = __ballot_sync(kFull, mine);
            tmask &= ~peers;
            const int m = __popc(peers);          // members: lanes lead .. lead + m - 1
            const int tbi = __shfl_sync(kFull, bi, lead);
            const BoxDev& b = g.boxes[tbi];
            Cell tc;
            tc.cx = __shfl_sync(kFull, c.cx, lead);
            tc.cy = __shfl_sync(kFull, c.cy, lead);
            tc.cz = __shfl_sync(kFull, c.cz, lead);
            // coordinates are finite and >= 0 (x + 0 turns -0 into +0), so
            // their bit patterns order like the values: one integer
            // reduction per bound
            TeamBox tbx;
            {
                const unsigned ux = __float_as_uint(p.x + 0.f), uy = __float_as_uint(p.y + 0.f),
                               uz = __float_as_uint(p.z + 0.f);
                const unsigned hi = 0x7f800000u;  // +inf: ignored by the minimum
                tbx.lx = __uint_as_float(__reduce_min_sync(kFull, mine ? ux : hi));
                tbx.ly = __uint_as_float(__reduce_min_sync(kFull, mine ? uy : hi));
                tbx.lz = __uint_as_float(__reduce_min_sync(kFull, mine ? uz : hi));
                tbx.hx = __uint_as_float(__reduce_max_sync(kFull, mine ? ux : 0u));
                tbx.hy = __uint_as_float(__reduce_max_sync(kFull, mine ? uy : 0u));
                tbx.hz = __uint_as_float(__reduce_max_sync(kFull, mine ? uz : 0u));
            }
            const unsigned reach = mine ? reach_mask(p, b, tc) : 0u;
            const unsigned team_reach = __reduce_or_sync(kFull, reach);
            if (mine) {
                S.mpos[lane - lead] = make_float4(p.x, p.y, p.z, __int_as_float((int)reach));
                S.mroot[lane - lead] = ufind<kVar>(parent, (int)s, uf);
            }
            const int first = (int)__shfl_sync(kFull, s, lead);
            const int cell_end = __shfl_sync(kFull, c1, lead);
            const int cell_size = cell_end - __shfl_sync(kFull, c0, lead);
            // lane k < 13: neighbour k's range, if the team reaches it and
            // the dense kernels do not own it; lane 13: the own cell's
            // particles after the first member, for cells k_team_self skips
            int j0k = 0, cntk = 0;
            if (lane < 13 && ((team_reach >> lane) & 1u) && !nbr_duplicate(b, tc, lane, key)) {
                const int64_t nk = nbr_key_tab(b, tc, lane, spread_tab);
                const int j0 = cell_start[nk], j1 = cell_start[nk + 1];
                if (j1 > j0 && !is_sub(j1 - j0, b, dense_min)) {
                    j0k = j0;
                    cntk = j1 - j0;
                }
            } else if (lane == kOwnCell && cell_size > kTeamSelfMax) {
                j0k = first + 1;
                cntk = cell_end - first - 1;
            }
            if (lane < 13) {
                int dx, dy, dz;
                fwd_offset(lane, dx, dy, dz);
                S.shift[lane] = make_float4(tc.cx + dx < 0 ? -b.Lf : (tc.cx + dx >= b.nc ? b.Lf : 0.f),
                                            tc.cy + dy < 0 ? -b.Lf : (tc.cy + dy >= b.nc ? b.Lf : 0.f),
                                            tc.cz + dz >= b.nc ? b.Lf : 0.f, 0.f);
            }
            // Neighbours k < 9 lie one cell up in z.  A team cell there (sorted
            // by z in k_team_self) is cut to the prefix that the box filter can
            // pass: past it, the z gap to the team alone squares above
            // bb_reach2 (the filter's sum only adds non-negative terms, and
            // the gap only grows along the z order).
            // The prefix end is the first slot past the cut (a monotone
            // predicate along the z order), bracketed by two rounds of a
            // 4-ary search: the three lanes 3k, 3k+1, 3k+2 probe neighbour
            // k's range at its quarters in one round.  The cut keeps [0, hi):
            // every slot from hi on is past the cut, so it is conservative
            // (the box filter drops the few kept slots between the first
            // slot past the cut and hi).
            {
                const int gk = lane / 3, sub = lane - 3 * gk;
                const int src = gk < 9 ? gk : 0;
                const int jg = __shfl_sync(kFull, j0k, src), cg = __shfl_sync(kFull, cntk, src);
                const bool act = gk < 9 && b.nc >= 3 && cg >= kSortMin && cg >= b.team_min && cg <= kTeamSelfMax;
                const float sz = tc.cz + 1 >= b.nc ? b.Lf : 0.f;
                int lo = 0, hi = act ? cg : 0;
                for (int round = 0; round < 2 && __any_sync(kFull, lo < hi); ++round) {
                    const int len = hi - lo;
                    const int p0 = lo + len / 4, p1 = lo + len / 2, p2 = lo + (3 * len) / 4;
                    bool beyond = false;
                    if (lo < hi) {
                        const int pr = sub == 0 ? p0 : (sub == 1 ? p1 : p2);
                        const float d = __fsub_rn(__fadd_rn(sorted[jg + pr].z, sz), tbx.hz);
                        beyond = d > 0.f && __fmul_rn(d, d) > b.bb_reach2;
                    }
                    const unsigned g3 = (__ballot_sync(kFull, beyond) >> (3 * src)) & 7u;
                    if (lo < hi) {
                        if (g3 & 1u) {
                            hi = p0;
                        } else if (g3 & 2u) {
                            lo = p0 + 1;
                            hi = p1;
                        } else if (g3 & 4u) {
                            lo = p1 + 1;
                            hi = p2;
                        } else {
                            lo = p2 + 1;
                        }
                    }
                }
                const int cut = __shfl_sync(kFull, hi, 3 * (lane < 9 ? lane : 0));   // lo <= answer <= hi
                if (lane < 9 && b.nc >= 3 && cntk >= kSortMin && cntk >= b.team_min && cntk <= kTeamSelfMax)
                    cntk = cut;
            }
            if (lane == 0)
                S.box = tbx;
            __syncwarp();
            team_cell<kVar>(S, parent, sorted, b, lane, lead, m, first, j0k, cntk, S.box, b.nc >= 3, uf);
        }

        // ---- sparse particles: their (particle, cell) items, then their
        // (particle, candidate) pairs, pooled across the warp ----
        const bool sparse = valid && !team && !sub;
        unsigned reach_s = 0u;
        int own_n = 0;
        if (sparse) {
            const BoxDev& b = g.boxes[bi];
            reach_s = reach_mask(p, b, c);
            if (b.nc < 3)
                for (int k = 0; k < 13; ++k)
                    if (((reach_s >> k) & 1u) && nbr_duplicate(b, c, k, self))
                        reach_s &= ~(1u << k);
            own_n = c1 - (int)s - 1;
        }
        const int nit = sparse ? (own_n > 0) + __popc(reach_s) : 0;
        const int istart = warp_incl(nit, lane) - nit;
        const int T = __shfl_sync(kFull, istart + nit, 31);
        for (int ib = 0; ib < T; ib += kWarp) {
            // item ib + lane: owner o, and its candidate range [j0, j0 + cnt)
            const int t = ib + lane;
            const bool iv = t < T;
            const int o = owner_lane(istart, iv ? t : T - 1);
            const int r = t - __shfl_sync(kFull, istart, o);
            const int own_o = __shfl_sync(kFull, own_n, o);
            const unsigned reach_o = __shfl_sync(kFull, reach_s, o);
            const int obi = __shfl_sync(kFull, bi, o);
            Cell oc;
            oc.cx = __shfl_sync(kFull, c.cx, o);
            oc.cy = __shfl_sync(kFull, c.cy, o);
            oc.cz = __shfl_sync(kFull, c.cz, o);
            int j0 = 0, cnt = 0;
            if (iv) {
                if (own_o > 0 && r == 0) {
                    j0 = (int)(base + o) + 1;
                    cnt = own_o;
                } else {
                    const BoxDev& b = g.boxes[obi];
                    const int k = nth_bit(reach_o, r - (own_o > 0));
                    const int64_t nk = nbr_key_tab(b, oc, k, spread_tab);
                    const int a0 = cell_start[nk], a1 = cell_start[nk + 1];
                    if (!is_sub(a1 - a0, b, dense_min)) {
                        j0 = a0;
                        cnt = a1 - a0;
                    }
                }
            }
            const int cstart = warp_incl(cnt, lane) - cnt;
            const int C = __shfl_sync(kFull, cstart + cnt, 31);
            for (int cb = 0; cb < C; cb += kWarp) {
                const int u = cb + lane;
                const bool uv = u < C;
                const int it = owner_lane(cstart, uv ? u : C - 1);
                int jj = __shfl_sync(kFull, j0, it) + (u - __shfl_sync(kFull, cstart, it));
                const int oo = __shfl_sync(kFull, o, it);
                const float4 po = shfl4(p, oo);
                const int pbi = __shfl_sync(kFull, bi, oo);
                if (uv) {
                    const BoxDev& b = g.boxes[pbi];
                    FOF_DCHECK_SLOT(jj, b, uf.err);
                    if (linked(po, sorted[jj], b))
                        uunion<kVar>(parent, (int)(base + oo), jj, uf);
                }
            }
        }
    }
}

// Self task of a team cell (team_min..kTeamSelfMax particles, not split
// into sub-cells), one warp per cell.  The cell's particles are staged in
// shared memory; the adjacency of the cell is built as bit rows, one
// 32 x 32 block at a time: lane i tests (i, j) for the 32 j of a block,
// collecting row i's word, and a ballot over the lanes gives row j's word of
// the mirrored block, so each unordered pair is tested once outside the
// diagonal blocks.  The components are then traced by breadth-first search
// over bit sets (frontier rows OR-reduced across the warp), in ascending
// order of their smallest member s, and every member's parent is set to s.
// Isolated particles keep parent = self.  The kernel runs before any kernel
// that links across cells, so no other thread touches these parents.
// The kernel is instantiated for cells of up to 128 particles (half the
// shared memory and registers, twice the resident warps) and for 129..256.
constexpr int kTeamWarps = 4;

// Cells of up to 128 particles copy the next cell's positions ahead into
// shared memory (cp.async, buffer Q) instead of registers.
template <int kMax>
constexpr bool team_ahead_smem()
{
    return kMax <= 128;
}

template <int kMax>
struct TeamSmem {
    static constexpr int kWords = kMax / 32;
    static constexpr int kStride = kWords + 1;         // odd stride: conflict-free rows
    float4 P[kMax];
    float4 Q[team_ahead_smem<kMax>() ? kMax : 1];     // the next cell, copied ahead
    unsigned adj[kMax * kStride];
};

// resident blocks per SM the instantiation is compiled for (registers)
template <int kMax>
constexpr int team_blocks()
{
    return kMax <= 128 ? 8 : 4;
}

template <int kMax>
size_t team_smem_bytes()
{
    return sizeof(TeamSmem<kMax>) * kTeamWarps;
}

// Positions that link to nothing: rows and columns beyond the cell's
// particles.  Any difference with a real position or the other sentinel
// squares to +inf in float32, so the pre-test rejects it.
constexpr float kFar = 1e30f;

// Tests of lane i's particle against particles jb*32 + t, t < jn8 (a
// multiple of 8), returning row i's word of block jb.  For an off-diagonal
// block (kOff) the ballot of each test is row j's word of block ib; lane j
// keeps it and stores it once at the end.  The float32 pre-test decides a group of 4 pairs in an
// unrolled loop (groups of 8 hold twice the candidate registers and made
// the 128-particle instantiation spill); pairs in the uncertainty band take
// the exact test after the group, in a loop entered only when some lane has
// one, so the unrolled body stays small.  Inside one cell no pair needs the periodic wrap when
// the box has at least 3 cells per axis (the cell side is then below L/2,
// so the wrapped float32 separation equals the plain difference); kWrap
// takes the full predicate for boxes with fewer cells.
template <int kMax, bool kOff, bool kWrap>
__device__ __forceinline__ unsigned block_tests(const float4& pi, TeamSmem<kMax>& S, int jb, int ib, int jn8,
                                                int lane, const BoxDev& b)
{
    constexpr int kAdjStride = TeamSmem<kMax>::kStride;
    const float4* pj = &S.P[jb * 32];
    unsigned row = 0;
    unsigned col = 0;                          // off-diagonal: row (jb*32 + lane)'s word ib
    const float t_lo = b.t_lo, t_hi = b.t_hi;
    for (int t0 = 0; t0 < jn8; t0 += 4) {
        // 4 pre-tests: certainly linked (below t_lo) or undecided (the band)
        unsigned byte = 0, hib = 0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float4 q = pj[t0 + u];
            float s2;
            if (kWrap) {
                s2 = d2_f32(pi, q, b.Lf);
            } else {
                const float dx = __fsub_rn(pi.x, q.x);
                const float dy = __fsub_rn(pi.y, q.y);
                const float dz = __fsub_rn(pi.z, q.z);
                s2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
            }
            const bool lk = s2 < t_lo;
            byte |= (unsigned)lk << u;
            hib |= (unsigned)(s2 <= t_hi) << u;
            if (kOff) {
                const unsigned c = __ballot_sync(kFull, lk);
                col = lane == t0 + u ? c : col;
            }
        }
        // the exact test for the undecided pairs (rare)
        const unsigned band = hib & ~byte;
        if (__any_sync(kFull, band != 0u)) {
            for (int u = 0; u < 4; ++u) {
                const bool ex = ((band >> u) & 1u) && linked_exact_inl(pi, pj[t0 + u], b.L, b.l2);
                byte |= (unsigned)ex << u;
                if (kOff) {
                    const unsigned c = __ballot_sync(kFull, ex);
                    col |= lane == t0 + u ? c : 0u;
                }
            }
        }
        row |= byte << t0;
    }
    // the mirrored words, one store per lane (rows past the block's
    // particles are never read)
    if (kOff)
        S.adj[(jb * 32 + lane) * kAdjStride + ib] = col;
    return row;
}

// Positions of a listed cell (size << 32 | first slot) into registers:
// lane k holds particles k, k + 32, ...
template <int kMin, int kMax>
__device__ __forceinline__ void team_fetch(float4 (&R)[kMax / 32], int64_t e, const float4* sorted, int lane)
{
    const int c0 = (int)(uint32_t)e, m = (int)(e >> 32);
    if (m <= kMin || m > kMax)                 // another instantiation's cell
        return;
#pragma unroll
    for (int r = 0; r < kMax / 32; ++r)
        if (lane + 32 * r < m)
            R[r] = sorted[c0 + lane + 32 * r];
}

// The same into shared memory (S.Q) with cp.async, one commit group.
template <int kMin, int kMax>
__device__ __forceinline__ void team_fetch_smem(TeamSmem<kMax>& S, int64_t e, const float4* sorted, int lane)
{
    const int c0 = (int)(uint32_t)e, m = (int)(e >> 32);
    if (m > kMin && m <= kMax) {
#pragma unroll
        for (int r = 0; r < kMax / 32; ++r)
            if (lane + 32 * r < m)
                cp_async16(&S.Q[lane + 32 * r], sorted + c0 + lane + 32 * r);
    }
    cp_async_commit();
}

// Sorts the staged cell (nw * 32 entries of S.P, sentinels after the cell's
// particles) by z in place: a bitonic network over the next power of two,
// padded with more sentinels.  Every z is finite and non-negative, the
// sentinels' z (kFar) exceeds every position, so the cell's particles come
// first in exact float order.
template <int kMax>
__device__ __forceinline__ void sort_cell_z(TeamSmem<kMax>& S, int nw, int lane)
{
    const int n = nw * 32;
    int n2 = 32;
    while (n2 < n) n2 <<= 1;                   // <= kMax
    for (int k = n + lane; k < n2; k += 32)
        S.P[k] = make_float4(kFar, kFar, kFar, 0.f);
    __syncwarp();
    for (int size = 2; size <= n2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            // pair p: its lower index i is p with a zero inserted at the
            // stride bit, so every lane has a pair and accesses stay dense
            for (int pr = lane; pr < (n2 >> 1); pr += 32) {
                const int i = ((pr & ~(stride - 1)) << 1) | (pr & (stride - 1));
                const int l = i | stride;
                const float4 a = S.P[i], c = S.P[l];
                if ((a.z > c.z) == ((i & size) == 0)) {
                    S.P[i] = c;
                    S.P[l] = a;
                }
            }
            __syncwarp();
        }
    }
}

template <int kMin, int kMax>
__global__ void __launch_bounds__(kTeamWarps * 32, team_blocks<kMax>())
    k_team_self(Geometry g, const int64_t* __restrict__ list, const int* __restrict__ n_list, int64_t back,
                float4* sorted, int* __restrict__ parent, int* __restrict__ minorig, int* err)
{
    // entries from the front of the list (back == 0) or from its back end
    auto entry = [&](int i) { return back ? list[back - 1 - i] : list[i]; };
    constexpr int kTeamMax = kMax;
    constexpr int kTeamWords = kMax / 32;
    constexpr int kAdjStride = TeamSmem<kMax>::kStride;
    extern __shared__ float4 team_raw[];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    TeamSmem<kMax>& S = reinterpret_cast<TeamSmem<kMax>*>(team_raw)[wid];
    const int n = *n_list;
    const int stride = gridDim.x * kTeamWarps;
    // software pipeline: the next cell's positions are loaded while this
    // cell is linked (into shared memory with cp.async for cells up to 128,
    // into registers for larger ones), and the entry after it is read
    int it = blockIdx.x * kTeamWarps + wid;
    int64_t e = it < n ? entry(it) : 0;
    constexpr bool kAhead = team_ahead_smem<kMax>();
    float4 R[kAhead ? 1 : kTeamWords];
    if constexpr (kAhead)
        team_fetch_smem<kMin, kMax>(S, e, sorted, lane);
    else
        team_fetch<kMin, kMax>(R, e, sorted, lane);
    int64_t e_next = it + stride < n ? entry(it + stride) : 0;
    for (; it < n; it += stride) {
        const int c0 = (int)(uint32_t)e, m = (int)(e >> 32);
        const int nw = (m + 31) >> 5;
        const bool in_range = m > kMin && m <= kMax;
        if constexpr (kAhead)
            cp_async_wait_all();               // each lane reads back only its own copies
        if (in_range) {
#pragma unroll
            for (int r = 0; r < kTeamWords; ++r) {   // the ragged tail links nothing
                const int k = lane + 32 * r;
                if (k < nw * 32) {
                    float4 v = make_float4(kFar, kFar, kFar, 0.f);
                    if (k < m) {
                        if constexpr (kAhead)
                            v = S.Q[k];
                        else
                            v = R[r];
                    }
                    S.P[k] = v;
                }
            }
        }
        __syncwarp();
        e = e_next;
        if (it + stride < n) {
            if constexpr (kAhead)
                team_fetch_smem<kMin, kMax>(S, e, sorted, lane);
            else
                team_fetch<kMin, kMax>(R, e, sorted, lane);
        }
        e_next = it + 2 * stride < n ? entry(it + 2 * stride) : 0;
        if (!in_range)                         // another instantiation's cell
            continue;
        const BoxDev& b = g.boxes[box_of(g.box_p0, g.nbox, c0)];

        // the cell in z order, also in global memory: the streams of the
        // neighbours below then read only a z-prefix of it (k_link), and
        // blocks of 32 here are z-slabs whose gaps prune block pairs.  No
        // kernel has read these slots' order yet (cross-cell links come later).
        // Cells below kSortMin are not sorted (k_link searches no smaller).
        if (m >= kSortMin) {
            sort_cell_z<kMax>(S, nw, lane);
            for (int k = lane; k < m; k += 32) {
                const float4 q = S.P[k];
                sorted[c0 + k] = q;
                minorig[c0 + k] = __float_as_int(q.w);
            }
        }

        // adjacency rows (row1: the only word when nw == 1)
        unsigned row1 = 0u;
        for (int ib = 0; ib < nw; ++ib) {
            const int i = ib * 32 + lane;
            const float4 pi = i < m ? S.P[i] : make_float4(-kFar, -kFar, -kFar, 0.f);
            for (int jb = ib; jb < nw; ++jb) {
                const int jn8 = (min(32, m - jb * 32) + 7) & ~7;
                unsigned row;
                // z-slabs of a sorted cell too far apart: every pair's float32
                // separation squared exceeds t_hi (rounding is monotone), so no link
                const float gap = jb > ib && m >= kSortMin ? __fsub_rn(S.P[jb * 32].z, S.P[ib * 32 + 31].z) : 0.f;
                if (b.nc >= 3 && gap > 0.f && __fmul_rn(gap, gap) > b.t_hi) {
                    row = 0u;
                    if (lane < min(32, m - jb * 32))
                        S.adj[(jb * 32 + lane) * kAdjStride + ib] = 0u;
                } else if (b.nc >= 3) {
                    row = jb == ib ? block_tests<kMax, false, false>(pi, S, jb, ib, jn8, lane, b)
                                   : block_tests<kMax, true, false>(pi, S, jb, ib, jn8, lane, b);
                } else {
                    row = jb == ib ? block_tests<kMax, false, true>(pi, S, jb, ib, jn8, lane, b)
                                   : block_tests<kMax, true, true>(pi, S, jb, ib, jn8, lane, b);
                }
                if (jb == ib)
                    row &= ~(1u << lane);      // the particle itself
                if (nw == 1)
                    row1 = i < m ? row : 0u;
                else if (i < m)
                    S.adj[i * kAdjStride + jb] = row;
            }
        }
        if (nw == 1) {
            // up to 32 particles: lane i keeps row i in a register, and a BFS
            // step is one OR-reduction of the frontier's rows
            unsigned todo = __ballot_sync(kFull, row1 != 0u);
            while (todo) {
                const int s = __ffs(todo) - 1;
                unsigned comp = 1u << s, front = comp;
                for (int step = 0; step < 32; ++step) {   // every step adds a vertex
                    const unsigned nxt =
                        __reduce_or_sync(kFull, ((front >> lane) & 1u) ? row1 : 0u) & ~comp;
                    if (!nxt)
                        break;
                    comp |= nxt;
                    front = nxt;
                }
                todo &= ~comp;
                if (((comp >> lane) & 1u) && lane != s)
                    parent[c0 + lane] = c0 + s;
            }
            __syncwarp();                      // smem reused by the next cell
            continue;
        }
        __syncwarp();

        // lane w < nw holds word w of each vertex set
        unsigned todo = 0;
        for (int ib = 0; ib < nw; ++ib) {
            const int v = ib * 32 + lane;
            unsigned any = 0;
            if (v < m)
                for (int k = 0; k < nw; ++k)
                    any |= S.adj[v * kAdjStride + k];
            const unsigned w = __ballot_sync(kFull, any != 0);
            todo = lane == ib ? w : todo;
        }
        for (;;) {
            const unsigned nz = __ballot_sync(kFull, todo != 0);
            if (!nz)
                break;
            const int w0 = __ffs(nz) - 1;
            const int s = w0 * 32 + __ffs(__shfl_sync(kFull, todo, w0)) - 1;
            unsigned comp = lane == w0 ? 1u << (s & 31) : 0u;
            unsigned front = comp;
            for (int step = 0; step < kTeamMax; ++step) {   // every step adds a vertex
                unsigned acc[kTeamWords];
#pragma unroll
                for (int k = 0; k < kTeamWords; ++k)
                    acc[k] = 0;
                for (int w = 0; w < nw; ++w) {
                    const unsigned fw = __shfl_sync(kFull, front, w);
                    if ((fw >> lane) & 1u) {
                        const unsigned* r = &S.adj[(w * 32 + lane) * kAdjStride];
#pragma unroll
                        for (int k = 0; k < kTeamWords; ++k)
                            if (k < nw) acc[k] |= r[k];
                    }
                }
                unsigned nxt = 0;
#pragma unroll
                for (int k = 0; k < kTeamWords; ++k)
                    if (k < nw) {
                        const unsigned r = __reduce_or_sync(kFull, acc[k]);
                        nxt = lane == k ? r : nxt;
                    }
                nxt &= ~comp;
                comp |= nxt;
                front = nxt;
                if (!__ballot_sync(kFull, nxt != 0))
                    break;
            }
            todo &= ~comp;
            for (int w = 0; w < nw; ++w) {
                const unsigned cw = __shfl_sync(kFull, comp, w);
                if ((cw >> lane) & 1u)
                    parent[c0 + w * 32 + lane] = c0 + s;
            }
        }
        __syncwarp();                          // smem reused by the next cell
    }
}

}  // namespace

cudaError_t launch_team_self(const Geometry& g, const Work& w, cudaStream_t s)
{
    if (g.total_n == 0)
        return cudaSuccess;
    // the shared-memory opt-in is per device; setting it again is harmless
    static bool configured[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !configured[dev]) {
        e = cudaFuncSetAttribute(k_team_self<0, kTeamSplit>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)team_smem_bytes<kTeamSplit>());
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k_team_self<kTeamSplit, kTeamSelfMax>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)team_smem_bytes<kTeamSelfMax>());
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) configured[dev] = true;
    }
    k_team_self<0, kTeamSplit><<<sm_count() * team_blocks<kTeamSplit>(), kTeamWarps * 32,
                                 team_smem_bytes<kTeamSplit>(), s>>>(
        g, w.team_list, w.n_team, 0, w.sorted, w.parent, w.minorig, &w.status->err);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_team_self<kTeamSplit, kTeamSelfMax><<<sm_count() * team_blocks<kTeamSelfMax>(), kTeamWarps * 32,
                                            team_smem_bytes<kTeamSelfMax>(), s>>>(
        g, w.team_list, w.n_team_hi, w.team_cap, w.sorted, w.parent, w.minorig, &w.status->err);
    return cudaGetLastError();
}

cudaError_t launch_link(const Geometry& g, const Work& w, int dense_min, const UfArgs& uf, cudaStream_t s)
{
    if (g.total_n == 0)
        return cudaSuccess;
    int64_t warps = (g.total_n + kWarp - 1) / kWarp;
    int64_t blocks = (warps * kWarp + kLinkThreads - 1) / kLinkThreads;
    int64_t cap = (int64_t)sm_count() * 8;
    if (blocks > cap) blocks = cap;
    if (uf.var)
        k_link<true><<<(unsigned)blocks, kLinkThreads, 0, s>>>(g, w.sorted, w.cell_start, w.parent, dense_min, uf);
    else
        k_link<false><<<(unsigned)blocks, kLinkThreads, 0, s>>>(g, w.sorted, w.cell_start, w.parent, dense_min, uf);
    return cudaGetLastError();
}

}  // namespace fofgpu
