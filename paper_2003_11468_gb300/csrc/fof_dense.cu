// Dense cells: the paper's self and pair tasks (Sec. 3.1, Fig. 1) for cells
// that hold many particles, done in shared memory.
//
// A cell with T <= m <= kDenseMax particles (T = dense_min) in a box whose
// cells can be split ("subdivided" cells) is cut into q^3 sub-cells of side
// hf with l_x/2 < hf <= l_x / (sqrt(3) (1 + 2^-7)).  Two facts follow from
// the float32 cell-index margin (fof_plan.cu, setup_box):
//   * every two particles of one sub-cell are linked (the sub-cell diameter
//     is below l_x even with the index rounding), so a sub-cell is a clique;
//   * every linked pair lies at most 2 sub-cells apart on each axis.
// Hence the groups inside a dense cell follow from cliques plus one linking
// pair per pair of sub-cells within +-2, found with early exit.
//
//   dense_self   one CTA per subdivided cell: counting sort into sub-cells
//                in shared memory, a shared-memory union-find over the
//                cell (cliques, then sub-cell pairs), the cell's forest
//                written to the global parent array (roots = smallest slot,
//                as union-by-root onto the lower offset gives), the cell's
//                root if it is one group; then every particle of the 26
//                neighbour cells that are NOT subdivided is linked against
//                the sub-cells within its +-2 window with the global CAS
//                union.
//   dense_pairs  one CTA per subdivided cell A: each forward neighbour B
//                that is subdivided too.  If both cells are one group each
//                and their roots already agree there is nothing to do;
//                otherwise B's particles are linked against A's sub-cells
//                (and, when both are single groups, the search stops at the
//                first link).
#include "fof_internal.cuh"

namespace fofgpu {

namespace {


struct DenseSmem {
    float4* P;           // [kDenseMax] positions of the cell, slot order
    int* lpar;           // [kDenseMax] shared-memory forest (local indices)
    unsigned short* skey;   // [kDenseMax] sub-cell of each particle
    unsigned short* order;  // [kDenseMax] local indices grouped by sub-cell
    int* sstart;         // [kMaxQ3 + 1] sub-cell starts in order[]
    int* groot;          // [kMaxQ3] global root of each sub-cell
    unsigned short* ne;  // [kMaxQ3] non-empty sub-cells
    int* misc;           // [8] scalars
    int* nbj0;           // [26] first slot of each neighbour cell
    int* nbpref;         // [27] prefix of the neighbour particle counts to visit
    int* nbflag;         // [26] per neighbour: 1 = both cells single groups
    int* nbdone;         // [26] per neighbour: a link was made (single groups)
    unsigned* rowmask;   // [kMaxQ * kMaxQ] per (z, y) row: bit x = sub-cell non-empty
};

// Two size classes of dense cells, each its own instantiation: cells up to
// kDenseSmall particles need a sixth of the shared memory, so six CTAs (of
// 256 threads) share an SM and barrier stalls of one cell overlap the work
// of five others; larger cells take two CTAs of 512 threads per SM.
constexpr int kDenseSmall = 768;

template <int kM>
__host__ __device__ constexpr size_t dense_smem_bytes()
{
    return (size_t)kM * (16 + 4 + 2 + 2) + (size_t)(kMaxQ3 + 1) * 4 + (size_t)kMaxQ3 * 4 +
           (size_t)kMaxQ3 * 2 + 512 + (size_t)kMaxQ * kMaxQ * 4;
}

template <int kM>
__device__ __forceinline__ DenseSmem carve(unsigned char* base)
{
    DenseSmem s;
    size_t off = 0;
    s.P = (float4*)(base + off);           off += (size_t)kM * 16;
    s.lpar = (int*)(base + off);           off += (size_t)kM * 4;
    s.sstart = (int*)(base + off);         off += (size_t)(kMaxQ3 + 1) * 4;
    s.groot = (int*)(base + off);          off += (size_t)kMaxQ3 * 4;
    s.misc = (int*)(base + off);
    s.nbj0 = s.misc + 8;
    s.nbpref = s.misc + 40;
    s.nbflag = s.misc + 72;
    s.nbdone = s.misc + 100;
    off += 512;
    s.rowmask = (unsigned*)(base + off);   off += (size_t)kMaxQ * kMaxQ * 4;
    s.skey = (unsigned short*)(base + off); off += (size_t)kM * 2;
    s.order = (unsigned short*)(base + off); off += (size_t)kM * 2;
    s.ne = (unsigned short*)(base + off);
    return s;
}

// shared-memory union-find over local indices (hook the larger root onto
// the smaller, like the global one); volatile so that a retry re-reads
// what other threads hooked
// Paths strictly decrease and every failed CAS means another hook
// succeeded, so both loops end within kDenseMax steps; the caps only turn
// a corrupted forest into a reported error instead of a hang.
__device__ __forceinline__ int lfind(int* lpar_, int x, int* err)
{
    volatile int* lpar = lpar_;
    int p = lpar[x];
    for (int step = 0; p != x; ++step) {
        int gp = lpar[p];
        if (gp == p)
            return p;
        if (gp > p || step > kDenseMax) {
            atomicOr(err, kErrInternal);
            return p;
        }
        lpar[x] = gp;
        x = gp;
        p = lpar[x];
    }
    return x;
}

__device__ __forceinline__ void lunion(int* lpar, int a, int b, int* err)
{
    for (int it = 0; it <= 2 * kDenseMax; ++it) {
        a = lfind(lpar, a, err);
        b = lfind(lpar, b, err);
        if (a == b)
            return;
        int hi = a > b ? a : b, lo = a > b ? b : a;
        if (atomicCAS(lpar + hi, hi, lo) == hi)
            return;
    }
    atomicOr(err, kErrInternal);
}

// Load cell [c0, c0+m) and build its sub-cell structure in shared memory.
// (ox, oy, oz) = fine coordinates of the cell's corner.  Returns the
// number of non-empty sub-cells; sets misc[1] on an inconsistency.
__device__ __forceinline__ int build_cell(const DenseSmem& S, const float4* __restrict__ sorted, int c0, int m,
                          const BoxDev& b, int ox, int oy, int oz, int* err)
{
    const int q = b.q, q3 = q * q * q;
    for (int a = threadIdx.x; a <= q3; a += blockDim.x) S.sstart[a] = 0;
    if (threadIdx.x == 0) S.misc[0] = 0;
    __syncthreads();
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        float4 p = sorted[c0 + k];
        S.P[k] = p;
        int sx = fine_coord(p.x, b) - ox, sy = fine_coord(p.y, b) - oy, sz = fine_coord(p.z, b) - oz;
        bool ok = sx >= 0 && sx < q && sy >= 0 && sy < q && sz >= 0 && sz < q;
        if (!ok) {
            atomicOr(err, kErrInternal);
            sx = sx < 0 ? 0 : (sx >= q ? q - 1 : sx);
            sy = sy < 0 ? 0 : (sy >= q ? q - 1 : sy);
            sz = sz < 0 ? 0 : (sz >= q ? q - 1 : sz);
        }
        int key = (sz * q + sy) * q + sx;
        S.skey[k] = (unsigned short)key;
        atomicAdd(S.sstart + key, 1);
    }
    __syncthreads();
    if (threadIdx.x < 32) {            // exclusive scan of q3 + 1 counts by one warp
        int carry = 0;
        for (int base = 0; base <= q3; base += 32) {
            int i = base + threadIdx.x;
            int v = i <= q3 ? S.sstart[i] : 0;
            int x = v;
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(kFull, x, o);
                if ((int)threadIdx.x >= o) x += y;
            }
            if (i <= q3) S.sstart[i] = carry + x - v;
            carry += __shfl_sync(kFull, x, 31);
        }
    }
    __syncthreads();
    for (int a = threadIdx.x; a < q3; a += blockDim.x) {
        S.groot[a] = S.sstart[a];      // cursor
        if (S.sstart[a + 1] > S.sstart[a]) {
            int slot = atomicAdd(S.misc, 1);
            S.ne[slot] = (unsigned short)a;
        }
    }
    for (int row = threadIdx.x; row < q * q; row += blockDim.x) {
        unsigned mask = 0;
        for (int x = 0; x < q; ++x) {
            int a = row * q + x;
            mask |= (unsigned)(S.sstart[a + 1] > S.sstart[a]) << x;
        }
        S.rowmask[row] = mask;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < m; k += blockDim.x) {
        int pos = atomicAdd(S.groot + S.skey[k], 1);
        S.order[pos] = (unsigned short)k;
    }
    __syncthreads();
    return S.misc[0];
}

// Link particle pj (current root rj) against the sub-cells of the cell in
// shared memory within its +-2 window; (rx, ry, rz) are pj's fine
// coordinates relative to the cell corner.  groot[a] holds a root of
// sub-cell a (possibly stale: equal roots prove one group, different ones
// only mean "test").  single: the cell is one group, so the first link is
// enough.  Returns pj's root after the unions it made.
template <bool kVar>
__device__ __forceinline__ int link_window(const DenseSmem& S, int* parent, const BoxDev& b,
                                           float4 pj, int rj, int rx, int ry, int rz, bool single,
                                           const UfArgs& uf, bool& linked_any)
{
    const int q = b.q;
    const int x0 = max(rx - 2, 0), x1 = min(rx + 2, q - 1);
    const int y0 = max(ry - 2, 0), y1 = min(ry + 2, q - 1);
    const int z0 = max(rz - 2, 0), z1 = min(rz + 2, q - 1);
    // pj's position inside its own fine cell, in fine units
    const float ux = __fmul_rn(pj.x, b.inv_hf) - (float)fine_coord(pj.x, b);
    const float uy = __fmul_rn(pj.y, b.inv_hf) - (float)fine_coord(pj.y, b);
    const float uz = __fmul_rn(pj.z, b.inv_hf) - (float)fine_coord(pj.z, b);
    const unsigned span = (x1 >= x0) ? ((2u << x1) - (1u << x0)) : 0u;   // bits x0..x1
    for (int z = z0; z <= z1; ++z) {
        // gap from pj to the sub-cell layer z, in fine units (0 when adjacent)
        float gz = z < rz ? (float)(rz - z - 1) + uz : (z > rz ? (float)(z - rz - 1) + (1.f - uz) : 0.f);
        if (gz * gz > b.reach2)
            continue;                            // the whole layer is out of reach
        for (int y = y0; y <= y1; ++y) {
            float gy = y < ry ? (float)(ry - y - 1) + uy : (y > ry ? (float)(y - ry - 1) + (1.f - uy) : 0.f);
            if (gy * gy + gz * gz > b.reach2)
                continue;                        // the whole row is out of reach
            unsigned bits = S.rowmask[z * q + y] & span;     // non-empty sub-cells only
            while (bits) {
                const int x = __ffs(bits) - 1;
                bits &= bits - 1u;
                float gx = x < rx ? (float)(rx - x - 1) + ux : (x > rx ? (float)(x - rx - 1) + (1.f - ux) : 0.f);
                if (gx * gx + gy * gy + gz * gz > b.reach2)
                    continue;                    // the whole sub-cell is out of reach
                int a = (z * q + y) * q + x;
                int beg = S.sstart[a], end = S.sstart[a + 1];
                if (beg == end || S.groot[a] == rj)
                    continue;
                for (int t = beg; t < end; ++t) {
                    if (linked_ool(pj, S.P[S.order[t]], b)) {
                        rj = uunion<kVar>(parent, rj, S.groot[a], uf);
                        linked_any = true;
                        if (single)
                            return rj;
                        break;
                    }
                }
            }
        }
    }
    return rj;
}

// fine coordinates of pj relative to the corner (ox, oy, oz), unwrapped
// into the window next to the cell (the box has at least 3 cells per axis)
__device__ __forceinline__ bool rel_fine(float4 pj, const BoxDev& b, int ox, int oy, int oz,
                                         int& rx, int& ry, int& rz)
{
    const int q = b.q, nf = b.nf;
    rx = fine_coord(pj.x, b) - ox;
    ry = fine_coord(pj.y, b) - oy;
    rz = fine_coord(pj.z, b) - oz;
    rx = rx < -2 ? rx + nf : (rx > q + 1 ? rx - nf : rx);
    ry = ry < -2 ? ry + nf : (ry > q + 1 ? ry - nf : ry);
    rz = rz < -2 ? rz + nf : (rz > q + 1 ? rz - nf : rz);
    return rx >= -2 && rx <= q + 1 && ry >= -2 && ry <= q + 1 && rz >= -2 && rz <= q + 1;
}

__device__ __forceinline__ int64_t nbr_cell(const BoxDev& b, int cx, int cy, int cz, int dx, int dy,
                                            int dz)
{
    return cell_key(b, wrap_cell(cx + dx, b.nc), wrap_cell(cy + dy, b.nc), wrap_cell(cz + dz, b.nc));
}

// prefix of S.nbpref[1..26] holding counts -> exclusive starts; one warp
__device__ __forceinline__ void neighbour_prefix(const DenseSmem& S)
{
    if (threadIdx.x < 32) {
        int lane = threadIdx.x;
        int v = (lane >= 1 && lane <= 26) ? S.nbpref[lane] : 0;
        int x = v;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(kFull, x, o);
            if (lane >= o) x += y;
        }
        if (lane <= 26) S.nbpref[lane] = x;    // nbpref[0] = 0, nbpref[k] = sum of counts < k
    }
}

// the neighbour k whose particles contain flat index t
__device__ __forceinline__ int neighbour_of(const DenseSmem& S, int t)
{
    int lo = 0, hi = 25;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (S.nbpref[mid] <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

template <bool kVar, int kLo, int kM, int kThreads, int kBlocks>
__global__ void __launch_bounds__(kThreads, kBlocks) k_dense_self(Geometry g, Work w, int dense_min,
                                                              UfArgs uf)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const DenseSmem S = carve<kM>(smem_raw);
    int* err = uf.err;
    const int n_dense = *w.n_dense;
    for (int it = blockIdx.x; it < n_dense; it += gridDim.x) {
        const int64_t key = w.dense_list[it];
        const int c0 = w.cell_start[key], c1 = w.cell_start[key + 1];
        const int m = c1 - c0;
        if (m <= kLo || m > kM)
            continue;                             // the other size class's cell (block-uniform)
        const BoxDev& b = g.boxes[box_of(g.box_p0, g.nbox, c0)];
        const int q = b.q;
        const float4 p0 = w.sorted[c0];
        const int cx = cell_coord(p0.x, b), cy = cell_coord(p0.y, b), cz = cell_coord(p0.z, b);
        const int ox = cx * q, oy = cy * q, oz = cz * q;
        // neighbour table, filled while the cell is built
        if (threadIdx.x < 26) {
            int k = threadIdx.x;
            int code = k < 13 ? k : k + 1;            // the 26 offsets, centre skipped
            int64_t nk = nbr_cell(b, cx, cy, cz, code % 3 - 1, (code / 3) % 3 - 1, code / 9 - 1);
            int j0 = w.cell_start[nk], j1 = w.cell_start[nk + 1];
            S.nbj0[k] = j0;
            S.nbpref[k + 1] = (j1 > j0 && !is_sub(j1 - j0, b, dense_min)) ? j1 - j0 : 0;
        }
        const int ne = build_cell(S, w.sorted, c0, m, b, ox, oy, oz, err);
        neighbour_prefix(S);

        // cliques: every member of a sub-cell hangs on its smallest member
        for (int t = threadIdx.x; t < ne; t += blockDim.x) {
            int a = S.ne[t];
            int beg = S.sstart[a], end = S.sstart[a + 1];
            int rep = S.order[beg];
            for (int u = beg + 1; u < end; ++u) rep = min(rep, (int)S.order[u]);
            for (int u = beg; u < end; ++u) S.lpar[S.order[u]] = rep;
            S.groot[a] = rep;
        }
        __syncthreads();
        // pairs of sub-cells within the cell, half of the +-2 stencil: the
        // three face offsets first; when they leave the cell one group the
        // other 59 offsets cannot change anything and are skipped
        for (int pass = 0; pass < 2; ++pass) {
            // pass 0: the 3 face offsets (one item each); pass 1: the 13
            // half-stencil rows (dz, dy) of the +-2 stencil, each a span of
            // dx, whose non-empty sub-cells come from the row masks
            const int nofs = pass == 0 ? 3 : 13;
            for (int item = threadIdx.x; item < ne * nofs; item += blockDim.x) {
                const int a = S.ne[item / nofs];
                const int o = item % nofs;
                const int ax = a % q, ay = (a / q) % q, az = a / (q * q);
                int dy, dz, dxlo, dxhi;
                if (pass == 0) {
                    dz = o == 2; dy = o == 1; dxlo = dxhi = o == 0;
                } else if (o < 10) {             // dz = 1, 2 and dy = -2..2
                    dz = 1 + o / 5; dy = o % 5 - 2; dxlo = -2; dxhi = 2;
                } else if (o < 12) {             // dz = 0, dy = 1, 2
                    dz = 0; dy = o - 9; dxlo = -2; dxhi = 2;
                } else {                         // dz = dy = 0, dx = 1, 2
                    dz = 0; dy = 0; dxlo = 1; dxhi = 2;
                }
                const int by = ay + dy, bz = az + dz;
                if (by < 0 || by >= q || bz >= q)
                    continue;
                const int xlo = max(ax + dxlo, 0), xhi = min(ax + dxhi, q - 1);
                if (xlo > xhi)
                    continue;
                unsigned bits = S.rowmask[bz * q + by] & ((2u << xhi) - (1u << xlo));
                while (bits) {
                    const int bx = __ffs(bits) - 1;
                    bits &= bits - 1u;
                    if (pass == 1 && ((bx - ax == 1 && dy == 0 && dz == 0) ||
                                      (bx == ax && dy == 1 && dz == 0) ||
                                      (bx == ax && dy == 0 && dz == 1)))
                        continue;                // a face offset, done in pass 0
                    const int bb = (bz * q + by) * q + bx;
                    int ra = lfind(S.lpar, S.groot[a], err), rb = lfind(S.lpar, S.groot[bb], err);
                    if (ra == rb)
                        continue;
                    const int a0 = S.sstart[a], a1 = S.sstart[a + 1];
                    const int b0 = S.sstart[bb], b1 = S.sstart[bb + 1];
                    bool done = false;
                    for (int u = a0; u < a1 && !done; ++u) {
                        float4 pu = S.P[S.order[u]];
                        for (int v = b0; v < b1; ++v)
                            if (linked_ool(pu, S.P[S.order[v]], b)) {
                                lunion(S.lpar, ra, rb, err);
                                done = true;
                                break;
                            }
                    }
                }
            }
            __syncthreads();
            if (pass == 0) {
                const int r0 = lfind(S.lpar, S.groot[S.ne[0]], err);
                int differs = 0;
                for (int t = threadIdx.x; t < ne; t += blockDim.x)
                    differs |= lfind(S.lpar, S.groot[S.ne[t]], err) != r0;
                if (!__syncthreads_or(differs))
                    break;                          // block-uniform
            }
        }
        if (threadIdx.x == 0) {
            S.misc[2] = INT_MAX;
            S.misc[3] = -1;
        }
        __syncthreads();
        // the cell's forest goes to global memory; roots are smallest slots
        int lo = INT_MAX, hi = -1;
        for (int k = threadIdx.x; k < m; k += blockDim.x) {
            int r = lfind(S.lpar, k, err);
            w.parent[c0 + k] = c0 + r;
            lo = min(lo, r);
            hi = max(hi, r);
        }
        lo = (int)__reduce_min_sync(kFull, (unsigned)lo);
        hi = (int)__reduce_max_sync(kFull, (unsigned)(hi + 1)) - 1;
        if ((threadIdx.x & 31) == 0) {
            atomicMin(S.misc + 2, lo);
            atomicMax(S.misc + 3, hi);
        }
        __syncthreads();
        for (int t = threadIdx.x; t < ne; t += blockDim.x) {
            int a = S.ne[t];
            S.groot[a] = c0 + lfind(S.lpar, S.groot[a], err);   // global root of the sub-cell
        }
        __threadfence();
        __syncthreads();
        const int single = (S.misc[2] == S.misc[3]) ? c0 + S.misc[2] : -1;
        if (threadIdx.x == 0)
            w.dense_root[c0 / dense_min] = single;

        // particles of the 26 neighbours that are not subdivided, all at
        // once: every pair of them with this cell belongs to this task
        const int total = S.nbpref[26];
        int ru = single;
        for (int t = threadIdx.x; t < total; t += blockDim.x) {
            int k = neighbour_of(S, t);
            int j = S.nbj0[k] + (t - S.nbpref[k]);
            FOF_DCHECK_SLOT(j, b, err);
            float4 pj = w.sorted[j];
            int rx, ry, rz;
            if (!rel_fine(pj, b, ox, oy, oz, rx, ry, rz))
                continue;
            int rj = ufind<kVar>(w.parent, j, uf);
            if (single >= 0) {
                ru = ufind<kVar>(w.parent, ru, uf);
                if (rj == ru)
                    continue;
            }
            bool any = false;
            int r = link_window<kVar>(S, w.parent, b, pj, rj, rx, ry, rz, single >= 0, uf, any);
            if (any && single >= 0)
                ru = r;
        }
        __syncthreads();
    }
}

template <bool kVar, int kLo, int kM, int kThreads, int kBlocks>
__global__ void __launch_bounds__(kThreads, kBlocks) k_dense_pairs(Geometry g, Work w, int dense_min,
                                                               UfArgs uf)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const DenseSmem S = carve<kM>(smem_raw);
    int* err = uf.err;
    const int n_dense = *w.n_dense;
    for (int it = blockIdx.x; it < n_dense; it += gridDim.x) {
        const int64_t key = w.dense_list[it];
        const int c0 = w.cell_start[key], c1 = w.cell_start[key + 1];
        const int m = c1 - c0;
        if (m <= kLo || m > kM)
            continue;                             // the other size class's cell (block-uniform)
        const BoxDev& b = g.boxes[box_of(g.box_p0, g.nbox, c0)];
        const int q = b.q;
        const float4 p0 = w.sorted[c0];
        const int cx = cell_coord(p0.x, b), cy = cell_coord(p0.y, b), cz = cell_coord(p0.z, b);
        const int ox = cx * q, oy = cy * q, oz = cz * q;
        const int ua = w.dense_root[c0 / dense_min];
        // the 13 forward neighbours that are subdivided and not yet joined
        if (threadIdx.x < 32) {
            int k = threadIdx.x;
            int cnt = 0;
            if (k < 13) {
                int dx, dy, dz;
                fwd_offset(k, dx, dy, dz);
                int64_t nk = nbr_cell(b, cx, cy, cz, dx, dy, dz);
                int j0 = w.cell_start[nk], j1 = w.cell_start[nk + 1];
                int both = 0;
                if (is_sub(j1 - j0, b, dense_min) && !is_big(j1 - j0, b)) {
                    int ub = w.dense_root[j0 / dense_min];
                    both = ua >= 0 && ub >= 0;
                    cnt = (both && ufind<kVar>(w.parent, ua, uf) == ufind<kVar>(w.parent, ub, uf)) ? 0 : j1 - j0;
                }
                S.nbj0[k] = j0;
                S.nbflag[k] = both;
                S.nbdone[k] = 0;
            }
            int x = cnt;
            for (int o = 1; o < 32; o <<= 1) {
                int y = __shfl_up_sync(kFull, x, o);
                if (k >= o) x += y;
            }
            if (k < 13) S.nbpref[k + 1] = x;
            if (k == 0) S.nbpref[0] = 0;
        }
        __syncthreads();
        const int total = S.nbpref[13];
        __syncthreads();                          // everyone has read the table's total
        if (total == 0)
            continue;                             // block-uniform
        build_cell(S, w.sorted, c0, m, b, ox, oy, oz, err);
        for (int a = threadIdx.x; a < q * q * q; a += blockDim.x)
            if (S.sstart[a + 1] > S.sstart[a])
                S.groot[a] = ufind<kVar>(w.parent, c0 + S.order[S.sstart[a]], uf);
        __syncthreads();
        for (int t = threadIdx.x; t < total; t += blockDim.x) {
            int lo = 0, hi = 12;
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (S.nbpref[mid] <= t) lo = mid; else hi = mid - 1;
            }
            const int k = lo;
            const bool single = S.nbflag[k] != 0;
            if (single && *(volatile int*)(S.nbdone + k))
                continue;                         // the two cells are joined already
            int j = S.nbj0[k] + (t - S.nbpref[k]);
            FOF_DCHECK_SLOT(j, b, err);
            float4 pj = w.sorted[j];
            int rx, ry, rz;
            if (!rel_fine(pj, b, ox, oy, oz, rx, ry, rz))
                continue;
            int rj = ufind<kVar>(w.parent, j, uf);
            bool any = false;
            link_window<kVar>(S, w.parent, b, pj, rj, rx, ry, rz, single, uf, any);
            if (any && single)
                S.nbdone[k] = 1;
        }
        __syncthreads();
    }
}

}  // namespace

size_t dense_smem()
{
    return dense_smem_bytes<kDenseMax>();
}

template <bool kVar, int kLo, int kM, int kThreads, int kBlocks>
cudaError_t configure_dense()
{
    cudaError_t e = cudaFuncSetAttribute(k_dense_self<kVar, kLo, kM, kThreads, kBlocks>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dense_smem_bytes<kM>());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_dense_pairs<kVar, kLo, kM, kThreads, kBlocks>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dense_smem_bytes<kM>());
}

template <bool kVar, int kLo, int kM, int kThreads, int kBlocks>
void run_dense(const Geometry& g, const Work& w, int dense_min, const UfArgs& uf, bool pairs, cudaStream_t s)
{
    const int blocks = sm_count() * kBlocks;
    if (pairs)
        k_dense_pairs<kVar, kLo, kM, kThreads, kBlocks><<<blocks, kThreads, dense_smem_bytes<kM>(), s>>>(
            g, w, dense_min, uf);
    else
        k_dense_self<kVar, kLo, kM, kThreads, kBlocks><<<blocks, kThreads, dense_smem_bytes<kM>(), s>>>(
            g, w, dense_min, uf);
}

cudaError_t launch_dense(const Geometry& g, const Work& w, int dense_min, const UfArgs& uf, bool pairs,
                         cudaStream_t s)
{
    // the shared-memory opt-in is per device; setting it again is harmless
    static bool configured[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64 || !configured[dev]) {
        if ((e = configure_dense<false, 0, kDenseSmall, 256, 6>()) != cudaSuccess) return e;
        if ((e = configure_dense<false, kDenseSmall, kDenseMax, 512, 2>()) != cudaSuccess) return e;
        if ((e = configure_dense<true, 0, kDenseSmall, 256, 6>()) != cudaSuccess) return e;
        if ((e = configure_dense<true, kDenseSmall, kDenseMax, 512, 2>()) != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) configured[dev] = true;
    }
    if (uf.var) {
        run_dense<true, 0, kDenseSmall, 256, 6>(g, w, dense_min, uf, pairs, s);
        run_dense<true, kDenseSmall, kDenseMax, 512, 2>(g, w, dense_min, uf, pairs, s);
    } else {
        run_dense<false, 0, kDenseSmall, 256, 6>(g, w, dense_min, uf, pairs, s);
        run_dense<false, kDenseSmall, kDenseMax, 512, 2>(g, w, dense_min, uf, pairs, s);
    }
    return cudaGetLastError();
}

}  // namespace fofgpu
