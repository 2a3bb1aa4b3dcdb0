// Big cells: subdivided cells with more than kDenseMax particles, too many
// to stage in shared memory.  They get the same sub-cell method as the dense
// cells (fof_dense.cu) with the particles kept in global memory:
//   * every two particles of one sub-cell (side <= l_x / sqrt(3) with the
//     index margins of setup_box) are linked, so a sub-cell is a clique;
//   * a linked pair lies at most 2 sub-cells apart on each axis.
// So the work per particle stays bounded by the occupancy of a 5^3 window of
// sub-cells, whatever the size of the cell, instead of growing with it.
//
//   big_sort   one CTA per big cell, before the dense kernels: the cell's
//              slots are sorted by sub-cell (counting sort through the
//              brick-order buffer, which is free once binning is done), each
//              particle's parent is set to the first slot of its sub-cell
//              (the smallest, as union by root onto the lower offset gives),
//              and every pair of non-empty sub-cells within the half +-2
//              stencil is joined at its first linked pair (the paper's self
//              task, Sec. 3.1).
//   big_pairs  one CTA per big cell, after the dense kernels (every cell's
//              slot order is final then): each particle of the 26 neighbour
//              cells -- all of them that are not big, and the big ones among
//              the 13 forward neighbours, so each big pair is done once -- is
//              linked against the sub-cells of its +-2 window (pair tasks).
#include "fof_internal.cuh"

namespace fofgpu {

namespace {

constexpr int kBigThreads = 512;

struct BigSmem {
    int start[kMaxQ3 + 1];     // sub-cell starts (slot offsets in the cell)
    int cur[kMaxQ3];           // scatter cursors / sub-cell root snapshots
    unsigned rowmask[kMaxQ * kMaxQ];
    unsigned short ne[kMaxQ3]; // non-empty sub-cells
    int n_ne;
    int nbj0[26];              // neighbour cell ranges (big_pairs)
    int nbpref[27];
};

__device__ __forceinline__ int sub_key(const float4& p, const BoxDev& b, int ox, int oy, int oz, int* err)
{
    const int q = b.q;
    int sx = fine_coord(p.x, b) - ox, sy = fine_coord(p.y, b) - oy, sz = fine_coord(p.z, b) - oz;
    if (sx < 0 || sx >= q || sy < 0 || sy >= q || sz < 0 || sz >= q) {
        atomicOr(err, kErrInternal);
        sx = min(max(sx, 0), q - 1);
        sy = min(max(sy, 0), q - 1);
        sz = min(max(sz, 0), q - 1);
    }
    return (sz * q + sy) * q + sx;
}

// Exclusive scan of S.start[0..q3] in place by warp 0, then the row masks
// and the list of non-empty sub-cells.
__device__ __forceinline__ void finish_starts(BigSmem& S, int q)
{
    const int q3 = q * q * q;
    if (threadIdx.x < 32) {
        int carry = 0;
        for (int base = 0; base <= q3; base += 32) {
            const int i = base + threadIdx.x;
            const int v = i <= q3 ? S.start[i] : 0;
            int x = v;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(kFull, x, o);
                if ((int)threadIdx.x >= o) x += y;
            }
            if (i <= q3) S.start[i] = carry + x - v;
            carry += __shfl_sync(kFull, x, 31);
        }
    }
    if (threadIdx.x == 0)
        S.n_ne = 0;
    __syncthreads();
    for (int a = threadIdx.x; a < q3; a += blockDim.x)
        if (S.start[a + 1] > S.start[a])
            S.ne[atomicAdd(&S.n_ne, 1)] = (unsigned short)a;
    for (int row = threadIdx.x; row < q * q; row += blockDim.x) {
        unsigned m = 0;
        for (int x = 0; x < q; ++x)
            m |= (unsigned)(S.start[row * q + x + 1] > S.start[row * q + x]) << x;
        S.rowmask[row] = m;
    }
    __syncthreads();
}

// Cell key and fine corner of a big cell from its first particle.
__device__ __forceinline__ void big_cell(const Work& w, int64_t key, const BoxDev& b, int c0, int& cx, int& cy,
                                         int& cz)
{
    const float4 p0 = w.sorted[c0];
    cx = cell_coord(p0.x, b);
    cy = cell_coord(p0.y, b);
    cz = cell_coord(p0.z, b);
}

template <bool kVar>
__global__ void __launch_bounds__(kBigThreads) k_big_sort(Geometry g, Work w, UfArgs uf)
{
    __shared__ BigSmem S;
    const int n_big = *w.n_big;
    for (int it = blockIdx.x; it < n_big; it += gridDim.x) {
        const int64_t key = w.big_list[it];
        const int c0 = w.cell_start[key], c1 = w.cell_start[key + 1];
        const int m = c1 - c0;
        const BoxDev& b = g.boxes[box_of(g.box_p0, g.nbox, c0)];
        const int q = b.q, q3 = q * q * q;
        int cx, cy, cz;
        big_cell(w, key, b, c0, cx, cy, cz);
        const int ox = cx * q, oy = cy * q, oz = cz * q;
        for (int a = threadIdx.x; a <= q3; a += blockDim.x) S.start[a] = 0;
        __syncthreads();
        for (int k = threadIdx.x; k < m; k += blockDim.x)
            atomicAdd(&S.start[sub_key(w.sorted[c0 + k], b, ox, oy, oz, uf.err)], 1);
        __syncthreads();
        finish_starts(S, q);
        for (int a = threadIdx.x; a < q3; a += blockDim.x) S.cur[a] = S.start[a];
        __syncthreads();
        // counting sort by sub-cell through the brick-order buffer
        for (int k = threadIdx.x; k < m; k += blockDim.x) {
            const float4 p = w.sorted[c0 + k];
            const int at = atomicAdd(&S.cur[sub_key(p, b, ox, oy, oz, uf.err)], 1);
            w.tmp[c0 + at] = p;
        }
        __syncthreads();
        // back in place; every particle hangs on the first slot of its sub-cell
        for (int k = threadIdx.x; k < m; k += blockDim.x) {
            const float4 p = w.tmp[c0 + k];
            w.sorted[c0 + k] = p;
            w.minorig[c0 + k] = __float_as_int(p.w);
            const int a = sub_key(p, b, ox, oy, oz, uf.err);
            w.parent[c0 + k] = c0 + S.start[a];
        }
        __syncthreads();
        // pairs of sub-cells inside the cell: the 62 offsets of the half
        // +-2 stencil, as 13 rows (dz, dy) of a dx span
        for (int item = threadIdx.x; item < S.n_ne * 13; item += blockDim.x) {
            const int a = S.ne[item / 13];
            const int o = item % 13;
            const int ax = a % q, ay = (a / q) % q, az = a / (q * q);
            int dy, dz, dxlo, dxhi;
            if (o < 10) {
                dz = 1 + o / 5; dy = o % 5 - 2; dxlo = -2; dxhi = 2;
            } else if (o < 12) {
                dz = 0; dy = o - 9; dxlo = -2; dxhi = 2;
            } else {
                dz = 0; dy = 0; dxlo = 1; dxhi = 2;
            }
            const int by = ay + dy, bz = az + dz;
            if (by < 0 || by >= q || bz >= q)
                continue;
            const int xlo = max(ax + dxlo, 0), xhi = min(ax + dxhi, q - 1);
            if (xlo > xhi)
                continue;
            unsigned bits = S.rowmask[bz * q + by] & ((2u << xhi) - (1u << xlo));
            const int a0 = S.start[a], a1 = S.start[a + 1];
            while (bits) {
                const int bx = __ffs(bits) - 1;
                bits &= bits - 1u;
                const int bb = (bz * q + by) * q + bx;
                const int b0 = S.start[bb], b1 = S.start[bb + 1];
                int ra = ufind<kVar>(w.parent, c0 + a0, uf);
                const int rb = ufind<kVar>(w.parent, c0 + b0, uf);
                if (ra == rb)
                    continue;
                bool done = false;
                for (int u = a0; u < a1 && !done; ++u) {
                    const float4 pu = w.sorted[c0 + u];
                    for (int v = b0; v < b1; ++v)
                        if (linked_ool(pu, w.sorted[c0 + v], b)) {
                            uunion<kVar>(w.parent, ra, rb, uf);
                            done = true;
                            break;
                        }
                }
            }
        }
        __syncthreads();
    }
}

template <bool kVar>
__global__ void __launch_bounds__(kBigThreads) k_big_pairs(Geometry g, Work w, int dense_min, UfArgs uf)
{
    __shared__ BigSmem S;
    const int n_big = *w.n_big;
    for (int it = blockIdx.x; it < n_big; it += gridDim.x) {
        const int64_t key = w.big_list[it];
        const int c0 = w.cell_start[key], c1 = w.cell_start[key + 1];
        const int m = c1 - c0;
        const BoxDev& b = g.boxes[box_of(g.box_p0, g.nbox, c0)];
        const int q = b.q, q3 = q * q * q;
        int cx, cy, cz;
        big_cell(w, key, b, c0, cx, cy, cz);
        const int ox = cx * q, oy = cy * q, oz = cz * q;
        // sub-cell starts again (the slots are in sub-cell order)
        for (int a = threadIdx.x; a <= q3; a += blockDim.x) S.start[a] = 0;
        if (threadIdx.x < 26) {
            const int k = threadIdx.x;
            const int code = k < 13 ? k : k + 1;          // the 26 offsets, centre skipped
            const int dx = code % 3 - 1, dy = (code / 3) % 3 - 1, dz = code / 9 - 1;
            const int64_t nk = cell_key(b, wrap_cell(cx + dx, b.nc), wrap_cell(cy + dy, b.nc),
                                        wrap_cell(cz + dz, b.nc));
            const int j0 = w.cell_start[nk], j1 = w.cell_start[nk + 1];
            // forward in the order of the 27-cell code: dz > 0, or dz == 0 and
            // (dy > 0, or dy == 0 and dx > 0)
            const bool forward = code > 13;
            const bool take = j1 > j0 && (!is_big(j1 - j0, b) || forward) && nk != key;
            S.nbj0[k] = j0;
            S.nbpref[k + 1] = take ? j1 - j0 : 0;
        }
        __syncthreads();
        for (int k = threadIdx.x; k < m; k += blockDim.x)
            atomicAdd(&S.start[sub_key(w.sorted[c0 + k], b, ox, oy, oz, uf.err)], 1);
        if (threadIdx.x < 32) {
            const int lane = threadIdx.x;
            const int v = (lane >= 1 && lane <= 26) ? S.nbpref[lane] : 0;
            int x = v;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(kFull, x, o);
                if (lane >= o) x += y;
            }
            if (lane <= 26) S.nbpref[lane] = x;
        }
        __syncthreads();
        finish_starts(S, q);
        for (int t = threadIdx.x; t < S.n_ne; t += blockDim.x) {
            const int a = S.ne[t];
            S.cur[a] = ufind<kVar>(w.parent, c0 + S.start[a], uf);   // root snapshot
        }
        __syncthreads();
        const int total = S.nbpref[26];
        for (int t = threadIdx.x; t < total; t += blockDim.x) {
            int lo = 0, hi = 25;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (S.nbpref[mid] <= t) lo = mid; else hi = mid - 1;
            }
            int j = S.nbj0[lo] + (t - S.nbpref[lo]);
            FOF_DCHECK_SLOT(j, b, uf.err);
            const float4 pj = w.sorted[j];
            // pj's fine coordinates relative to the cell corner, unwrapped
            const int nf = b.nf;
            int rx = fine_coord(pj.x, b) - ox, ry = fine_coord(pj.y, b) - oy, rz = fine_coord(pj.z, b) - oz;
            rx = rx < -2 ? rx + nf : (rx > q + 1 ? rx - nf : rx);
            ry = ry < -2 ? ry + nf : (ry > q + 1 ? ry - nf : ry);
            rz = rz < -2 ? rz + nf : (rz > q + 1 ? rz - nf : rz);
            if (rx < -2 || rx > q + 1 || ry < -2 || ry > q + 1 || rz < -2 || rz > q + 1)
                continue;
            int rj = ufind<kVar>(w.parent, j, uf);
            const int x0 = max(rx - 2, 0), x1 = min(rx + 2, q - 1);
            const int y0 = max(ry - 2, 0), y1 = min(ry + 2, q - 1);
            const int z0 = max(rz - 2, 0), z1 = min(rz + 2, q - 1);
            if (x0 > x1 || y0 > y1 || z0 > z1)
                continue;
            const float ux = __fmul_rn(pj.x, b.inv_hf) - (float)fine_coord(pj.x, b);
            const float uy = __fmul_rn(pj.y, b.inv_hf) - (float)fine_coord(pj.y, b);
            const float uz = __fmul_rn(pj.z, b.inv_hf) - (float)fine_coord(pj.z, b);
            const unsigned span = (2u << x1) - (1u << x0);
            for (int z = z0; z <= z1; ++z) {
                const float gz = z < rz ? (float)(rz - z - 1) + uz : (z > rz ? (float)(z - rz - 1) + (1.f - uz) : 0.f);
                for (int y = y0; y <= y1; ++y) {
                    const float gy = y < ry ? (float)(ry - y - 1) + uy : (y > ry ? (float)(y - ry - 1) + (1.f - uy) : 0.f);
                    unsigned bits = S.rowmask[z * q + y] & span;
                    while (bits) {
                        const int x = __ffs(bits) - 1;
                        bits &= bits - 1u;
                        const float gx = x < rx ? (float)(rx - x - 1) + ux : (x > rx ? (float)(x - rx - 1) + (1.f - ux) : 0.f);
                        if (gx * gx + gy * gy + gz * gz > b.reach2)
                            continue;                // the whole sub-cell is out of reach
                        const int a = (z * q + y) * q + x;
                        if (S.cur[a] == rj)
                            continue;
                        for (int u = S.start[a]; u < S.start[a + 1]; ++u)
                            if (linked_ool(pj, w.sorted[c0 + u], b)) {
                                rj = uunion<kVar>(w.parent, rj, S.cur[a], uf);
                                break;
                            }
                    }
                }
            }
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_big(const Geometry& g, const Work& w, int dense_min, const UfArgs& uf, bool pairs,
                       cudaStream_t s)
{
    if (g.total_n == 0)
        return cudaSuccess;
    const int blocks = sm_count() * 2;
    const bool var = uf.var != 0;
    if (pairs) {
        if (var)
            k_big_pairs<true><<<blocks, kBigThreads, 0, s>>>(g, w, dense_min, uf);
        else
            k_big_pairs<false><<<blocks, kBigThreads, 0, s>>>(g, w, dense_min, uf);
    } else {
        if (var)
            k_big_sort<true><<<blocks, kBigThreads, 0, s>>>(g, w, uf);
        else
            k_big_sort<false><<<blocks, kBigThreads, 0, s>>>(g, w, uf);
    }
    return cudaGetLastError();
}

}  // namespace fofgpu
