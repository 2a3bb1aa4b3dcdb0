// Binning: a two-level counting sort of the particles into cells of side
// >= l_x (the paper matches tree-node size to the linking length for the
// neighbour search, Sec. 3.1; here the tree is a uniform periodic grid).
//
//   bin_count    validate every coordinate, histogram of bricks
//   scan         exclusive prefix sum of the brick counts
//   bin_scatter  each particle to its brick (float4: x, y, z, local index)
//   brick_sort   one CTA per brick: cell histogram and scan in shared
//                memory, scatter into cell order, cell_start of the brick,
//                and the forest initialisation parent[s] = s (Sec. 3.1)
//
// Bricks exist so that both atomics (brick cursors) and the scattered
// writes stay in L2: the brick count is small enough that every brick's
// write head is L2-resident, which turns the random-order scatter into
// full-sector DRAM writes.
#include "fof_internal.cuh"

namespace fofgpu {

namespace {

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ bool coord_ok(float x, float xmax)
{
    return x >= 0.0f && x <= xmax;     // false for NaN
}

// brick of particle i (concatenated brick index) and its float4 record
__device__ __forceinline__ int64_t brick_of(const float* __restrict__ pos, int64_t i,
                                            const BoxDev& b, float4& rec, bool& ok)
{
    float x = __ldg(pos + 3 * i);
    float y = __ldg(pos + 3 * i + 1);
    float z = __ldg(pos + 3 * i + 2);
    ok = coord_ok(x, b.xmax) && coord_ok(y, b.xmax) && coord_ok(z, b.xmax);
    rec = make_float4(x, y, z, __int_as_float((int)(i - b.p0)));
    return b.brick0 + brick_local(b, cell_coord(x, b), cell_coord(y, b), cell_coord(z, b));
}

__global__ void __launch_bounds__(256) k_bin_count(const float* __restrict__ pos, Geometry g,
                                                   int* __restrict__ bcount, int* __restrict__ err)
{
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int bad = 0;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < g.total_n; base += stride) {
        int64_t i = base + threadIdx.x;
        bool valid = i < g.total_n;
        unsigned active = __ballot_sync(kFull, valid);
        if (!valid)
            continue;
        const BoxDev& b = g.boxes[box_of(g.box_p0, g.nbox, i)];
        float4 rec;
        bool ok;
        int64_t brick = brick_of(pos, i, b, rec, ok);
        bad |= !ok;
        // brick indices fit in 31 bits (checked when the plan is made); the
        // 32-bit match is much cheaper than the 64-bit one
        unsigned peers = __match_any_sync(active, (int)brick);
        int leader = __ffs(peers) - 1;
        if (lane == leader)
            atomicAdd(bcount + brick, __popc(peers));
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0)
        atomicOr(err, kErrRange);
}

__global__ void __launch_bounds__(256) k_bin_scatter(const float* __restrict__ pos, Geometry g,
                                                     const int* __restrict__ bstart,
                                                     int* __restrict__ bcursor,
                                                     float4* __restrict__ tmp, int* __restrict__ err)
{
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < g.total_n; base += stride) {
        int64_t i = base + threadIdx.x;
        bool valid = i < g.total_n;
        unsigned active = __ballot_sync(kFull, valid);
        if (!valid)
            continue;
        const BoxDev& b = g.boxes[box_of(g.box_p0, g.nbox, i)];
        float4 rec;
        bool ok;
        int64_t brick = brick_of(pos, i, b, rec, ok);
        unsigned peers = __match_any_sync(active, (int)brick);
        int leader = __ffs(peers) - 1;
        int rank = __popc(peers & lanemask_lt());
        int off = 0;
        if (lane == leader)
            off = atomicAdd(bcursor + brick, __popc(peers));
        off = __shfl_sync(active, off, leader);
        int64_t slot = (int64_t)__ldg(bstart + brick) + off + rank;
        if (slot < __ldg(bstart + brick + 1))
            tmp[slot] = rec;
        else
            atomicOr(err, kErrInternal);
    }
}

// ------------------------------------------------------------------------
// device-wide exclusive scan (reduce, scan of partials, apply)
// ------------------------------------------------------------------------

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;   // 2048

__device__ __forceinline__ int block_exclusive_scan(int v, int* smem_warp, int& total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int nw = blockDim.x >> 5;
        int t = lane < nw ? smem_warp[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(kFull, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) smem_warp[lane] = t;   // inclusive warp totals
    }
    __syncthreads();
    int warp_off = wid ? smem_warp[wid - 1] : 0;
    total = smem_warp[(blockDim.x >> 5) - 1];
    __syncthreads();
    return warp_off + x - v;
}

// The same for 64-bit words (fields that never carry into each other).
__device__ __forceinline__ unsigned long long block_exclusive_scan64(unsigned long long v,
                                                                     unsigned long long* smem_warp,
                                                                     unsigned long long& total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) smem_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        unsigned long long t = lane < nw ? smem_warp[lane] : 0ull;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(kFull, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) smem_warp[lane] = t;
    }
    __syncthreads();
    const unsigned long long warp_off = wid ? smem_warp[wid - 1] : 0ull;
    total = smem_warp[(blockDim.x >> 5) - 1];
    __syncthreads();
    return warp_off + x - v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const int* __restrict__ in, int64_t len,
                                                              int* __restrict__ part)
{
    __shared__ int sw[32];
    int64_t base = (int64_t)blockIdx.x * kScanTile;
    int s = 0;
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + (int64_t)k * kScanThreads + threadIdx.x;
        if (i < len) s += in[i];
    }
    int total;
    block_exclusive_scan(s, sw, total);
    if (threadIdx.x == 0) part[blockIdx.x] = total;
}

// single block, exclusive scan of part[0..m) in place, m arbitrary
__global__ void __launch_bounds__(1024) k_scan_partials(int* __restrict__ part, int64_t m)
{
    __shared__ int sw[32];
    int carry = 0;
    for (int64_t base = 0; base < m; base += blockDim.x) {
        int64_t i = base + threadIdx.x;
        int v = i < m ? part[i] : 0;
        int total;
        int ex = block_exclusive_scan(v, sw, total);
        if (i < m) part[i] = carry + ex;
        carry += total;
    }
}

// out[i] for i in [0, len]: out[len] is the grand total (a virtual zero is
// appended to the input, so the scan covers len + 1 entries)
__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const int* __restrict__ in, int* __restrict__ out,
                                                             int64_t len, const int* __restrict__ part)
{
    __shared__ int sw[32];
    int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int v[kScanItems];
    int s = 0;
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        v[k] = i < len ? in[i] : 0;
        s += v[k];
    }
    int total;
    int ex = block_exclusive_scan(s, sw, total) + part[blockIdx.x];
    for (int k = 0; k < kScanItems; ++k) {
        int64_t i = base + k;
        if (i <= len) out[i] = ex;
        ex += v[k];
    }
}

// ------------------------------------------------------------------------
// per-brick cell sort
// ------------------------------------------------------------------------

constexpr int kSortThreads = 1024;
constexpr int kMaxR3 = 4096;   // r <= 16

__global__ void __launch_bounds__(kSortThreads) k_brick_sort(Geometry g, const float4* __restrict__ tmp,
                                                             const int* __restrict__ bstart,
                                                             float4* __restrict__ sorted,
                                                             int* __restrict__ parent,
                                                             int* __restrict__ minorig,
                                                             int* __restrict__ cnt,
                                                             int* __restrict__ cell_start,
                                                             int* __restrict__ err,
                                                             int64_t* __restrict__ dense_list,
                                                             int* __restrict__ n_dense,
                                                             int dense_min,
                                                             int64_t* __restrict__ team_list,
                                                             int* __restrict__ n_team,
                                                             int* __restrict__ n_team_hi,
                                                             int64_t team_cap,
                                                             int64_t* __restrict__ big_list,
                                                             int* __restrict__ n_big)
{
    __shared__ int hist[kMaxR3];
    __shared__ int sw[32];
    __shared__ unsigned long long sw64[32];
    __shared__ int list_base[4];
    for (int64_t gb = blockIdx.x; gb < g.total_bricks; gb += gridDim.x) {
        const int bi = box_of(g.box_brick0, g.nbox, gb);
        const BoxDev& b = g.boxes[bi];
        const int r3 = b.r * b.r * b.r;
        const int m = b.r - 1;
        const int s0 = bstart[gb], s1 = bstart[gb + 1];
        for (int c = threadIdx.x; c < r3; c += blockDim.x) hist[c] = 0;
        __syncthreads();
        for (int k = s0 + threadIdx.x; k < s1; k += blockDim.x) {
            float4 p = tmp[k];
            int lc = local_code(cell_coord(p.x, b) & m, cell_coord(p.y, b) & m, cell_coord(p.z, b) & m);
            atomicAdd(hist + lc, 1);
        }
        __syncthreads();
        // exclusive scan of hist[0..r3): each thread owns a contiguous run
        const int per = (r3 + blockDim.x - 1) / blockDim.x;
        const int c0 = threadIdx.x * per;
        int run = 0;
        for (int c = c0; c < c0 + per && c < r3; ++c) run += hist[c];
        int total;
        int ex = block_exclusive_scan(run, sw, total);
        const int ex0 = ex;
        const int64_t cbase = b.cell0 + (gb - b.brick0) * (int64_t)r3;
        int nd = 0, nt = 0, nth = 0, nbg = 0;   // this thread's dense, team (small, large) and big cells
        for (int c = c0; c < c0 + per && c < r3; ++c) {
            const int h = hist[c];
            ex += h;
            if (is_big(h, b))
                ++nbg;
            else if (is_sub(h, b, dense_min))
                ++nd;
            else if (h >= b.team_min && h <= kTeamSplit)
                ++nt;
            else if (h >= b.team_min && h <= kTeamSelfMax)
                ++nth;
        }
        // list slots: one reservation per brick (a shared counter per cell
        // would serialise millions of atomics on one address).  The four
        // counts (each at most kMaxR3 per brick) share one scan as 16-bit
        // fields of a 64-bit word.
        unsigned long long tot4;
        const unsigned long long o4 = block_exclusive_scan64(
            (unsigned long long)nd | ((unsigned long long)nt << 16) | ((unsigned long long)nth << 32) |
                ((unsigned long long)nbg << 48),
            sw64, tot4);
        const int nd_tot = (int)(tot4 & 0xffffu), nt_tot = (int)((tot4 >> 16) & 0xffffu);
        const int nth_tot = (int)((tot4 >> 32) & 0xffffu), nb_tot = (int)(tot4 >> 48);
        int od = (int)(o4 & 0xffffu), ot = (int)((o4 >> 16) & 0xffffu);
        int oth = (int)((o4 >> 32) & 0xffffu), obg = (int)(o4 >> 48);
        if (threadIdx.x == 0) {
            list_base[0] = nd_tot ? atomicAdd(n_dense, nd_tot) : 0;
            list_base[1] = nt_tot ? atomicAdd(n_team, nt_tot) : 0;
            list_base[2] = nb_tot ? atomicAdd(n_big, nb_tot) : 0;
            list_base[3] = nth_tot ? atomicAdd(n_team_hi, nth_tot) : 0;
        }
        __syncthreads();
        od += list_base[0];
        ot += list_base[1];
        obg += list_base[2];
        oth += list_base[3];
        ex = ex0;
        for (int c = c0; c < c0 + per && c < r3; ++c) {
            const int h = hist[c];
            const int start = s0 + ex;
            hist[c] = ex;                       // becomes the cursor
            ex += h;
            if (is_big(h, b))
                big_list[obg++] = cbase + c;
            else if (is_sub(h, b, dense_min))
                dense_list[od++] = cbase + c;
            else if (h >= b.team_min && h <= kTeamSplit)
                team_list[ot++] = ((int64_t)h << 32) | (uint32_t)start;
            else if (h >= b.team_min && h <= kTeamSelfMax)
                team_list[team_cap - 1 - oth++] = ((int64_t)h << 32) | (uint32_t)start;
        }
        __syncthreads();
        for (int k = s0 + threadIdx.x; k < s1; k += blockDim.x) {
            float4 p = tmp[k];
            int lc = local_code(cell_coord(p.x, b) & m, cell_coord(p.y, b) & m, cell_coord(p.z, b) & m);
            int slot = s0 + atomicAdd(hist + lc, 1);
            if (slot >= s1) {
                atomicOr(err, kErrInternal);
                continue;
            }
            sorted[slot] = p;
            minorig[slot] = __float_as_int(p.w);
        }
        for (int k = s0 + threadIdx.x; k < s1; k += blockDim.x) {
            parent[k] = k;
            cnt[k] = 1;
        }
        // the cursors now hold each cell's end: the cell starts, written
        // coalesced (cell c + 1 starts where c ends; the next brick writes
        // the same value at its first cell)
        __syncthreads();
        for (int c = threadIdx.x; c < r3; c += blockDim.x)
            cell_start[cbase + c + 1] = s0 + hist[c];
        if (threadIdx.x == 0)
            cell_start[cbase] = s0;
        __syncthreads();
    }
}

// ------------------------------------------------------------------------
// incremental re-binning (the group finder run again on moved particles)
// ------------------------------------------------------------------------

// For every binned slot s of the previous run: the particle's new position
// (pos[p0 + local index]) replaces its old one in sorted[s] and tmp[s], and
// flags record whether it left its cell (bit 0) or its brick (bit 1).  When
// no particle left its brick, the slots are still grouped by brick, so
// tmp[] is a valid brick-order array for k_brick_sort; when no particle left
// its cell, sorted[] and the cell starts and lists are valid as they are.
__global__ void __launch_bounds__(256) k_relink_check(const float* __restrict__ pos, Geometry g,
                                                      float4* __restrict__ sorted, float4* __restrict__ tmp,
                                                      int* __restrict__ flags, int* __restrict__ err)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int f = 0, bad = 0;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < g.total_n; s += stride) {
        const BoxDev& b = g.boxes[box_of(g.box_p0, g.nbox, s)];
        const float4 old = sorted[s];
        const int o = __float_as_int(old.w);
        const int64_t i = b.p0 + o;
        float4 rec;
        bool ok;
        const int64_t nb = brick_of(pos, i, b, rec, ok);
        bad |= !ok;
        const int ox = cell_coord(old.x, b), oy = cell_coord(old.y, b), oz = cell_coord(old.z, b);
        const int nx = cell_coord(rec.x, b), ny = cell_coord(rec.y, b), nz = cell_coord(rec.z, b);
        if (nx != ox || ny != oy || nz != oz)
            f |= 1;
        if (nb != b.brick0 + brick_local(b, ox, oy, oz))
            f |= 2;
        sorted[s] = rec;
        tmp[s] = rec;
    }
    f = __reduce_or_sync(kFull, f);
    if ((threadIdx.x & 31) == 0 && f)
        atomicOr(flags, f);
    if (__syncthreads_or(bad) && threadIdx.x == 0)
        atomicOr(err, kErrRange);
}

// Forest and label initialisation of the binned slots (what k_brick_sort
// does while it sorts): parent[s] = s, cnt[s] = 1, minorig[s] = local index.
__global__ void __launch_bounds__(256) k_forest_init(int64_t total, const float4* __restrict__ sorted,
                                                     int* __restrict__ parent, int* __restrict__ minorig,
                                                     int* __restrict__ cnt)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < total; s += stride) {
        parent[s] = (int)s;
        cnt[s] = 1;
        minorig[s] = __float_as_int(sorted[s].w);
    }
}

}  // namespace

// ------------------------------------------------------------------------
// launchers
// ------------------------------------------------------------------------

static int grid_for(int64_t items, int threads, int per_sm)
{
    int64_t want = (items + threads - 1) / threads;
    int64_t cap = (int64_t)sm_count() * per_sm;
    if (want < 1) want = 1;
    return (int)(want < cap ? want : cap);
}

cudaError_t launch_bin_count(const float* pos, const Geometry& g, const Work& w, cudaStream_t s)
{
    if (g.total_n == 0)
        return cudaSuccess;
    k_bin_count<<<grid_for(g.total_n, 256, 8), 256, 0, s>>>(pos, g, w.bcount, &w.status->err);
    return cudaGetLastError();
}

int64_t scan_tmp_elems(int64_t len)
{
    return (len + 1 + kScanTile - 1) / kScanTile + 1;
}

cudaError_t launch_scan(const int* in, int* out, int64_t len, int* tmp, int64_t tmp_len, cudaStream_t s)
{
    int64_t blocks = (len + 1 + kScanTile - 1) / kScanTile;   // len + 1 outputs
    if (blocks + 1 > tmp_len)
        return cudaErrorInvalidValue;
    k_scan_reduce<<<(unsigned)blocks, kScanThreads, 0, s>>>(in, len, tmp);
    k_scan_partials<<<1, 1024, 0, s>>>(tmp, blocks);
    k_scan_apply<<<(unsigned)blocks, kScanThreads, 0, s>>>(in, out, len, tmp);
    return cudaGetLastError();
}

cudaError_t launch_bin_scatter(const float* pos, const Geometry& g, const Work& w, cudaStream_t s)
{
    if (g.total_n == 0)
        return cudaSuccess;
    k_bin_scatter<<<grid_for(g.total_n, 256, 8), 256, 0, s>>>(pos, g, w.bstart, w.bcursor, w.tmp,
                                                            &w.status->err);
    return cudaGetLastError();
}

cudaError_t launch_brick_sort(const Geometry& g, const Work& w, int dense_min, cudaStream_t s)
{
    if (g.total_bricks == 0)
        return cudaSuccess;
    int64_t blocks = g.total_bricks;
    int64_t cap = (int64_t)sm_count() * 4 * 16;
    if (blocks > cap) blocks = cap;
    k_brick_sort<<<(unsigned)blocks, kSortThreads, 0, s>>>(g, w.tmp, w.bstart, w.sorted, w.parent,
                                                         w.minorig, w.cnt, w.cell_start,
                                                         &w.status->err, w.dense_list, w.n_dense,
                                                         dense_min, w.team_list, w.n_team, w.n_team_hi,
                                                         w.team_cap, w.big_list, w.n_big);
    return cudaGetLastError();
}

cudaError_t launch_relink_check(const float* pos, const Geometry& g, const Work& w, int* flags,
                                cudaStream_t s)
{
    if (g.total_n == 0)
        return cudaSuccess;
    k_relink_check<<<grid_for(g.total_n, 256, 8), 256, 0, s>>>(pos, g, w.sorted, w.tmp, flags,
                                                             &w.status->err);
    return cudaGetLastError();
}

cudaError_t launch_forest_init(const Geometry& g, const Work& w, cudaStream_t s)
{
    if (g.total_n == 0)
        return cudaSuccess;
    k_forest_init<<<grid_for(g.total_n, 256, 8), 256, 0, s>>>(g.total_n, w.sorted, w.parent, w.minorig,
                                                             w.cnt);
    return cudaGetLastError();
}

}  // namespace fofgpu
