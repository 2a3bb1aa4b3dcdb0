// Flattening the forest into outputs.
//
//   finalize   full pointer jumping: parent[s] = root(s) for every slot; each
//              non-root adds itself to its root's size and offers its input
//              index to the root's minimum.  Roots were initialised with
//              size 1 and their own index, so they take part in no atomic:
//              the paper's early elimination of singletons (Sec. 3.4.2),
//              with the atomic additions of its parallel size count
//              (Sec. 3.4.1) aggregated per warp.
//   outputs    ids[i] = smallest index of i's group; sizes[label] = size,
//              0 elsewhere (two passes, see below); per-box group counts;
//              catalogue entries counted per label tile.
//   catalogue  prefix sum over the label tiles, then each tile writes its
//              (label, size) entries in ascending label order.
#include "fof_internal.cuh"

namespace fofgpu {

namespace {

// Root of slot s by a plain walk, then parent[s] = root.  `ordered`: every
// parent is at most its child (hooks onto the smaller root), checked.
__device__ __forceinline__ int final_root(int* __restrict__ parent, int s, bool ordered, int* err)
{
    const int p = parent[s];
    if (p == s)
        return s;
    int x = p;
    int q = parent[x];
    for (int step = 0; q != x; ++step) {
        if ((ordered && q > x) || step >= kFindCap) {   // corrupted forest: report
            atomicOr(err, kErrInternal);
            break;
        }
        x = q;
        q = parent[x];
    }
    if (p != x)
        parent[s] = x;
    return x;
}

__global__ void __launch_bounds__(256) k_finalize(int64_t total, int* __restrict__ parent,
                                                  int* __restrict__ minorig, int* __restrict__ cnt,
                                                  int* __restrict__ err, bool ordered)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < total; base += stride) {
        int64_t s = base + threadIdx.x;
        bool valid = s < total;
        unsigned active = __ballot_sync(kFull, valid);
        if (!valid)
            continue;
        const int root = final_root(parent, (int)s, ordered, err);
        bool nonroot = root != (int)s;
        unsigned nr = __ballot_sync(active, nonroot);
        if (!nonroot)
            continue;
        unsigned peers = __match_any_sync(nr, root);
        int leader = __ffs(peers) - 1;
        unsigned mn = __reduce_min_sync(peers, (unsigned)minorig[s]);
        if ((threadIdx.x & 31) == leader) {
            atomicAdd(cnt + root, __popc(peers));
            atomicMin(minorig + root, (int)mn);
        }
    }
}

// The same finalisation with the paper's hash-table size count (Sec. 3.4.1):
// each block gathers (root, count, smallest index) of the non-roots of
// kHashBatch consecutive slot tiles in an open-addressing table in shared
// memory, then adds each entry to the root with one atomic per entry (roots
// are not entered: their own contribution is the initial size 1, Sec.
// 3.4.2).  A slot whose probe sequence finds no room adds itself directly.
constexpr int kHashSlots = 4096;     // power of two
constexpr int kHashBatch = 8;        // tiles of 256 slots per flush: <= 2048 keys, load <= 1/2
constexpr int kHashProbes = 16;

__global__ void __launch_bounds__(256) k_finalize_hash(int64_t total, int* __restrict__ parent,
                                                       int* __restrict__ minorig, int* __restrict__ cnt,
                                                       int* __restrict__ err, bool ordered)
{
    __shared__ int hkey[kHashSlots];
    __shared__ int hcnt[kHashSlots];
    __shared__ int hmin[kHashSlots];
    for (int k = threadIdx.x; k < kHashSlots; k += blockDim.x)
        hkey[k] = -1;
    __syncthreads();
    const int64_t span = (int64_t)blockDim.x * kHashBatch;
    for (int64_t b0 = (int64_t)blockIdx.x * span; b0 < total; b0 += (int64_t)gridDim.x * span) {
        for (int t = 0; t < kHashBatch; ++t) {
            const int64_t s = b0 + (int64_t)t * blockDim.x + threadIdx.x;
            if (s >= total)
                break;
            const int root = final_root(parent, (int)s, ordered, err);
            if (root == (int)s)
                continue;
            const int mo = minorig[s];
            uint32_t h = uf_priority(root) & (kHashSlots - 1);
            bool placed = false;
            for (int probe = 0; probe < kHashProbes; ++probe, h = (h + 1) & (kHashSlots - 1)) {
                const int k = atomicCAS(&hkey[h], -1, root);
                if (k == -1 || k == root) {
                    if (k == -1) {            // the first insert initialises the entry
                        hcnt[h] = 0;
                        hmin[h] = INT_MAX;
                    }
                    placed = true;
                    break;
                }
            }
            if (!placed) {                    // no room on the probe path: add directly
                atomicAdd(cnt + root, 1);
                atomicMin(minorig + root, mo);
            }
            // entries are counted in the second pass, after every entry of
            // the batch has been initialised
        }
        __syncthreads();
        // second pass over the same slots: the table entries are initialised
        for (int t = 0; t < kHashBatch; ++t) {
            const int64_t s = b0 + (int64_t)t * blockDim.x + threadIdx.x;
            if (s >= total)
                break;
            const int root = parent[s];   // fully compressed by the first pass
            if (root == (int)s)
                continue;
            uint32_t h = uf_priority(root) & (kHashSlots - 1);
            for (int probe = 0; probe < kHashProbes; ++probe, h = (h + 1) & (kHashSlots - 1)) {
                if (hkey[h] == root) {
                    atomicAdd(&hcnt[h], 1);
                    atomicMin(&hmin[h], minorig[s]);
                    break;
                }
            }
        }
        __syncthreads();
        for (int k = threadIdx.x; k < kHashSlots; k += blockDim.x) {
            const int r = hkey[k];
            if (r >= 0) {
                atomicAdd(cnt + r, hcnt[k]);
                atomicMin(minorig + r, hmin[k]);
                hkey[k] = -1;
            }
        }
        __syncthreads();
    }
}

// Outputs go back to input order in two passes, so that no 4-byte value
// is written to a random address (a read-modify-write of a whole sector):
//   bucket  for every binned slot: label and size of its group, and one
//           (offset, value) pair appended to the bucket of its input index's
//           chunk of kOutChunk indices.  A chunk holds exactly kOutChunk
//           inputs (the last one fewer), so bucket c starts at c*kOutChunk
//           with no prefix sum, and the ~n/kOutChunk write heads stay in L2.
//   place   one CTA per chunk: the pairs are placed in shared memory and
//           ids and sizes written out coalesced.
// A pair is (offset | is_label << 31, value): value = size when the input
// is its group's label (then the label is the input's own box-local
// index), else the label.
__global__ void __launch_bounds__(256) k_outputs_bucket(Geometry g, const float4* __restrict__ sorted,
                                                        const int* __restrict__ parent,
                                                        const int* __restrict__ minorig,
                                                        const int* __restrict__ cnt, int32_t thr,
                                                        unsigned long long* __restrict__ n_groups,
                                                        unsigned long long* __restrict__ n_cat,
                                                        int* __restrict__ tile_cnt,
                                                        int* __restrict__ out_cursor,
                                                        int2* __restrict__ pairs, int* __restrict__ err)
{
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int acc_box = -1;                           // per-warp box counts not yet added
    unsigned long long acc_ng = 0, acc_nk = 0;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < g.total_n; base += stride) {
        int64_t s = base + threadIdx.x;
        bool valid = s < g.total_n;
        unsigned active = __ballot_sync(kFull, valid);
        if (!valid)
            continue;
        int bi = box_of(g.box_p0, g.nbox, s);
        int64_t p0 = g.boxes[bi].p0;
        // the input index o of slot s: minorig keeps it for every non-root
        // (the label pass only lowers roots' entries) and for singleton
        // roots; only a root of a larger group reads it from the binned record
        const int root = parent[s];
        const bool root_s = root == (int)s;
        int o, label, size;
        if (!root_s) {
            o = minorig[s];
            label = minorig[root];
            size = o == label ? cnt[root] : 0;
        } else {
            size = cnt[s];
            label = minorig[s];
            o = size == 1 ? label : __float_as_int(sorted[s].w);
        }
        const bool is_label = o == label;
        int64_t gidx = p0 + o;
        int chunk = (int)(gidx >> kOutChunkLog);
        unsigned peers = __match_any_sync(active, chunk);
        int leader = __ffs(peers) - 1;
        int rank = __popc(peers & ((1u << lane) - 1u));
        int off = 0;
        if (lane == leader)
            off = atomicAdd(out_cursor + chunk, __popc(peers));
        off = __shfl_sync(active, off, leader) + rank;
        if (off < kOutChunk) {
            int word0 = (int)(gidx & (kOutChunk - 1)) | (is_label ? (int)0x80000000u : 0);
            pairs[((int64_t)chunk << kOutChunkLog) + off] = make_int2(word0, is_label ? size : label);
        } else {
            atomicOr(err, kErrInternal);
        }
        bool is_root = root == (int)s;
        bool in_cat = is_root && size >= thr;
        // per-box counts: summed in registers while the warp stays inside one
        // box and added once per box (one counter per box would otherwise
        // take an atomic from every warp, all on one address)
        const int bi0 = __shfl_sync(active, bi, 0);
        const unsigned roots = __ballot_sync(active, is_root), cats = __ballot_sync(active, in_cat);
        if (__all_sync(active, bi == bi0)) {
            if (bi0 != acc_box) {
                if (lane == 0 && acc_box >= 0) {
                    if (acc_ng) atomicAdd(n_groups + acc_box, acc_ng);
                    if (acc_nk) atomicAdd(n_cat + acc_box, acc_nk);
                }
                acc_box = bi0;
                acc_ng = acc_nk = 0;
            }
            acc_ng += __popc(roots);
            acc_nk += __popc(cats);
        } else {
            unsigned bpeers = __match_any_sync(active, bi);
            int bleader = __ffs(bpeers) - 1;
            int ng = __popc(roots & bpeers);
            int nk = __popc(cats & bpeers);
            if (lane == bleader) {
                if (ng) atomicAdd(n_groups + bi, (unsigned long long)ng);
                if (nk) atomicAdd(n_cat + bi, (unsigned long long)nk);
            }
        }
        if (in_cat)
            atomicAdd(tile_cnt + (p0 + label) / kCatTile, 1);
    }
    // lane 0 took part in every iteration (its slot is the warp's smallest)
    if (lane == 0 && acc_box >= 0) {
        if (acc_ng) atomicAdd(n_groups + acc_box, acc_ng);
        if (acc_nk) atomicAdd(n_cat + acc_box, acc_nk);
    }
}

__global__ void __launch_bounds__(512) k_outputs_place(Geometry g, const int2* __restrict__ pairs,
                                                       int32_t* __restrict__ ids,
                                                       int32_t* __restrict__ sizes)
{
    __shared__ int s_ids[kOutChunk];
    __shared__ int s_sizes[kOutChunk];
    const int64_t n_chunks = (g.total_n + kOutChunk - 1) >> kOutChunkLog;
    for (int64_t c = blockIdx.x; c < n_chunks; c += gridDim.x) {
        const int64_t base = c << kOutChunkLog;
        const int len = (int)min((int64_t)kOutChunk, g.total_n - base);
        for (int k = threadIdx.x; k < len; k += blockDim.x) {
            int2 e = pairs[base + k];
            int off = e.x & (kOutChunk - 1);
            if (e.x < 0) {                       // the input is its group's label
                int64_t gidx = base + off;
                int bi = box_of(g.box_p0, g.nbox, gidx);
                s_ids[off] = (int)(gidx - g.boxes[bi].p0);
                s_sizes[off] = e.y;
            } else {
                s_ids[off] = e.y;
                s_sizes[off] = 0;
            }
        }
        __syncthreads();
        for (int k = threadIdx.x; k < len; k += blockDim.x) {
            ids[base + k] = s_ids[k];
            sizes[base + k] = s_sizes[k];
        }
        __syncthreads();
    }
}

constexpr int kCatThreads = 256;
constexpr int kCatItems = kCatTile / kCatThreads;   // 8

__device__ __forceinline__ int block_excl(int v, int* sw, int& total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sw[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int nw = blockDim.x >> 5;
        int t = lane < nw ? sw[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(kFull, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) sw[lane] = t;
    }
    __syncthreads();
    int off = wid ? sw[wid - 1] : 0;
    total = sw[(blockDim.x >> 5) - 1];
    __syncthreads();
    return off + x - v;
}

// One block per tile of kCatTile labels: entries of the tile in ascending
// label order at tile_off[tile].
__global__ void __launch_bounds__(kCatThreads) k_catalogue(Geometry g, const int32_t* __restrict__ sizes,
                                                           const int* __restrict__ tile_cnt,
                                                           const int* __restrict__ tile_off,
                                                           int32_t thr, int2* __restrict__ cat,
                                                           int64_t cap, Status* status)
{
    __shared__ int sw[32];
    for (int64_t tile = blockIdx.x; tile * kCatTile < g.total_n; tile += gridDim.x) {
        if (tile_cnt[tile] == 0)
            continue;      // block-uniform
        int64_t base = tile * kCatTile + (int64_t)threadIdx.x * kCatItems;
        int v[kCatItems];
        int f = 0;
        for (int k = 0; k < kCatItems; ++k) {
            int64_t i = base + k;
            v[k] = i < g.total_n ? sizes[i] : 0;
            f += v[k] >= thr;
        }
        int total;
        int64_t off = tile_off[tile] + block_excl(f, sw, total);
        for (int k = 0; k < kCatItems; ++k) {
            if (v[k] >= thr) {
                int64_t i = base + k;
                if (off < cap) {
                    int bi = box_of(g.box_p0, g.nbox, i);
                    cat[off] = make_int2((int)(i - g.boxes[bi].p0), v[k]);
                }
                ++off;
            }
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        int64_t nt = (g.total_n + kCatTile - 1) / kCatTile;
        status->n_cat_total = tile_off[nt];
    }
}

}  // namespace

static int grid_for(int64_t items, int threads, int per_sm)
{
    int64_t want = (items + threads - 1) / threads;
    int64_t cap = (int64_t)sm_count() * per_sm;
    if (want < 1) want = 1;
    return (int)(want < cap ? want : cap);
}

cudaError_t launch_finalize(const Geometry& g, const Work& w, const UfArgs& uf, int size_count,
                            cudaStream_t s)
{
    if (g.total_n == 0)
        return cudaSuccess;
    const bool ordered = uf.link == 0;
    if (size_count == 1)
        k_finalize_hash<<<grid_for(g.total_n, 256 * kHashBatch, 4), 256, 0, s>>>(
            g.total_n, w.parent, w.minorig, w.cnt, &w.status->err, ordered);
    else
        k_finalize<<<grid_for(g.total_n, 256, 8), 256, 0, s>>>(g.total_n, w.parent, w.minorig, w.cnt,
                                                              &w.status->err, ordered);
    return cudaGetLastError();
}

cudaError_t launch_outputs(const Geometry& g, const Work& w, int32_t* ids, int32_t* sizes,
                           int32_t min_size, cudaStream_t s)
{
    if (g.total_n == 0)
        return cudaSuccess;
    int32_t thr = min_size < 1 ? 1 : min_size;
    int2* pairs = (int2*)w.tmp;            // the brick-order copy is dead by now
    k_outputs_bucket<<<grid_for(g.total_n, 256, 8), 256, 0, s>>>(
        g, w.sorted, w.parent, w.minorig, w.cnt, thr, w.n_groups, w.n_cat, w.tile_cnt, w.out_cursor,
        pairs, &w.status->err);
    int64_t n_chunks = (g.total_n + kOutChunk - 1) >> kOutChunkLog;
    int blocks = (int)(n_chunks < (int64_t)sm_count() * 4 ? n_chunks : (int64_t)sm_count() * 4);
    k_outputs_place<<<blocks, 512, 0, s>>>(g, pairs, ids, sizes);
    return cudaGetLastError();
}

cudaError_t launch_catalogue(const Geometry& g, const Work& w, const int32_t* sizes, int32_t min_size,
                             int2* cat, int64_t cap, cudaStream_t s)
{
    if (g.total_n == 0)
        return cudaSuccess;
    int32_t thr = min_size < 1 ? 1 : min_size;
    cudaError_t e = launch_scan(w.tile_cnt, w.tile_off, w.n_tiles, w.scan_tmp, w.scan_tmp_len, s);
    if (e != cudaSuccess)
        return e;
    int blocks = grid_for(w.n_tiles * kCatThreads, kCatThreads, 8);
    k_catalogue<<<blocks, kCatThreads, 0, s>>>(g, sizes, w.tile_cnt, w.tile_off, thr, cat, cap, w.status);
    return cudaGetLastError();
}

}  // namespace fofgpu
