// Internal declarations of the GB300 Friends-of-Friends library.
//
// Device building blocks shared by the kernels:
//   * BoxDev: per-box geometry (a single box is a batch of one box);
//   * cell index of a coordinate, in float32, with a proven margin;
//   * the link predicate: a float32 pre-test whose error bound is derived in
//     fof_plan.cu (setup_box), and the exact double-precision predicate for
//     every pair the pre-test cannot settle;
//   * the concurrent union-find: Find with path halving (writes only on
//     paths of depth >= 2, paper Sec. 3.4.3) and Union by CAS hooking of the
//     larger root onto the smaller one (Sec. 3.1, Sec. 3.2), retried while
//     the hooked root changed under us, with a bounded retry count.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fofgpu {

constexpr int kWarp = 32;
constexpr unsigned kFull = 0xffffffffu;

// device error bits (combined into the status word with atomicOr)
constexpr int kErrRange = 1;     // a coordinate outside [0, L) or not finite
constexpr int kErrTimeout = 2;   // a union ran out of CAS retries
constexpr int kErrInternal = 4;  // an internal consistency check failed
constexpr int kFindCap = 1 << 26; // steps of one Find walk (a forest path is shorter)

// Debug builds (FOF_DEBUG_CHECKS, libfof_gb300_debug.so) check every
// neighbour-candidate slot a kernel computes against its box's slot range
// before the access; a bad slot is recorded as an internal error and the
// access goes to the box's first slot instead (never a trap).
#ifdef FOF_DEBUG_CHECKS
#define FOF_DCHECK_SLOT(j, b, err)                                        \
    do {                                                                  \
        if ((int64_t)(j) < (b).p0 || (int64_t)(j) >= (b).p0 + (b).n) {   \
            atomicOr((err), kErrInternal);                                \
            (j) = (int)(b).p0;                                            \
        }                                                                 \
    } while (0)
#else
#define FOF_DCHECK_SLOT(j, b, err) \
    do {                           \
    } while (0)
#endif

struct BoxDev {
    int64_t p0;       // first particle of the box in the concatenated arrays
    int64_t n;        // particles in the box
    int64_t brick0;   // first brick of the box (concatenated brick arrays)
    int64_t cell0;    // first cell of the box (concatenated cell arrays)
    double L;         // box side
    double l2;        // l_x * l_x rounded to double once
    int32_t nb;       // bricks per axis
    int32_t r;        // cells per brick per axis (power of two)
    int32_t log2r;
    int32_t nc;       // cells per axis = nb * r
    int32_t q;        // sub-cells per cell axis (1: cells are not split)
    int32_t nf;       // fine cells per axis = nc * q
    uint32_t magic_q; // ceil(2^32 / q): g / q == __umulhi(g, magic_q) for g < 2^14
    float inv_hf;     // float32(nf / L): fine index = min(nf-1, (int)(x * inv_hf))
    float Lf;         // float32(L) for the float32 pre-test
    float xmax;       // largest float32 strictly below L (valid: 0 <= x <= xmax)
    float t_lo;       // pre-test: d2f < t_lo  => linked
    float t_hi;       // pre-test: d2f > t_hi  => not linked
    float reach2;     // (l_x / hf)^2 (1 + 2^-6): a sub-cell whose box is farther
                      // than this (in fine units, squared) holds no partner
    int32_t team_min; // occupancy from which k_link links a cell as a warp team
    float bb_reach2;  // (l_x + 8 L 2^-24)^2 (1 + 2^-20): squared float32 gap from a
                      // bounding box beyond which no partner lies
};

// A cell is "subdivided" (linked by the sub-cell kernels, never pair by
// pair) when its box splits cells (q > 1) and it holds at least dense_min
// particles: up to kDenseMax particles it is a dense cell, staged in shared
// memory (fof_dense.cu); above, a big cell, sorted by sub-cell in global
// memory (fof_big.cu).
constexpr int kDenseMax = 3072;   // particles of a dense cell (shared memory)
// Largest team cell whose own pairs one warp links in shared memory
// (k_team_self); larger unsplit cells link their own pairs in k_link.
constexpr int kTeamSelfMax = 256;
// Team cells up to kTeamSplit particles are listed from the front of the
// team list, larger ones from its back, so each of k_team_self's two
// instantiations walks only its own cells.
constexpr int kTeamSplit = 128;
// Team cells from this size on are stored in z order by k_team_self, and the
// kernels that stream them from the cell below read only the z-prefix that
// can pair; sorting the many smaller cells costs more than it saves (measured
// on the 1024^3 box at 0.30 particles per cell: from 25 on, together with a
// team threshold of 10, the step is 1.5 ms shorter than from 17 with 8).
constexpr int kSortMin = 25;
constexpr int kMaxQ = 12;
constexpr int kMaxQ3 = kMaxQ * kMaxQ * kMaxQ;

// Per-run device status.
struct Status {
    int err;
    int pad;
    long long n_cat_total;
};

// ------------------------------------------------------------------------
// box lookup: box index of a concatenated particle / brick index
// ------------------------------------------------------------------------

__device__ __forceinline__ int box_of(const int64_t* __restrict__ starts, int nbox, int64_t i)
{
    int lo = 0, hi = nbox - 1;
    while (lo < hi) {                 // last box with starts[b] <= i
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(starts + mid) <= i) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ------------------------------------------------------------------------
// cells
// ------------------------------------------------------------------------

// Fine coordinate along one axis: (int)fl32(x * fl32(nf / L)), clamped so
// that every input (even an invalid one) stays inside the grid.  The cell
// coordinate is the fine one divided by q; the margins that make linked
// pairs land in adjacent cells (and sub-cells within +-2, and sub-cells
// cliques) are derived in fof_plan.cu (setup_box).
__device__ __forceinline__ int fine_coord(float x, const BoxDev& b)
{
    int c = (int)__fmul_rn(x, b.inv_hf);
    c = c < 0 ? 0 : c;
    return c > b.nf - 1 ? b.nf - 1 : c;
}

__device__ __forceinline__ int cell_coord(float x, const BoxDev& b)
{
    int g = fine_coord(x, b);
    return b.q == 1 ? g : (int)__umulhi((unsigned)g, b.magic_q);
}

__device__ __forceinline__ bool is_sub(int m, const BoxDev& b, int dense_min)
{
    return b.q > 1 && m >= dense_min;
}

__device__ __forceinline__ bool is_big(int m, const BoxDev& b)
{
    return b.q > 1 && m > kDenseMax;
}

__device__ __forceinline__ uint32_t spread3(uint32_t v)   // 5 bits -> every 3rd bit
{
    v &= 0x1fu;
    v = (v | (v << 8)) & 0x100fu;
    v = (v | (v << 4)) & 0x10c3u;
    v = (v | (v << 2)) & 0x1249u;
    return v;
}

// Morton order of a cell inside its brick (r <= 32).
__device__ __forceinline__ uint32_t local_code(int lx, int ly, int lz)
{
    return spread3((uint32_t)lx) | (spread3((uint32_t)ly) << 1) | (spread3((uint32_t)lz) << 2);
}

__device__ __forceinline__ int64_t brick_local(const BoxDev& b, int cx, int cy, int cz)
{
    int s = b.log2r;
    return ((int64_t)(cz >> s) * b.nb + (cy >> s)) * b.nb + (cx >> s);
}

// Concatenated cell index: cells are ordered brick by brick (row-major
// bricks), Morton order inside a brick.
__device__ __forceinline__ int64_t cell_key(const BoxDev& b, int cx, int cy, int cz)
{
    int m = b.r - 1;
    int64_t r3 = (int64_t)b.r * b.r * b.r;
    return b.cell0 + brick_local(b, cx, cy, cz) * r3 + local_code(cx & m, cy & m, cz & m);
}

__device__ __forceinline__ int wrap_cell(int c, int nc)
{
    return c < 0 ? c + nc : (c >= nc ? c - nc : c);
}

// The 13 forward neighbours of the half stencil: dz > 0, or dz == 0 and
// dy > 0, or dz == dy == 0 and dx > 0.  Offsets packed as (dx+1) + 3(dy+1)
// + 9(dz+1).
__device__ __forceinline__ void fwd_offset(int k, int& dx, int& dy, int& dz)
{
    // k = 0..12
    int code = k < 9 ? 18 + k : (k < 12 ? 15 + (k - 9) : 14);
    dx = code % 3 - 1;
    dy = (code / 3) % 3 - 1;
    dz = code / 9 - 1;
}

// ------------------------------------------------------------------------
// the link predicate
// ------------------------------------------------------------------------

__device__ __forceinline__ float sep_f32(float a, float b, float Lf)
{
    float d = fabsf(__fsub_rn(a, b));
    return fminf(d, __fsub_rn(Lf, d));
}

__device__ __forceinline__ float d2_f32(const float4& p, const float4& q, float Lf)
{
    float mx = sep_f32(p.x, q.x, Lf);
    float my = sep_f32(p.y, q.y, Lf);
    float mz = sep_f32(p.z, q.z, Lf);
    return __fmaf_rn(mz, mz, __fmaf_rn(my, my, __fmul_rn(mx, mx)));
}

__device__ __forceinline__ double wrap64(double d, double L)
{
    double half = 0.5 * L;
    if (d > half)
        d = __dsub_rn(d, L);
    else if (d < -half)
        d = __dadd_rn(d, L);
    return d;
}

// Exact predicate: s = (dx*dx + dy*dy) + dz*dz in IEEE double with every
// operation rounded to nearest and no contraction; linked iff s <= l2.
__device__ __forceinline__ bool linked_exact_inl(const float4& p, const float4& q, double L, double l2)
{
    double dx = wrap64(__dsub_rn((double)p.x, (double)q.x), L);
    double dy = wrap64(__dsub_rn((double)p.y, (double)q.y), L);
    double dz = wrap64(__dsub_rn((double)p.z, (double)q.z), L);
    double s = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
    s = __dadd_rn(s, __dmul_rn(dz, dz));
    return s <= l2;
}

// Out of line where register pressure matters: the band is rarely entered.
static __device__ __noinline__ bool linked_exact(float4 p, float4 q, double L, double l2)
{
    return linked_exact_inl(p, q, L, l2);
}

// Pre-test in float32, exact test only inside the uncertainty band.
__device__ __forceinline__ bool linked(const float4& p, const float4& q, const BoxDev& b)
{
    float s = d2_f32(p, q, b.Lf);
    if (s > b.t_hi)
        return false;
    if (s < b.t_lo)
        return true;
    return linked_exact_inl(p, q, b.L, b.l2);
}

// The same predicate with the band test out of line: fewer registers where
// the caller keeps much state live (the dense cell kernels).
__device__ __forceinline__ bool linked_ool(const float4& p, const float4& q, const BoxDev& b)
{
    float s = d2_f32(p, q, b.Lf);
    if (s > b.t_hi)
        return false;
    if (s < b.t_lo)
        return true;
    return linked_exact(p, q, b.L, b.l2);
}

// ------------------------------------------------------------------------
// union-find on the parent array (indices into the binned particle order)
// ------------------------------------------------------------------------

// Loads and stores at gpu scope, served by L2, so that a retry after a
// failed CAS sees the other SMs' hooks (L1 is not coherent).
__device__ __forceinline__ int ld_relaxed(const int* p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(int* p, int v)
{
    asm volatile("st.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Find with path halving.  Every value parent[x] ever holds is an ancestor
// of x (hooks only change roots, halving only skips to a grandparent), so
// racing writes are harmless; the walk strictly decreases x and ends.  The
// step cap only guards against a corrupted forest (it reports, never hangs).
__device__ __forceinline__ int uf_find(int* parent, int x, int* err)
{
    int p = ld_relaxed(parent + x);
    for (int step = 0; p != x; ++step) {
        int gp = ld_relaxed(parent + p);
        if (gp == p)
            return p;
        if (step >= kFindCap || gp > p) {
            atomicOr(err, kErrInternal);
            return p;
        }
        st_relaxed(parent + x, gp);
        x = gp;
        p = ld_relaxed(parent + x);
    }
    return x;
}

// The Finds of x and y (the same walk and halving as uf_find), with the two
// walks interleaved: each step issues the loads of both before using
// either, so the two chains of dependent loads overlap.
__device__ __forceinline__ void uf_find2(int* parent, int& x, int& y, int* err)
{
    int px = ld_relaxed(parent + x);
    int py = ld_relaxed(parent + y);
    for (int step = 0; px != x || py != y; ++step) {
        const bool wx = px != x, wy = py != y;
        const int gx = wx ? ld_relaxed(parent + px) : px;
        const int gy = wy ? ld_relaxed(parent + py) : py;
        if (step >= kFindCap || (wx && gx > px) || (wy && gy > py)) {
            atomicOr(err, kErrInternal);
            x = px;
            y = py;
            return;
        }
        if (wx) {
            if (gx == px) {
                x = px;                        // px is the root
            } else {
                st_relaxed(parent + x, gx);
                x = gx;
                px = ld_relaxed(parent + x);
            }
        }
        if (wy) {
            if (gy == py) {
                y = py;
            } else {
                st_relaxed(parent + y, gy);
                y = gy;
                py = ld_relaxed(parent + y);
            }
        }
    }
}

// Union by root: hook the larger root onto the smaller with CAS, which only
// succeeds while the larger is still a root; otherwise re-find and retry.
// Keeps parent[x] <= x, hence no cycles.  Returns the root reached.
__device__ __forceinline__ int uf_union(int* parent, int a, int b, int cap, int* err)
{
    for (int it = 0; it < cap; ++it) {
        uf_find2(parent, a, b, err);
        if (a == b)
            return a;
        int hi = a > b ? a : b;
        int lo = a > b ? b : a;
        if (atomicCAS(parent + hi, hi, lo) == hi)
            return lo;
    }
    atomicOr(err, kErrTimeout);
    return a < b ? a : b;
}

// ------------------------------------------------------------------------
// union-find variants (measured against the default; same partition)
// ------------------------------------------------------------------------

// Arguments of every union-find call of a kernel.  `find` and `link` select
// the variants of fof.h (FOF_FIND_*, FOF_LINK_*); they are read only by the
// kernels' variant instantiation (kVar = true), so the default path carries
// no runtime switch.
struct UfArgs {
    int cap;     // CAS attempts per union
    int* err;    // status word
    int find;    // 0 halving on paths of depth >= 2, 1 halving at every depth,
                 // 2 full compression, 3 none
    int link;    // 0 hook the larger root onto the smaller, 1 randomised
    int var;     // run the variant instantiation (a variant is selected, or forced)
};

// Random priority of a root for randomised linking: the 32-bit finaliser of
// MurmurHash3, a bijection, so distinct roots never tie.
__device__ __forceinline__ uint32_t uf_priority(int x)
{
    uint32_t h = (uint32_t)x;
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

// Find under the selected compression.  Every value parent[x] ever holds is
// an ancestor of x in every variant, so racing writes stay harmless.  The
// ordering check (a parent never exceeds its child) holds only when roots
// hook onto smaller roots.
__device__ __forceinline__ int uf_find_var(int* parent, int x, const UfArgs& u)
{
    const bool ordered = u.link == 0;
    if (u.find == 2) {                              // full compression
        // The first walk records the nodes it passes; every one of them has
        // the root r found as an ancestor for good (trees only merge), so
        // pointing them at r is safe.  Walking the path a second time would
        // not be: other threads may have re-pointed it past r, and writing r
        // into an ancestor of r would close a cycle.
        constexpr int kPath = 16;
        int path[kPath];
        int len = 0;
        int r = x;
        int p = ld_relaxed(parent + r);
        for (int step = 0; p != r; ++step) {
            if (step >= kFindCap || (ordered && p > r)) {
                atomicOr(u.err, kErrInternal);
                return p;
            }
            if (len < kPath)
                path[len++] = r;
            r = p;
            p = ld_relaxed(parent + r);
        }
        for (int k = 0; k + 1 < len; ++k)            // the last one already points at r
            st_relaxed(parent + path[k], r);
        return r;
    }
    int p = ld_relaxed(parent + x);
    for (int step = 0; p != x; ++step) {
        const int gp = ld_relaxed(parent + p);
        if (step >= kFindCap || (ordered && gp > p)) {
            atomicOr(u.err, kErrInternal);
            return p;
        }
        if (gp == p) {
            if (u.find == 1)
                st_relaxed(parent + x, gp);         // the depth-1 rewrite (same value)
            return p;
        }
        if (u.find == 3) {                          // no compression: plain walk
            x = p;
            p = gp;
            continue;
        }
        st_relaxed(parent + x, gp);
        x = gp;
        p = ld_relaxed(parent + x);
    }
    return x;
}

__device__ __forceinline__ int uf_union_var(int* parent, int a, int b, const UfArgs& u)
{
    for (int it = 0; it < u.cap; ++it) {
        a = uf_find_var(parent, a, u);
        b = uf_find_var(parent, b, u);
        if (a == b)
            return a;
        int hi, lo;                                 // hi is hooked onto lo
        if (u.link == 1) {
            const bool a_wins = uf_priority(a) > uf_priority(b);
            lo = a_wins ? a : b;
            hi = a_wins ? b : a;
        } else {
            hi = a > b ? a : b;
            lo = a > b ? b : a;
        }
        if (atomicCAS(parent + hi, hi, lo) == hi)
            return lo;
    }
    atomicOr(u.err, kErrTimeout);
    return a < b ? a : b;
}

template <bool kVar>
__device__ __forceinline__ int ufind(int* parent, int x, const UfArgs& u)
{
    return kVar ? uf_find_var(parent, x, u) : uf_find(parent, x, u.err);
}

template <bool kVar>
__device__ __forceinline__ int uunion(int* parent, int a, int b, const UfArgs& u)
{
    return kVar ? uf_union_var(parent, a, b, u) : uf_union(parent, a, b, u.cap, u.err);
}

// ------------------------------------------------------------------------
// kernel launchers (one per phase); each returns cudaGetLastError()
// ------------------------------------------------------------------------

struct Geometry {
    const BoxDev* boxes;       // [nbox]
    const int64_t* box_p0;     // [nbox] first particle of each box
    const int64_t* box_brick0; // [nbox] first brick of each box
    int nbox;
    int64_t total_n;           // particles over all boxes
    int64_t total_bricks;
    int64_t total_cells;
};

struct Work {
    float4* tmp;        // [total_n] particles in brick order
    float4* sorted;     // [total_n] particles in cell order, w = box-local index
    int* parent;        // [total_n] union-find forest over cell-order slots
    int* minorig;       // [total_n] smallest box-local index per root
    int* cnt;           // [total_n] group size per root
    int* cell_start;    // [total_cells + 1]
    int* bcount;        // [total_bricks + 1]
    int* bstart;        // [total_bricks + 1]
    int* bcursor;       // [total_bricks]
    int* scan_tmp;      // scan partials
    int64_t scan_tmp_len;
    int* tile_cnt;      // [n_tiles + 1] catalogue entries per label tile
    int* tile_off;      // [n_tiles + 1]
    int* out_cursor;    // [total_n / kOutChunk + 1] fill of each output bucket
    int64_t n_tiles;
    Status* status;     // device status
    unsigned long long* n_groups;  // [nbox]
    unsigned long long* n_cat;     // [nbox]
    int64_t* dense_list; // [dense_cap] cell keys of the subdivided cells
    int* n_dense;        // number of entries in dense_list
    int* dense_root;     // [total_n / dense_min + 1] by first slot / dense_min:
                         // root of a subdivided cell that is one group, else -1
    int64_t* big_list;   // [big_cap] cell keys of the big cells (subdivided, > kDenseMax)
    int* n_big;          // number of entries in big_list
    int64_t* team_list;  // [team_cap] team cells (team_min..kTeamSelfMax particles, not
                         // subdivided): size << 32 | first slot
    int* n_team;         // entries at the front of team_list (cells up to kTeamSplit)
    int* n_team_hi;      // entries at its back (cells above kTeamSplit)
    int64_t team_cap;    // capacity of team_list
};

constexpr int kCatTile = 2048;  // labels per catalogue tile
constexpr int kOutChunkLog = 12;                 // outputs: input indices per chunk
constexpr int kOutChunk = 1 << kOutChunkLog;

int sm_count();

cudaError_t launch_bin_count(const float* pos, const Geometry& g, const Work& w, cudaStream_t s);
cudaError_t launch_scan(const int* in, int* out, int64_t len, int* tmp, int64_t tmp_len,
                        cudaStream_t s);
int64_t scan_tmp_elems(int64_t len);
cudaError_t launch_bin_scatter(const float* pos, const Geometry& g, const Work& w, cudaStream_t s);
cudaError_t launch_brick_sort(const Geometry& g, const Work& w, int dense_min, cudaStream_t s);
// incremental re-binning: flags |= 1 if a particle left its cell, 2 if it left its brick
cudaError_t launch_relink_check(const float* pos, const Geometry& g, const Work& w, int* flags,
                                cudaStream_t s);
cudaError_t launch_forest_init(const Geometry& g, const Work& w, cudaStream_t s);
cudaError_t launch_dense(const Geometry& g, const Work& w, int dense_min, const UfArgs& uf, bool pairs,
                         cudaStream_t s);
size_t dense_smem();
cudaError_t launch_link(const Geometry& g, const Work& w, int dense_min, const UfArgs& uf,
                        cudaStream_t s);
cudaError_t launch_team_self(const Geometry& g, const Work& w, cudaStream_t s);
// big cells: sort by sub-cell + own pairs (before the dense kernels), then
// their pairs with every neighbour (after them)
cudaError_t launch_big(const Geometry& g, const Work& w, int dense_min, const UfArgs& uf, bool pairs,
                       cudaStream_t s);
// size_count: 0 warp-aggregated atomics, 1 per-block shared-memory hash table
cudaError_t launch_finalize(const Geometry& g, const Work& w, const UfArgs& uf, int size_count,
                            cudaStream_t s);
cudaError_t launch_outputs(const Geometry& g, const Work& w, int32_t* ids, int32_t* sizes,
                           int32_t min_size, cudaStream_t s);
cudaError_t launch_catalogue(const Geometry& g, const Work& w, const int32_t* sizes,
                             int32_t min_size, int2* cat, int64_t cap, cudaStream_t s);

}  // namespace fofgpu
