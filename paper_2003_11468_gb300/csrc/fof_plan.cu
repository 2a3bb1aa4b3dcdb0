// Plan, workspace and C ABI of the Friends-of-Friends library (fof.h).
//
// A plan holds the geometry of one or more independent periodic boxes, a
// device workspace sized for them, and a small pinned host block for the
// status read-back.  fof_link enqueues binning and linking; fof_groups
// enqueues finalisation and outputs and reads the status back once.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "fof.h"
#include "fof_internal.cuh"

using namespace fofgpu;

namespace fofgpu {

int sm_count()
{
    static int cached = 0;
    if (cached == 0) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
            cached = v;
        else
            return 152;
    }
    return cached;
}

}  // namespace fofgpu

namespace {

enum Phase {
    kPhBinCount, kPhScanBricks, kPhBinScatter, kPhBrickSort, kPhTeamSelf, kPhBigSort, kPhDenseSelf,
    kPhDensePairs, kPhBigPairs, kPhLink, kPhFinalize, kPhOutputs, kPhCatalogue, kNumPhases
};

const char* kPhaseNames[kNumPhases] = {
    "bin_count", "scan_bricks", "bin_scatter", "brick_sort", "team_self", "big_sort", "dense_self",
    "dense_pairs", "big_pairs", "link", "finalize", "outputs", "catalogue",
};
const int kPhaseLaunches[kNumPhases] = {1, 3, 1, 1, 2, 1, 2, 2, 1, 1, 1, 2, 4};

constexpr int64_t kMaxTotal = 2147483646LL;   // slots and labels are int32
constexpr int kDefaultRetryCap = 1 << 20;
constexpr int kDefaultDenseMin = 256;
constexpr double kDefaultOccupancy = 0.30;
constexpr int kDefaultTeamMin = 10;
constexpr int kMinTeamMin = 2;                 // smallest accepted team threshold (sizes team_list)
constexpr int kMaxCellsPerAxis = 4096;        // float32 cell-index precision (unsplit cells)
constexpr int kMaxFinePerAxis = 16384;        // float32 index precision (sub-cells)

// Results block (device and pinned host copy): status, then per-box counts.
struct ResultsLayout {
    size_t status_off, groups_off, cat_off, bytes;
};

ResultsLayout results_layout(int nbox)
{
    ResultsLayout r;
    r.status_off = 0;
    r.groups_off = 64;
    r.cat_off = r.groups_off + sizeof(long long) * (size_t)nbox;
    r.bytes = r.cat_off + sizeof(long long) * (size_t)nbox;
    return r;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

float float_up(double v)        // smallest float >= v
{
    float f = (float)v;
    while ((double)f < v) f = std::nextafter(f, INFINITY);
    return f;
}

float float_down(double v)      // largest float <= v
{
    float f = (float)v;
    while ((double)f > v) f = std::nextafter(f, -INFINITY);
    return f;
}

// Geometry and predicate constants of one box.
//
// Cell size.  Cells per axis nc <= floor(L / (l_x (1 + 2^-9))) and
// nc <= 4096, so the cell side h = L/nc >= l_x (1 + 2^-9).  The device
// computes a cell coordinate as (int)fl32(x * fl32(nc/L)); two roundings of
// relative size 2^-24 shift a coordinate by at most nc 2^-23 <= 2^-11 cell,
// and two coordinates by at most 2^-10 cell.  A pair that the exact
// predicate links is at most l_x (1 + 2^-50) apart per axis, i.e. less
// than 1 - 2^-9 + 2^-18 cells, so its computed cells differ by at most one
// (periodically).  Hence the 27-cell stencil finds every linked pair.
//
// Float32 pre-test.  For coordinates a, b in [0, L) the device computes per
// axis m = min(|fl(a - b)|, fl(fl32(L) - |fl(a - b)|)).  With u = 2^-24,
// |m - t| <= E1 = 3.01 u L where t = min(|a - b|, L - |a - b|) is the exact
// periodic separation (one rounding of the difference, one of L, one of the
// second difference).  The sum sf = fma(mz,mz, fma(my,my, mx*mx)) is within
// a factor (1 +- 3.01 u) of |m|^2.  The exact double predicate deviates from
// |t| by at most 2^-51 L per axis (roundings of the difference and of the
// wrap) and compares against l2 = l_x^2 (1 +- 2^-53).  Therefore, with
// E = E1 + 2^-51 L and sqrt(3) < 1.733:
//   linked exactly  =>  sf <= (l_x (1 + 2^-50) + 1.733 E)^2 (1 + 3.01 u)
//   sf < (l_x (1 - 2^-50) - 1.733 E)^2 (1 - 3.01 u)  =>  linked exactly.
// Both bounds get a further relative slack of 2^-20 and are rounded outward
// to float32.  Pairs between them take the exact double test.
// Cells per brick side for nc cells per axis.
int brick_side(int64_t nc)
{
    return nc >= 128 ? 16 : (nc >= 32 ? 8 : (nc >= 8 ? 4 : (nc >= 4 ? 2 : 1)));
}

// Sub-cells per cell side for nc cells per axis (1: the cells cannot be
// split).  The conditions are derived below, at the sub-cell comment of
// setup_box.
int sub_cells_for(double L, double l_x, int64_t nc)
{
    const double h = L / (double)nc;
    const double want = std::ceil(h * std::sqrt(3.0) * (1.0 + std::ldexp(1.0, -7)) / l_x);
    if (want >= 2.0 && want <= kMaxQ && nc >= 3 && nc * (int64_t)want <= kMaxFinePerAxis) {
        const double hf = h / want;
        if (hf >= l_x * (1.0 + std::ldexp(1.0, -7)) / 2.0 &&
            hf * std::sqrt(3.0) * (1.0 + std::ldexp(1.0, -7)) <= l_x)
            return (int)want;
    }
    return 1;
}

int setup_box(double L, double l_x, int64_t n, const fof_options* o, BoxDev& b)
{
    if (!std::isfinite(L) || !(L > 0.0) || !std::isfinite(l_x) || !(l_x > 0.0) ||
        !(l_x < 0.5 * L) || n < 0 || n > kMaxTotal || L > 1e30)
        return FOF_ERR_ARG;
    if (o && (o->tie_rule < 0 || o->tie_rule > FOF_TIE_LT || o->find_variant < 0 ||
              o->find_variant > FOF_FIND_NONE || o->size_count < 0 || o->size_count > FOF_SIZE_HASH ||
              o->link_order < 0 || o->link_order > FOF_LINK_RANDOM ||
              (o->debug_flags & ~(FOF_DEBUG_UNION_NO_RETRY | FOF_DEBUG_VARIANT_KERNELS)) != 0 || o->reserved[0] != 0 ||
              o->reserved[1] != 0 || o->team_min < 0 || o->dense_min < 0 || o->retry_cap < 0))
        return FOF_ERR_ARG;
    std::memset(&b, 0, sizeof(b));
    double q = std::floor(L / (l_x * (1.0 + std::ldexp(1.0, -9))));
    int64_t nc_max = q < 1.0 ? 1 : (q > kMaxCellsPerAxis ? kMaxCellsPerAxis : (int64_t)q);
    int64_t nc;
    if (o && o->cells_per_axis > 0) {
        if (o->cells_per_axis > nc_max)
            return FOF_ERR_ARG;
        nc = o->cells_per_axis;
    } else {
        double occ = (o && o->occupancy > 0.0) ? o->occupancy : kDefaultOccupancy;
        double t = std::floor(std::cbrt((double)n / occ));
        nc = t < 1.0 ? 1 : (int64_t)t;
        if (nc > nc_max) nc = nc_max;
    }
    int r;
    if (o && o->brick_cells > 0) {
        r = o->brick_cells;
        if ((r & (r - 1)) != 0 || r > 16 || r > nc)
            return FOF_ERR_ARG;
    } else {
        r = brick_side(nc);
    }
    int64_t nb = nc / r;
    nc = nb * r;
    // The library's own cell count: when those cells cannot be split into
    // sub-cells (their side falls between the ranges some q covers), take
    // the nearest coarser grid (then finer) whose cells can, so that dense
    // cells get the sub-cell method instead of pair-by-pair linking.
    if (!(o && o->cells_per_axis > 0) && nc >= 3 && sub_cells_for(L, l_x, nc) == 1) {
        for (int64_t d = 1; d <= nc; ++d) {
            bool found = false;
            for (int sgn = 0; sgn < 2 && !found; ++sgn) {
                const int64_t c = sgn == 0 ? nc - d : nc + d;
                if (c < 3 || c > nc_max)
                    continue;
                const int rc = (o && o->brick_cells > 0) ? r : brick_side(c);
                if (rc > c)
                    continue;
                const int64_t cr = (c / rc) * rc;
                if (cr >= 3 && cr <= nc_max && sub_cells_for(L, l_x, cr) > 1) {
                    nc = cr;
                    r = rc;
                    nb = cr / rc;
                    found = true;
                }
            }
            if (found)
                break;
        }
    }
    int log2r = 0;
    while ((1 << log2r) < r) ++log2r;

    // Sub-cells.  q sub-cells per cell side, fine side hf = h/q with
    //   l_x (1 + 2^-7) / 2 <= hf <= l_x / (sqrt(3) (1 + 2^-7)),
    // nf = nc q <= 16384 fine cells per axis and nc >= 3.  The fine index
    // (int)fl32(x * fl32(nf/L)) is within nf 2^-23 <= 2^-9 fine cells of
    // x nf / L, so (a) the members of one fine cell span at most
    // hf (1 + 2^-8) per axis, a diameter below sqrt(3) hf (1 + 2^-8) <
    // l_x (1 - 2^-9): every pair inside a fine cell is linked exactly; and
    // (b) a linked pair, at most l_x (1 + 2^-50) <= hf (2 - 2^-6) apart per
    // axis, has fine indices at most 2 apart, hence cell indices at most 1
    // apart.  When no q meets these bounds the box keeps q = 1 and cells
    // are never split.
    const int qs = sub_cells_for(L, l_x, nc);
    b.n = n;
    b.L = L;
    b.l2 = l_x * l_x;
    // "distance < l_x" (the naive listing's test, Sec. 3.1): for doubles,
    // s < l2 exactly when s <= the largest double below l2.  Every margin
    // below is relative and far wider than this one step.
    if (o && o->tie_rule == FOF_TIE_LT)
        b.l2 = std::nextafter(b.l2, 0.0);
    b.nb = (int32_t)nb;
    b.r = r;
    b.log2r = log2r;
    b.nc = (int32_t)nc;
    b.q = qs;
    b.nf = (int32_t)(nc * qs);
    b.magic_q = qs > 1 ? (uint32_t)((((uint64_t)1 << 32) + qs - 1) / qs) : 0u;
    b.inv_hf = (float)((double)b.nf / L);
    b.Lf = (float)L;
    // A partner of p lies within l_x (1 + 2^-50) of p.  The gap between p and
    // a sub-cell, measured from p's float32 fine coordinate (error below
    // 2^-8 fine units, both roundings included), underestimates the true gap
    // by less than 2^-8 per axis; comparing its square with
    // (l_x/hf + 2^-6)^2 therefore never drops a sub-cell holding a partner.
    {
        double rf = l_x / (L / (double)b.nf) + std::ldexp(1.0, -6);
        b.reach2 = (float)(rf * rf * (1.0 + std::ldexp(1.0, -20)));
    }
    b.team_min = (o && o->team_min > 0) ? o->team_min : kDefaultTeamMin;
    if (b.team_min < kMinTeamMin)
        b.team_min = kMinTeamMin;
    // Team bounding-box filter.  A neighbour particle shifted by +-float32(L)
    // and the float32 gaps to the box are each within L 2^-24 (shift: the
    // sum and float32(L); gap: one subtraction) per axis, 3 L 2^-24 together,
    // sqrt(3) * 3 < 5.2 over three axes; a partner is at most l_x (1 + 2^-50)
    // away; so a linked pair has squared gap below (l_x + 8 L 2^-24)^2, and
    // the final 2^-20 covers the rounding of the squares and their sum.
    {
        double rb = l_x * (1.0 + std::ldexp(1.0, -50)) + 8.0 * L * std::ldexp(1.0, -24);
        b.bb_reach2 = float_up(rb * rb * (1.0 + std::ldexp(1.0, -20)));
    }
    b.xmax = (float)L;
    while ((double)b.xmax >= L) b.xmax = std::nextafter(b.xmax, 0.0f);

    const double u = std::ldexp(1.0, -24);
    const double E = 3.01 * u * L + std::ldexp(L, -51);
    const double slack = std::ldexp(1.0, -20);
    double rhi = l_x * (1.0 + std::ldexp(1.0, -50)) + 1.733 * E;
    double thi = rhi * rhi * (1.0 + 3.01 * u) * (1.0 + slack);
    double rlo = l_x * (1.0 - std::ldexp(1.0, -50)) - 1.733 * E;
    double tlo = rlo > 0.0 ? rlo * rlo * (1.0 - 3.01 * u) * (1.0 - slack) : 0.0;
    b.t_hi = float_up(thi);
    b.t_lo = tlo > 0.0 ? float_down(tlo) : 0.0f;
    return FOF_OK;
}

// Pinned status blocks come from one process-wide slab cut into 4 KB
// chunks, so creating and destroying plans never calls cudaMallocHost /
// cudaFreeHost (the latter waits for the whole device).  Plans whose block
// is larger than a chunk (batches of more than 250 boxes) allocate their own.
constexpr size_t kPinChunk = 4096;
constexpr int kPinChunks = 1024;
std::mutex g_pin_mu;
char* g_pin_slab = nullptr;
bool g_pin_used[kPinChunks];

char* pinned_alloc(size_t bytes, bool& from_slab)
{
    from_slab = false;
    if (bytes <= kPinChunk) {
        std::lock_guard<std::mutex> lock(g_pin_mu);
        if (!g_pin_slab) {
            if (cudaHostAlloc((void**)&g_pin_slab, kPinChunk * kPinChunks, cudaHostAllocPortable) !=
                cudaSuccess) {
                cudaGetLastError();
                g_pin_slab = nullptr;
            }
        }
        if (g_pin_slab)
            for (int k = 0; k < kPinChunks; ++k)
                if (!g_pin_used[k]) {
                    g_pin_used[k] = true;
                    from_slab = true;
                    return g_pin_slab + k * kPinChunk;
                }
    }
    char* p = nullptr;
    if (cudaMallocHost((void**)&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void pinned_free(char* p, bool from_slab)
{
    if (!p)
        return;
    if (from_slab) {
        std::lock_guard<std::mutex> lock(g_pin_mu);
        g_pin_used[(p - g_pin_slab) / kPinChunk] = false;
    } else {
        cudaFreeHost(p);
    }
}

struct PhaseTimer {
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    bool pending = false;
    double ms = 0.0;
    int64_t launches = 0;
};

}  // namespace

struct fof_plan {
    int nbox = 0;
    std::vector<BoxDev> boxes;
    std::vector<int64_t> p0, brick0;
    Geometry g{};
    Work w{};
    char* ws = nullptr;
    size_t ws_bytes = 0;
    bool own_ws = false;
    char* results_dev = nullptr;
    char* results_host = nullptr;   // pinned
    bool results_from_slab = false;
    ResultsLayout rl{};
    int dense_min = kDefaultDenseMin;
    int retry_cap = kDefaultRetryCap;
    int find_variant = 0;
    int link_order = 0;
    int size_count = 0;
    bool force_var = false;
    bool linked = false;
    bool binned = false;      // the binned order of the last fof_link is in place
    int last_relink_path = -1;
    bool pending = false;
    int64_t last_cap = 0;
    bool timing = false;
    bool capturing = false;
    PhaseTimer phase[kNumPhases];
    int64_t launches = 0;
    // fof_run_host staging
    float* pos_d = nullptr;
    int32_t* ids_d = nullptr;
    int32_t* sizes_d = nullptr;
    int2* cat_d = nullptr;
    int64_t cat_d_cap = 0;
    // fof_run_host_many: two staging sets, copy streams and their events
    float* pos2[2] = {nullptr, nullptr};
    int32_t* ids2[2] = {nullptr, nullptr};
    int32_t* sizes2[2] = {nullptr, nullptr};
    int2* cat2[2] = {nullptr, nullptr};
    int64_t cat2_cap = 0;
    cudaStream_t copy_in = nullptr, copy_out = nullptr;
    cudaEvent_t ev_h2d[2] = {nullptr, nullptr}, ev_comp[2] = {nullptr, nullptr},
                ev_d2h[2] = {nullptr, nullptr};
    // graph
    cudaGraphExec_t gexec = nullptr;
    int64_t graph_cap = 0;
};

namespace {

struct Layout {
    size_t boxes, p0, brick0, results, bcount, bstart, bcursor, scan_tmp, tile_cnt, tile_off,
        cell_start, tmp, sorted, parent, minorig, cnt, dense_list, n_dense, dense_root, out_cursor,
        team_list, n_team, n_team_hi, big_list, n_big, total;
    int64_t scan_len, n_tiles, dense_cap, team_cap;
};

Layout layout(int nbox, int64_t total_n, int64_t total_bricks, int64_t total_cells,
              int dense_min = kDefaultDenseMin)
{
    Layout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t at = off;
        off = align_up(off + (bytes ? bytes : 1), 256);
        return at;
    };
    L.n_tiles = (total_n + kCatTile - 1) / kCatTile;
    int64_t s1 = scan_tmp_elems(total_bricks), s2 = scan_tmp_elems(L.n_tiles);
    L.scan_len = s1 > s2 ? s1 : s2;
    L.boxes = take(sizeof(BoxDev) * (size_t)nbox);
    L.p0 = take(8 * (size_t)nbox);
    L.brick0 = take(8 * (size_t)nbox);
    L.results = take(results_layout(nbox).bytes);
    L.bcount = take(4 * (size_t)(total_bricks + 1));
    L.bstart = take(4 * (size_t)(total_bricks + 1));
    L.bcursor = take(4 * (size_t)(total_bricks + 1));
    L.scan_tmp = take(4 * (size_t)L.scan_len);
    L.tile_cnt = take(4 * (size_t)(L.n_tiles + 1));
    L.tile_off = take(4 * (size_t)(L.n_tiles + 1));
    L.cell_start = take(4 * (size_t)(total_cells + 1));
    L.tmp = take(16 * (size_t)total_n);
    L.sorted = take(16 * (size_t)total_n);
    L.parent = take(4 * (size_t)total_n);
    L.minorig = take(4 * (size_t)total_n);
    L.cnt = take(4 * (size_t)total_n);
    L.dense_cap = total_n / dense_min + 1;
    L.dense_list = take(8 * (size_t)L.dense_cap);
    L.n_dense = take(4);
    L.dense_root = take(4 * (size_t)(total_n / dense_min + 2));
    L.out_cursor = take(4 * (size_t)((total_n >> kOutChunkLog) + 2));
    L.team_cap = total_n / kMinTeamMin + 1;
    L.team_list = take(8 * (size_t)L.team_cap);
    L.n_team = take(4);
    L.n_team_hi = take(4);
    L.big_list = take(8 * (size_t)(total_n / (kDenseMax + 1) + 1));
    L.n_big = take(4);
    L.total = off;
    return L;
}

int dense_min_of(const fof_options* opt)
{
    return (opt && opt->dense_min > 0) ? opt->dense_min : kDefaultDenseMin;
}

int setup_batch(int32_t nbox, const double* box, const double* l_x, const int64_t* n,
                const fof_options* opt, std::vector<BoxDev>& boxes, int64_t& tn, int64_t& tb,
                int64_t& tc)
{
    if (nbox < 1 || !box || !l_x || !n)
        return FOF_ERR_ARG;
    boxes.resize(nbox);
    tn = tb = tc = 0;
    for (int i = 0; i < nbox; ++i) {
        int rc = setup_box(box[i], l_x[i], n[i], opt, boxes[i]);
        if (rc != FOF_OK)
            return rc;
        BoxDev& b = boxes[i];
        b.p0 = tn;
        b.brick0 = tb;
        b.cell0 = tc;
        int64_t nb3 = (int64_t)b.nb * b.nb * b.nb;
        tn += b.n;
        tb += nb3;
        tc += nb3 * (int64_t)b.r * b.r * b.r;
        // slots and brick indices are matched and scanned as int32
        if (tn > kMaxTotal || tb > kMaxTotal)
            return FOF_ERR_ARG;
    }
    return FOF_OK;
}

int cuda_rc(cudaError_t e)
{
    if (e == cudaSuccess)
        return FOF_OK;
    if (e == cudaErrorMemoryAllocation)
        return FOF_ERR_OOM;
    return FOF_ERR_CUDA;
}

#define FOF_TRY(expr)                                  \
    do {                                               \
        cudaError_t e_ = (expr);                       \
        if (e_ != cudaSuccess) return cuda_rc(e_);     \
    } while (0)

void phase_begin(fof_plan* h, int ph, cudaStream_t s)
{
    h->launches += kPhaseLaunches[ph];
    h->phase[ph].launches += kPhaseLaunches[ph];
    if (h->timing && !h->capturing) {
        cudaEventRecord(h->phase[ph].ev0, s);
    }
}

void phase_end(fof_plan* h, int ph, cudaStream_t s)
{
    if (h->timing && !h->capturing) {
        cudaEventRecord(h->phase[ph].ev1, s);
        h->phase[ph].pending = true;
    }
}

void collect_times(fof_plan* h)
{
    for (int k = 0; k < kNumPhases; ++k) {
        PhaseTimer& t = h->phase[k];
        if (!t.pending)
            continue;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, t.ev0, t.ev1) == cudaSuccess)
            t.ms += ms;
        t.pending = false;
    }
}

int create_plan(int32_t nbox, const double* box, const double* l_x, const int64_t* n,
                const fof_options* opt, void* workspace, size_t workspace_bytes, fof_handle* out)
{
    if (!out)
        return FOF_ERR_ARG;
    *out = nullptr;
    std::vector<BoxDev> boxes;
    int64_t tn, tb, tc;
    int rc = setup_batch(nbox, box, l_x, n, opt, boxes, tn, tb, tc);
    if (rc != FOF_OK)
        return rc;
    Layout L = layout(nbox, tn, tb, tc, dense_min_of(opt));
    if (workspace && (workspace_bytes < L.total || ((uintptr_t)workspace & 255u)))
        return FOF_ERR_ARG;

    fof_plan* h = new (std::nothrow) fof_plan();
    if (!h)
        return FOF_ERR_OOM;
    h->nbox = nbox;
    h->boxes = boxes;
    if (opt && opt->dense_min > 0) h->dense_min = opt->dense_min;
    if (opt && opt->retry_cap > 0) h->retry_cap = opt->retry_cap;
    // the retry-cap test: a union that must hook gives up before its first CAS
    if (opt && (opt->debug_flags & FOF_DEBUG_UNION_NO_RETRY)) h->retry_cap = 0;
    if (opt) {
        h->find_variant = opt->find_variant;
        h->link_order = opt->link_order;
        h->size_count = opt->size_count;
        h->force_var = (opt->debug_flags & FOF_DEBUG_VARIANT_KERNELS) != 0;
    }
    h->rl = results_layout(nbox);
    if (workspace) {
        h->ws = (char*)workspace;
        h->own_ws = false;
    } else {
        cudaError_t e = cudaMalloc((void**)&h->ws, L.total);
        if (e != cudaSuccess) {
            delete h;
            cudaGetLastError();
            return FOF_ERR_OOM;
        }
        h->own_ws = true;
    }
    h->ws_bytes = L.total;
    h->results_host = pinned_alloc(h->rl.bytes, h->results_from_slab);
    if (!h->results_host) {
        fof_destroy(h);
        return FOF_ERR_OOM;
    }
    std::memset(h->results_host, 0, h->rl.bytes);
    for (int k = 0; k < kNumPhases; ++k) {
        if (cudaEventCreate(&h->phase[k].ev0) != cudaSuccess ||
            cudaEventCreate(&h->phase[k].ev1) != cudaSuccess) {
            fof_destroy(h);
            return FOF_ERR_CUDA;
        }
    }
    char* ws = h->ws;
    h->p0.resize(nbox);
    h->brick0.resize(nbox);
    for (int i = 0; i < nbox; ++i) {
        h->p0[i] = boxes[i].p0;
        h->brick0[i] = boxes[i].brick0;
    }
    Geometry& g = h->g;
    g.boxes = (const BoxDev*)(ws + L.boxes);
    g.box_p0 = (const int64_t*)(ws + L.p0);
    g.box_brick0 = (const int64_t*)(ws + L.brick0);
    g.nbox = nbox;
    g.total_n = tn;
    g.total_bricks = tb;
    g.total_cells = tc;
    Work& w = h->w;
    h->results_dev = ws + L.results;
    w.status = (Status*)(h->results_dev + h->rl.status_off);
    w.n_groups = (unsigned long long*)(h->results_dev + h->rl.groups_off);
    w.n_cat = (unsigned long long*)(h->results_dev + h->rl.cat_off);
    w.bcount = (int*)(ws + L.bcount);
    w.bstart = (int*)(ws + L.bstart);
    w.bcursor = (int*)(ws + L.bcursor);
    w.scan_tmp = (int*)(ws + L.scan_tmp);
    w.scan_tmp_len = L.scan_len;
    w.tile_cnt = (int*)(ws + L.tile_cnt);
    w.tile_off = (int*)(ws + L.tile_off);
    w.n_tiles = L.n_tiles;
    w.cell_start = (int*)(ws + L.cell_start);
    w.tmp = (float4*)(ws + L.tmp);
    w.sorted = (float4*)(ws + L.sorted);
    w.parent = (int*)(ws + L.parent);
    w.minorig = (int*)(ws + L.minorig);
    w.cnt = (int*)(ws + L.cnt);
    w.dense_list = (int64_t*)(ws + L.dense_list);
    w.n_dense = (int*)(ws + L.n_dense);
    w.dense_root = (int*)(ws + L.dense_root);
    w.out_cursor = (int*)(ws + L.out_cursor);
    w.team_list = (int64_t*)(ws + L.team_list);
    w.n_team = (int*)(ws + L.n_team);
    w.n_team_hi = (int*)(ws + L.n_team_hi);
    w.team_cap = L.team_cap;
    w.big_list = (int64_t*)(ws + L.big_list);
    w.n_big = (int*)(ws + L.n_big);

    cudaError_t e = cudaMemcpy(ws + L.boxes, boxes.data(), sizeof(BoxDev) * nbox, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(ws + L.p0, h->p0.data(), 8 * (size_t)nbox, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(ws + L.brick0, h->brick0.data(), 8 * (size_t)nbox, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        fof_destroy(h);
        return cuda_rc(e);
    }
    *out = h;
    return FOF_OK;
}

UfArgs uf_args(const fof_plan* h)
{
    UfArgs u;
    u.cap = h->retry_cap;
    u.err = &h->w.status->err;
    u.find = h->find_variant;
    u.link = h->link_order;
    u.var = (u.find != 0 || u.link != 0 || h->force_var) ? 1 : 0;
    return u;
}

// Linking on the binned particles: self tasks of team cells, dense cells,
// then the rest (shared by fof_link and fof_relink).
int enqueue_linking(fof_plan* h, cudaStream_t s)
{
    const Geometry& g = h->g;
    const Work& w = h->w;
    const UfArgs uf = uf_args(h);
    phase_begin(h, kPhTeamSelf, s);
    FOF_TRY(launch_team_self(g, w, s));
    phase_end(h, kPhTeamSelf, s);
    phase_begin(h, kPhBigSort, s);
    FOF_TRY(launch_big(g, w, h->dense_min, uf, false, s));
    phase_end(h, kPhBigSort, s);
    phase_begin(h, kPhDenseSelf, s);
    FOF_TRY(launch_dense(g, w, h->dense_min, uf, false, s));
    phase_end(h, kPhDenseSelf, s);
    phase_begin(h, kPhDensePairs, s);
    FOF_TRY(launch_dense(g, w, h->dense_min, uf, true, s));
    phase_end(h, kPhDensePairs, s);
    phase_begin(h, kPhBigPairs, s);
    FOF_TRY(launch_big(g, w, h->dense_min, uf, true, s));
    phase_end(h, kPhBigPairs, s);
    phase_begin(h, kPhLink, s);
    FOF_TRY(launch_link(g, w, h->dense_min, uf, s));
    phase_end(h, kPhLink, s);
    h->linked = true;
    return FOF_OK;
}

int enqueue_link(fof_plan* h, const float* pos, cudaStream_t s)
{
    const Geometry& g = h->g;
    const Work& w = h->w;
    const UfArgs uf = uf_args(h);
    FOF_TRY(cudaMemsetAsync(h->results_dev, 0, h->rl.bytes, s));
    if (g.total_n == 0) {
        h->linked = true;
        return FOF_OK;
    }
    FOF_TRY(cudaMemsetAsync(w.bcount, 0, 4 * (size_t)(g.total_bricks + 1), s));
    FOF_TRY(cudaMemsetAsync(w.bcursor, 0, 4 * (size_t)(g.total_bricks + 1), s));
    phase_begin(h, kPhBinCount, s);
    FOF_TRY(launch_bin_count(pos, g, w, s));
    phase_end(h, kPhBinCount, s);
    phase_begin(h, kPhScanBricks, s);
    FOF_TRY(launch_scan(w.bcount, w.bstart, g.total_bricks, w.scan_tmp, w.scan_tmp_len, s));
    phase_end(h, kPhScanBricks, s);
    phase_begin(h, kPhBinScatter, s);
    FOF_TRY(launch_bin_scatter(pos, g, w, s));
    phase_end(h, kPhBinScatter, s);
    FOF_TRY(cudaMemsetAsync(w.n_dense, 0, 4, s));
    FOF_TRY(cudaMemsetAsync(w.n_team, 0, 4, s));
    FOF_TRY(cudaMemsetAsync(w.n_team_hi, 0, 4, s));
    FOF_TRY(cudaMemsetAsync(w.n_big, 0, 4, s));
    phase_begin(h, kPhBrickSort, s);
    FOF_TRY(launch_brick_sort(g, w, h->dense_min, s));
    phase_end(h, kPhBrickSort, s);
    int rc_ = enqueue_linking(h, s);
    if (rc_ != FOF_OK)
        return rc_;
    h->binned = true;
    return FOF_OK;
}

int enqueue_groups(fof_plan* h, int32_t* ids, int32_t* sizes, fof_group* cat, int64_t cap,
                   int32_t min_size, cudaStream_t s)
{
    const Geometry& g = h->g;
    const Work& w = h->w;
    if (g.total_n > 0) {
        // status.err is kept from fof_link; counts start from zero
        FOF_TRY(cudaMemsetAsync(h->results_dev + h->rl.groups_off, 0,
                                h->rl.bytes - h->rl.groups_off, s));
        FOF_TRY(cudaMemsetAsync(w.tile_cnt, 0, 4 * (size_t)(w.n_tiles + 1), s));
        FOF_TRY(cudaMemsetAsync(w.out_cursor, 0, 4 * (size_t)((g.total_n >> kOutChunkLog) + 2), s));
        phase_begin(h, kPhFinalize, s);
        FOF_TRY(launch_finalize(g, w, uf_args(h), h->size_count, s));
        phase_end(h, kPhFinalize, s);
        phase_begin(h, kPhOutputs, s);
        FOF_TRY(launch_outputs(g, w, ids, sizes, min_size, s));
        phase_end(h, kPhOutputs, s);
        phase_begin(h, kPhCatalogue, s);
        FOF_TRY(launch_catalogue(g, w, sizes, min_size, (int2*)cat, cap, s));
        phase_end(h, kPhCatalogue, s);
    }
    FOF_TRY(cudaMemcpyAsync(h->results_host, h->results_dev, h->rl.bytes, cudaMemcpyDeviceToHost, s));
    h->pending = true;
    h->last_cap = cat ? cap : INT64_MAX;     // no catalogue wanted: no capacity error
    return FOF_OK;
}

int read_result(fof_plan* h, int64_t* n_groups, int64_t* n_cat, cudaStream_t s)
{
    if (!h->pending)
        return FOF_ERR_STATE;
    FOF_TRY(cudaStreamSynchronize(s));
    h->pending = false;
    collect_times(h);
    const Status* st = (const Status*)(h->results_host + h->rl.status_off);
    const long long* ng = (const long long*)(h->results_host + h->rl.groups_off);
    const long long* nk = (const long long*)(h->results_host + h->rl.cat_off);
    for (int i = 0; i < h->nbox; ++i) {
        if (n_groups) n_groups[i] = ng[i];
        if (n_cat) n_cat[i] = nk[i];
    }
    if (st->err & kErrInternal)
        return FOF_ERR_INTERNAL;
    if (st->err & kErrRange)
        return FOF_ERR_RANGE;
    if (st->err & kErrTimeout)
        return FOF_ERR_TIMEOUT;
    if (st->n_cat_total > h->last_cap)
        return FOF_ERR_CAPACITY;
    return FOF_OK;
}

int check_out_args(fof_plan* h, int32_t* ids, int32_t* sizes, fof_group* cat, int64_t cap)
{
    if (!h || cap < 0)
        return FOF_ERR_ARG;
    if (h->g.total_n > 0 && (!ids || !sizes))
        return FOF_ERR_ARG;
    if (cap > 0 && !cat)
        return FOF_ERR_ARG;
    return FOF_OK;
}

}  // namespace

// ==========================================================================
// C ABI
// ==========================================================================

extern "C" {

int fof_create(double box, double l_x, int64_t n, fof_handle* out)
{
    return create_plan(1, &box, &l_x, &n, nullptr, nullptr, 0, out);
}

int fof_create_ex(double box, double l_x, int64_t n, const fof_options* opt, void* workspace_dev,
                  size_t workspace_bytes, fof_handle* out)
{
    return create_plan(1, &box, &l_x, &n, opt, workspace_dev, workspace_bytes, out);
}

size_t fof_workspace_bytes(double box, double l_x, int64_t n, const fof_options* opt)
{
    return fof_batch_workspace_bytes(1, &box, &l_x, &n, opt);
}

int fof_batch_create(int32_t nbox, const double* box, const double* l_x, const int64_t* n,
                     const fof_options* opt, void* workspace_dev, size_t workspace_bytes,
                     fof_handle* out)
{
    return create_plan(nbox, box, l_x, n, opt, workspace_dev, workspace_bytes, out);
}

size_t fof_batch_workspace_bytes(int32_t nbox, const double* box, const double* l_x, const int64_t* n,
                                 const fof_options* opt)
{
    std::vector<BoxDev> boxes;
    int64_t tn, tb, tc;
    if (setup_batch(nbox, box, l_x, n, opt, boxes, tn, tb, tc) != FOF_OK)
        return 0;
    return layout(nbox, tn, tb, tc, dense_min_of(opt)).total;
}

int fof_link(fof_handle h, const float* pos_dev, void* stream)
{
    if (!h || (h->g.total_n > 0 && !pos_dev))
        return FOF_ERR_ARG;
    return enqueue_link(h, pos_dev, (cudaStream_t)stream);
}

int fof_relink(fof_handle h, const float* pos_dev, int32_t* path_out, void* stream)
{
    if (!h || (h->g.total_n > 0 && !pos_dev))
        return FOF_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const Geometry& g = h->g;
    const Work& w = h->w;
    int path = 2;
    if (h->binned && !h->capturing && g.total_n > 0) {
        // which particles left their cell or brick: one flag word, read back
        FOF_TRY(cudaMemsetAsync(h->results_dev, 0, h->rl.bytes, s));
        phase_begin(h, kPhBinCount, s);
        FOF_TRY(launch_relink_check(pos_dev, g, w, &w.status->pad, s));
        phase_end(h, kPhBinCount, s);
        FOF_TRY(cudaMemcpyAsync(h->results_host, h->results_dev, sizeof(Status), cudaMemcpyDeviceToHost, s));
        FOF_TRY(cudaStreamSynchronize(s));
        const Status* st = (const Status*)h->results_host;
        if (st->err == 0 && (st->pad & 2) == 0)
            path = (st->pad & 1) ? 1 : 0;
    }
    h->binned = false;
    if (path == 2) {
        int rc = enqueue_link(h, pos_dev, s);
        if (rc != FOF_OK)
            return rc;
    } else {
        if (path == 1) {
            // every particle kept its brick: the slots are still grouped by
            // brick, so the per-brick cell sort runs on the new positions
            FOF_TRY(cudaMemsetAsync(w.n_dense, 0, 4, s));
            FOF_TRY(cudaMemsetAsync(w.n_team, 0, 4, s));
            FOF_TRY(cudaMemsetAsync(w.n_team_hi, 0, 4, s));
            FOF_TRY(cudaMemsetAsync(w.n_big, 0, 4, s));
            phase_begin(h, kPhBrickSort, s);
            FOF_TRY(launch_brick_sort(g, w, h->dense_min, s));
            phase_end(h, kPhBrickSort, s);
        } else {
            // every particle kept its cell: cells, starts and lists stand
            phase_begin(h, kPhBrickSort, s);
            FOF_TRY(launch_forest_init(g, w, s));
            phase_end(h, kPhBrickSort, s);
        }
        int rc = enqueue_linking(h, s);
        if (rc != FOF_OK)
            return rc;
        h->binned = true;
    }
    h->last_relink_path = path;
    if (path_out)
        *path_out = path;
    return FOF_OK;
}

int fof_groups_async(fof_handle h, int32_t* ids_dev, int32_t* sizes_dev, fof_group* catalogue_dev,
                     int64_t cat_capacity, int32_t min_size, void* stream)
{
    int rc = check_out_args(h, ids_dev, sizes_dev, catalogue_dev, cat_capacity);
    if (rc != FOF_OK)
        return rc;
    if (!h->linked)
        return FOF_ERR_STATE;
    return enqueue_groups(h, ids_dev, sizes_dev, catalogue_dev, cat_capacity, min_size,
                          (cudaStream_t)stream);
}

int fof_result(fof_handle h, int64_t* n_groups_out, int64_t* n_cat_out, void* stream)
{
    if (!h)
        return FOF_ERR_ARG;
    return read_result(h, n_groups_out, n_cat_out, (cudaStream_t)stream);
}

int fof_groups(fof_handle h, int32_t* ids_dev, int32_t* sizes_dev, fof_group* catalogue_dev,
               int64_t cat_capacity, int32_t min_size, int64_t* n_groups_out, int64_t* n_cat_out,
               void* stream)
{
    int rc = fof_groups_async(h, ids_dev, sizes_dev, catalogue_dev, cat_capacity, min_size, stream);
    if (rc != FOF_OK)
        return rc;
    return read_result(h, n_groups_out, n_cat_out, (cudaStream_t)stream);
}

int fof_run_host(fof_handle h, const float* pos_host, int32_t* ids_host, int32_t* sizes_host,
                 fof_group* catalogue_host, int64_t cat_capacity, int32_t min_size,
                 int64_t* n_groups_out, int64_t* n_cat_out, void* stream)
{
    if (!h || cat_capacity < 0 || (h->g.total_n > 0 && (!pos_host || !ids_host || !sizes_host)) ||
        (cat_capacity > 0 && !catalogue_host))
        return FOF_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = h->g.total_n;
    if (n > 0 && !h->pos_d) {
        if (cudaMalloc((void**)&h->pos_d, 12 * (size_t)n) != cudaSuccess ||
            cudaMalloc((void**)&h->ids_d, 4 * (size_t)n) != cudaSuccess ||
            cudaMalloc((void**)&h->sizes_d, 4 * (size_t)n) != cudaSuccess) {
            cudaGetLastError();
            return FOF_ERR_OOM;
        }
    }
    if (cat_capacity > h->cat_d_cap) {
        if (h->cat_d) cudaFree(h->cat_d);
        h->cat_d = nullptr;
        h->cat_d_cap = 0;
        if (cudaMalloc((void**)&h->cat_d, 8 * (size_t)cat_capacity) != cudaSuccess) {
            cudaGetLastError();
            return FOF_ERR_OOM;
        }
        h->cat_d_cap = cat_capacity;
    }
    if (n > 0)
        FOF_TRY(cudaMemcpyAsync(h->pos_d, pos_host, 12 * (size_t)n, cudaMemcpyHostToDevice, s));
    int rc = enqueue_link(h, h->pos_d, s);
    if (rc != FOF_OK)
        return rc;
    rc = enqueue_groups(h, h->ids_d, h->sizes_d, (fof_group*)h->cat_d, cat_capacity, min_size, s);
    if (rc != FOF_OK)
        return rc;
    if (n > 0) {
        FOF_TRY(cudaMemcpyAsync(ids_host, h->ids_d, 4 * (size_t)n, cudaMemcpyDeviceToHost, s));
        FOF_TRY(cudaMemcpyAsync(sizes_host, h->sizes_d, 4 * (size_t)n, cudaMemcpyDeviceToHost, s));
    }
    std::vector<int64_t> ng(h->nbox), nk(h->nbox);
    rc = read_result(h, ng.data(), nk.data(), s);
    if (rc != FOF_OK && rc != FOF_ERR_CAPACITY)
        return rc;
    const Status* st = (const Status*)(h->results_host + h->rl.status_off);
    int64_t total = st->n_cat_total;
    int64_t ncopy = total < cat_capacity ? total : cat_capacity;
    if (ncopy > 0) {
        FOF_TRY(cudaMemcpyAsync(catalogue_host, h->cat_d, 8 * (size_t)ncopy, cudaMemcpyDeviceToHost, s));
        FOF_TRY(cudaStreamSynchronize(s));
    }
    for (int i = 0; i < h->nbox; ++i) {
        if (n_groups_out) n_groups_out[i] = ng[i];
        if (n_cat_out) n_cat_out[i] = nk[i];
    }
    return rc;
}

int fof_run_host_many(fof_handle h, int32_t nsteps, const float* const* pos_host, int32_t* const* ids_host,
                      int32_t* const* sizes_host, fof_group* const* catalogue_host, int64_t cat_capacity,
                      int32_t min_size, int64_t* n_groups_out, int64_t* n_cat_out, void* stream)
{
    if (!h || nsteps < 0 || cat_capacity < 0 || (nsteps > 0 && (!pos_host || !ids_host || !sizes_host)) ||
        (cat_capacity > 0 && !catalogue_host))
        return FOF_ERR_ARG;
    const int64_t n = h->g.total_n;
    for (int k = 0; k < nsteps; ++k)
        if ((n > 0 && (!pos_host[k] || !ids_host[k] || !sizes_host[k])) ||
            (cat_capacity > 0 && !catalogue_host[k]))
            return FOF_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    // staging, streams and events on first use (kept by the handle)
    if (!h->copy_in) {
        FOF_TRY(cudaStreamCreateWithFlags(&h->copy_in, cudaStreamNonBlocking));
        FOF_TRY(cudaStreamCreateWithFlags(&h->copy_out, cudaStreamNonBlocking));
        for (int b = 0; b < 2; ++b) {
            FOF_TRY(cudaEventCreateWithFlags(&h->ev_h2d[b], cudaEventDisableTiming));
            FOF_TRY(cudaEventCreateWithFlags(&h->ev_comp[b], cudaEventDisableTiming));
            FOF_TRY(cudaEventCreateWithFlags(&h->ev_d2h[b], cudaEventDisableTiming));
        }
    }
    for (int b = 0; b < 2 && n > 0; ++b)
        if (!h->pos2[b]) {
            if (cudaMalloc((void**)&h->pos2[b], 12 * (size_t)n) != cudaSuccess ||
                cudaMalloc((void**)&h->ids2[b], 4 * (size_t)n) != cudaSuccess ||
                cudaMalloc((void**)&h->sizes2[b], 4 * (size_t)n) != cudaSuccess) {
                cudaGetLastError();
                return FOF_ERR_OOM;
            }
        }
    if (cat_capacity > h->cat2_cap) {
        FOF_TRY(cudaDeviceSynchronize());       // the old catalogue buffers may be in use
        for (int b = 0; b < 2; ++b) {
            if (h->cat2[b]) cudaFree(h->cat2[b]);
            h->cat2[b] = nullptr;
        }
        h->cat2_cap = 0;
        for (int b = 0; b < 2; ++b)
            if (cudaMalloc((void**)&h->cat2[b], 8 * (size_t)cat_capacity) != cudaSuccess) {
                cudaGetLastError();
                return FOF_ERR_OOM;
            }
        h->cat2_cap = cat_capacity;
    }
    auto drain = [&]() {
        cudaStreamSynchronize(h->copy_in);
        cudaStreamSynchronize(s);
        cudaStreamSynchronize(h->copy_out);
    };
    auto h2d = [&](int k) -> cudaError_t {
        const int b = k & 1;
        // the buffer was last read by step k - 2's binning
        cudaError_t e = cudaStreamWaitEvent(h->copy_in, h->ev_comp[b], 0);
        if (e == cudaSuccess && n > 0)
            e = cudaMemcpyAsync(h->pos2[b], pos_host[k], 12 * (size_t)n, cudaMemcpyHostToDevice, h->copy_in);
        if (e == cudaSuccess)
            e = cudaEventRecord(h->ev_h2d[b], h->copy_in);
        return e;
    };
    int result = FOF_OK;
    if (nsteps > 0) {
        cudaError_t e = h2d(0);
        if (e != cudaSuccess) { drain(); return cuda_rc(e); }
    }
    std::vector<int64_t> ng(h->nbox), nk(h->nbox);
    for (int k = 0; k < nsteps; ++k) {
        const int b = k & 1;
        cudaError_t e = cudaSuccess;
        if (k + 1 < nsteps)
            e = h2d(k + 1);                      // the next input moves while this one runs
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->ev_h2d[b], 0);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->ev_d2h[b], 0);   // step k - 2's outputs are out
        if (e != cudaSuccess) { drain(); return cuda_rc(e); }
        int rc = enqueue_link(h, h->pos2[b], s);
        if (rc == FOF_OK)
            rc = enqueue_groups(h, h->ids2[b], h->sizes2[b], (fof_group*)h->cat2[b], cat_capacity, min_size, s);
        if (rc == FOF_OK && cudaEventRecord(h->ev_comp[b], s) != cudaSuccess)
            rc = FOF_ERR_CUDA;
        if (rc != FOF_OK) { drain(); return rc; }
        rc = read_result(h, ng.data(), nk.data(), s);
        if (rc != FOF_OK && rc != FOF_ERR_CAPACITY) { drain(); return rc; }
        if (rc == FOF_ERR_CAPACITY)
            result = FOF_ERR_CAPACITY;
        const Status* st = (const Status*)(h->results_host + h->rl.status_off);
        const int64_t ncopy = st->n_cat_total < cat_capacity ? st->n_cat_total : cat_capacity;
        e = cudaStreamWaitEvent(h->copy_out, h->ev_comp[b], 0);
        if (e == cudaSuccess && n > 0)
            e = cudaMemcpyAsync(ids_host[k], h->ids2[b], 4 * (size_t)n, cudaMemcpyDeviceToHost, h->copy_out);
        if (e == cudaSuccess && n > 0)
            e = cudaMemcpyAsync(sizes_host[k], h->sizes2[b], 4 * (size_t)n, cudaMemcpyDeviceToHost, h->copy_out);
        if (e == cudaSuccess && ncopy > 0)
            e = cudaMemcpyAsync(catalogue_host[k], h->cat2[b], 8 * (size_t)ncopy, cudaMemcpyDeviceToHost,
                                h->copy_out);
        if (e == cudaSuccess) e = cudaEventRecord(h->ev_d2h[b], h->copy_out);
        if (e != cudaSuccess) { drain(); return cuda_rc(e); }
        for (int i = 0; i < h->nbox; ++i) {
            if (n_groups_out) n_groups_out[(int64_t)k * h->nbox + i] = ng[i];
            if (n_cat_out) n_cat_out[(int64_t)k * h->nbox + i] = nk[i];
        }
    }
    FOF_TRY(cudaStreamSynchronize(h->copy_out));
    return result;
}

int fof_graph_build(fof_handle h, const float* pos_dev, int32_t* ids_dev, int32_t* sizes_dev,
                    fof_group* catalogue_dev, int64_t cat_capacity, int32_t min_size, void* stream)
{
    int rc = check_out_args(h, ids_dev, sizes_dev, catalogue_dev, cat_capacity);
    if (rc != FOF_OK)
        return rc;
    if (!stream || (h->g.total_n > 0 && !pos_dev))
        return FOF_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (h->gexec) {
        cudaGraphExecDestroy(h->gexec);
        h->gexec = nullptr;
    }
    FOF_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    h->capturing = true;
    rc = enqueue_link(h, pos_dev, s);
    if (rc == FOF_OK)
        rc = enqueue_groups(h, ids_dev, sizes_dev, catalogue_dev, cat_capacity, min_size, s);
    h->capturing = false;
    h->pending = false;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &graph);
    if (rc != FOF_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess)
        return cuda_rc(e);
    e = cudaGraphInstantiate(&h->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        h->gexec = nullptr;
        return cuda_rc(e);
    }
    h->graph_cap = catalogue_dev ? cat_capacity : INT64_MAX;
    return FOF_OK;
}

int fof_graph_launch(fof_handle h, void* stream)
{
    if (!h || !h->gexec)
        return h ? FOF_ERR_STATE : FOF_ERR_ARG;
    FOF_TRY(cudaGraphLaunch(h->gexec, (cudaStream_t)stream));
    h->linked = true;
    h->pending = true;
    h->last_cap = h->graph_cap;
    // a graph replays every phase once
    for (int k = 0; k < kNumPhases; ++k) {
        if (h->g.total_n > 0) {
            h->launches += kPhaseLaunches[k];
            h->phase[k].launches += kPhaseLaunches[k];
        }
    }
    return FOF_OK;
}

int fof_box_geometry(double box, double l_x, int64_t n, const fof_options* opt, fof_geometry* out)
{
    if (!out)
        return FOF_ERR_ARG;
    BoxDev b;
    int rc = setup_box(box, l_x, n, opt, b);
    if (rc != FOF_OK)
        return rc;
    out->cells_per_axis = b.nc;
    out->brick_cells = b.r;
    out->bricks_per_axis = b.nb;
    out->sub_cells = b.q;
    out->fine_per_axis = b.nf;
    out->inv_fine = b.inv_hf;
    out->xmax = b.xmax;
    out->t_lo = b.t_lo;
    out->t_hi = b.t_hi;
    out->bb_reach2 = b.bb_reach2;
    return FOF_OK;
}

int fof_plan_info(fof_handle h, int32_t b, int32_t* cells_per_axis, int32_t* brick_cells,
                  int32_t* bricks_per_axis)
{
    if (!h || b < 0 || b >= h->nbox)
        return FOF_ERR_ARG;
    const BoxDev& x = h->boxes[b];
    if (cells_per_axis) *cells_per_axis = x.nc;
    if (brick_cells) *brick_cells = x.r;
    if (bricks_per_axis) *bricks_per_axis = x.nb;
    return FOF_OK;
}

int fof_set_timing(fof_handle h, int enable)
{
    if (!h)
        return FOF_ERR_ARG;
    h->timing = enable != 0;
    return FOF_OK;
}

int fof_phase_times(fof_handle h, double* ms, int64_t* launches, const char** names, int max)
{
    if (!h)
        return -FOF_ERR_ARG;
    collect_times(h);
    int m = max < kNumPhases ? max : kNumPhases;
    for (int k = 0; k < m; ++k) {
        if (ms) ms[k] = h->phase[k].ms;
        if (launches) launches[k] = h->phase[k].launches;
        if (names) names[k] = kPhaseNames[k];
    }
    return kNumPhases;
}

int fof_reset_times(fof_handle h)
{
    if (!h)
        return FOF_ERR_ARG;
    for (int k = 0; k < kNumPhases; ++k) {
        h->phase[k].ms = 0.0;
        h->phase[k].launches = 0;
        h->phase[k].pending = false;
    }
    return FOF_OK;
}

int64_t fof_kernel_launches(fof_handle h)
{
    return h ? h->launches : -1;
}

void fof_destroy(fof_handle h)
{
    if (!h)
        return;
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    for (int k = 0; k < kNumPhases; ++k) {
        if (h->phase[k].ev0) cudaEventDestroy(h->phase[k].ev0);
        if (h->phase[k].ev1) cudaEventDestroy(h->phase[k].ev1);
    }
    for (int b = 0; b < 2; ++b) {
        if (h->pos2[b]) cudaFree(h->pos2[b]);
        if (h->ids2[b]) cudaFree(h->ids2[b]);
        if (h->sizes2[b]) cudaFree(h->sizes2[b]);
        if (h->cat2[b]) cudaFree(h->cat2[b]);
        if (h->ev_h2d[b]) cudaEventDestroy(h->ev_h2d[b]);
        if (h->ev_comp[b]) cudaEventDestroy(h->ev_comp[b]);
        if (h->ev_d2h[b]) cudaEventDestroy(h->ev_d2h[b]);
    }
    if (h->copy_in) cudaStreamDestroy(h->copy_in);
    if (h->copy_out) cudaStreamDestroy(h->copy_out);
    if (h->pos_d) cudaFree(h->pos_d);
    if (h->ids_d) cudaFree(h->ids_d);
    if (h->sizes_d) cudaFree(h->sizes_d);
    if (h->cat_d) cudaFree(h->cat_d);
    if (h->own_ws && h->ws) cudaFree(h->ws);
    pinned_free(h->results_host, h->results_from_slab);
    delete h;
}

const char* fof_strerror(int code)
{
    switch (code) {
    case FOF_OK: return "ok";
    case FOF_ERR_ARG: return "invalid argument";
    case FOF_ERR_RANGE: return "position outside [0, box) or not finite";
    case FOF_ERR_CAPACITY: return "catalogue larger than its capacity";
    case FOF_ERR_STATE: return "call out of order (fof_groups before fof_link)";
    case FOF_ERR_OOM: return "out of memory";
    case FOF_ERR_CUDA: return "CUDA runtime error";
    case FOF_ERR_TIMEOUT: return "union retry limit reached";
    case FOF_ERR_INTERNAL: return "internal consistency check failed";
    case FOF_ERR_TOO_LARGE: return "problem needs more than the fixed scratch of fof_run_noalloc";
    default: return "unknown error";
    }
}

}  // extern "C"

// ==========================================================================
// fof_run_noalloc: one box, whole pipeline, no allocation of any kind.
//
// For callers that cannot allocate device memory: a host application that
// owns (and has already handed out) all GPU memory, or a loop that must not
// call cudaMalloc/cudaFree because they synchronise the device.  The
// workspace is the file-scope array below instead of a plan's allocation.
// ==========================================================================

namespace {

constexpr size_t kNoallocScratchBytes = (size_t)32 << 20;   // 32 MiB per device
constexpr int kNoallocMaxDevices = 64;

// Held by every GPU that loads the library, until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_noalloc_mu;
char* g_noalloc_ptr[kNoallocMaxDevices];                 // device address of the array, per device
unsigned long long g_noalloc_ctx[kNoallocMaxDevices];    // id of the context it belongs to

// The id of the calling thread's current context (driver entry points looked
// up through the runtime, so the library does not link the driver library).
// Context ids are unique for the life of the process: after a device reset
// the new context has a new id.
bool current_context_id(unsigned long long* id)
{
    typedef int (*GetCurrentFn)(void** ctx);
    typedef int (*GetIdFn)(void* ctx, unsigned long long* id);
    static GetCurrentFn get_current = nullptr;
    static GetIdFn get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {
        looked_up = true;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", (void**)&get_current, 12000, cudaEnableDefault,
                                             &q1) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess)
            get_current = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", (void**)&get_id, 12000, cudaEnableDefault, &q2) !=
                cudaSuccess ||
            q2 != cudaDriverEntryPointSuccess)
            get_id = nullptr;
        cudaGetLastError();
    }
    void* ctx = nullptr;
    if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx)
        return false;
    return get_id(ctx, id) == 0;
}

// Device address of the scratch array for the current device.  In host code
// the array's name is only a stand-in, so the address is looked up with
// cudaGetSymbolAddress, with that device current, once per device and
// context: a later call in the same context reuses it, and a call after the
// context was re-created (cudaDeviceReset) looks it up again instead of using
// an address of the old context.
int noalloc_scratch(char** out)
{
    int dev = 0;
    FOF_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoallocMaxDevices)
        return FOF_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    unsigned long long id = 0;
    if (g_noalloc_ptr[dev] && current_context_id(&id) && id == g_noalloc_ctx[dev]) {
        *out = g_noalloc_ptr[dev];
        return FOF_OK;
    }
    void* p = nullptr;
    FOF_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    if (current_context_id(&id)) {              // cache only what can be re-validated
        g_noalloc_ptr[dev] = (char*)p;
        g_noalloc_ctx[dev] = id;
    } else {
        g_noalloc_ptr[dev] = nullptr;
    }
    *out = (char*)p;
    return FOF_OK;
}

}  // namespace

extern "C" int fof_run_noalloc(double box, double l_x, int64_t n, const float* pos_dev,
                               int32_t* ids_dev, int32_t* sizes_dev, fof_group* catalogue_dev,
                               int64_t cat_capacity, int32_t min_size, int64_t* n_groups_out,
                               int64_t* n_cat_out, void* stream)
{
    if (cat_capacity < 0 || (cat_capacity > 0 && !catalogue_dev))
        return FOF_ERR_ARG;
    BoxDev b;
    int rc = setup_box(box, l_x, n, nullptr, b);
    if (rc != FOF_OK)
        return rc;
    const int64_t tb = (int64_t)b.nb * b.nb * b.nb;
    const int64_t tc = tb * (int64_t)b.r * b.r * b.r;
    const Layout L = layout(1, n, tb, tc);
    if (L.total > kNoallocScratchBytes)
        return FOF_ERR_TOO_LARGE;
    if (n > 0 && (!pos_dev || !ids_dev || !sizes_dev))
        return FOF_ERR_ARG;
    char* ws = nullptr;
    rc = noalloc_scratch(&ws);
    if (rc != FOF_OK)
        return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const ResultsLayout rl = results_layout(1);

    Geometry g{};
    g.boxes = (const BoxDev*)(ws + L.boxes);
    g.box_p0 = (const int64_t*)(ws + L.p0);
    g.box_brick0 = (const int64_t*)(ws + L.brick0);
    g.nbox = 1;
    g.total_n = n;
    g.total_bricks = tb;
    g.total_cells = tc;
    Work w{};
    char* res = ws + L.results;
    w.status = (Status*)(res + rl.status_off);
    w.n_groups = (unsigned long long*)(res + rl.groups_off);
    w.n_cat = (unsigned long long*)(res + rl.cat_off);
    w.bcount = (int*)(ws + L.bcount);
    w.bstart = (int*)(ws + L.bstart);
    w.bcursor = (int*)(ws + L.bcursor);
    w.scan_tmp = (int*)(ws + L.scan_tmp);
    w.scan_tmp_len = L.scan_len;
    w.tile_cnt = (int*)(ws + L.tile_cnt);
    w.tile_off = (int*)(ws + L.tile_off);
    w.n_tiles = L.n_tiles;
    w.cell_start = (int*)(ws + L.cell_start);
    w.tmp = (float4*)(ws + L.tmp);
    w.sorted = (float4*)(ws + L.sorted);
    w.parent = (int*)(ws + L.parent);
    w.minorig = (int*)(ws + L.minorig);
    w.cnt = (int*)(ws + L.cnt);
    w.dense_list = (int64_t*)(ws + L.dense_list);
    w.n_dense = (int*)(ws + L.n_dense);
    w.dense_root = (int*)(ws + L.dense_root);
    w.out_cursor = (int*)(ws + L.out_cursor);
    w.team_list = (int64_t*)(ws + L.team_list);
    w.n_team = (int*)(ws + L.n_team);
    w.n_team_hi = (int*)(ws + L.n_team_hi);
    w.team_cap = L.team_cap;
    w.big_list = (int64_t*)(ws + L.big_list);
    w.n_big = (int*)(ws + L.n_big);

    // The array keeps the previous call's contents: the box table is
    // rewritten and every counter that must start at zero is cleared here.
    const int64_t zero = 0;
    FOF_TRY(cudaMemcpyAsync(ws + L.boxes, &b, sizeof(BoxDev), cudaMemcpyHostToDevice, s));
    FOF_TRY(cudaMemcpyAsync(ws + L.p0, &zero, sizeof(zero), cudaMemcpyHostToDevice, s));
    FOF_TRY(cudaMemcpyAsync(ws + L.brick0, &zero, sizeof(zero), cudaMemcpyHostToDevice, s));
    FOF_TRY(cudaMemsetAsync(res, 0, rl.bytes, s));
    if (n > 0) {
        FOF_TRY(cudaMemsetAsync(w.bcount, 0, 4 * (size_t)(tb + 1), s));
        FOF_TRY(cudaMemsetAsync(w.bcursor, 0, 4 * (size_t)(tb + 1), s));
        FOF_TRY(cudaMemsetAsync(w.tile_cnt, 0, 4 * (size_t)(w.n_tiles + 1), s));
        FOF_TRY(cudaMemsetAsync(w.n_dense, 0, 4, s));
        FOF_TRY(cudaMemsetAsync(w.out_cursor, 0, 4 * (size_t)((n >> kOutChunkLog) + 2), s));
        FOF_TRY(launch_bin_count(pos_dev, g, w, s));
        FOF_TRY(launch_scan(w.bcount, w.bstart, tb, w.scan_tmp, w.scan_tmp_len, s));
        FOF_TRY(launch_bin_scatter(pos_dev, g, w, s));
        FOF_TRY(cudaMemsetAsync(w.n_team, 0, 4, s));
        FOF_TRY(cudaMemsetAsync(w.n_team_hi, 0, 4, s));
        FOF_TRY(cudaMemsetAsync(w.n_big, 0, 4, s));
        FOF_TRY(launch_brick_sort(g, w, kDefaultDenseMin, s));
        FOF_TRY(launch_team_self(g, w, s));
        UfArgs uf;
        uf.cap = kDefaultRetryCap;
        uf.err = &w.status->err;
        uf.find = 0;
        uf.link = 0;
        uf.var = 0;
        FOF_TRY(launch_big(g, w, kDefaultDenseMin, uf, false, s));
        FOF_TRY(launch_dense(g, w, kDefaultDenseMin, uf, false, s));
        FOF_TRY(launch_dense(g, w, kDefaultDenseMin, uf, true, s));
        FOF_TRY(launch_big(g, w, kDefaultDenseMin, uf, true, s));
        FOF_TRY(launch_link(g, w, kDefaultDenseMin, uf, s));
        FOF_TRY(launch_finalize(g, w, uf, 0, s));
        FOF_TRY(launch_outputs(g, w, ids_dev, sizes_dev, min_size, s));
        FOF_TRY(launch_catalogue(g, w, sizes_dev, min_size, (int2*)catalogue_dev, cat_capacity, s));
    }
    alignas(16) unsigned char host_res[128];
    FOF_TRY(cudaMemcpyAsync(host_res, res, rl.bytes, cudaMemcpyDeviceToHost, s));
    FOF_TRY(cudaStreamSynchronize(s));
    const Status* st = (const Status*)(host_res + rl.status_off);
    const long long* ng = (const long long*)(host_res + rl.groups_off);
    const long long* nk = (const long long*)(host_res + rl.cat_off);
    if (n_groups_out) *n_groups_out = ng[0];
    if (n_cat_out) *n_cat_out = nk[0];
    if (st->err & kErrInternal)
        return FOF_ERR_INTERNAL;
    if (st->err & kErrRange)
        return FOF_ERR_RANGE;
    if (st->err & kErrTimeout)
        return FOF_ERR_TIMEOUT;
    if (catalogue_dev && st->n_cat_total > cat_capacity)
        return FOF_ERR_CAPACITY;
    return FOF_OK;
}
