/*
 * fof.h -- C ABI of the GB300 Friends-of-Friends group finder.
 *
 * The library finds the Friends-of-Friends groups of float32 particle
 * positions in a periodic cubic box: the connected components of the graph
 * whose edges join particles at distance <= l_x (paper Sec. 1, footnote on
 * the graph definition; "at most l_x", abstract).  Particles without a
 * neighbour are groups of size one (Sec. 1).
 *
 * Method on the device (one GPU, sm_103a):
 *   fof_link    counting-sort binning of the particles into cells of side
 *               >= l_x (two-level: bricks, then cells inside each brick),
 *               self- and neighbour-cell link kernels, and a lock-free
 *               union-find forest in which the larger root is always hooked
 *               onto the smaller one with an atomic compare-and-swap, with
 *               path halving in Find (Sec. 2; Sec. 3.1; Sec. 3.2, CAS union;
 *               Sec. 3.4.3, compression of deep paths only).
 *   fof_groups  pointer-jumping finalisation of the forest, group sizes by
 *               atomic counting with roots excluded (Sec. 3.4.1 and 3.4.2),
 *               per-particle labels, the label-indexed size array and the
 *               catalogue of groups of at least min_size members.
 *
 * Link predicate (the paper leaves the arithmetic open; this is the reading
 * the library implements exactly): per axis d = (double)x_i - (double)x_j,
 * wrapped once by "if d > L/2: d -= L; else if d < -L/2: d += L"; then
 * s = (dx*dx + dy*dy) + dz*dz, each operation rounded to nearest in IEEE
 * double, no fused multiply-add; linked iff s <= l_x*l_x (rounded once).
 * The device evaluates this predicate exactly: a float32 pre-test with a
 * proven error bound settles clear cases, every other pair takes the
 * double-precision test above.
 *
 * Outputs (deterministic, independent of scheduling):
 *   ids[i]    smallest particle index of i's group (union-by-root onto the
 *             smaller offset makes the root the minimum, Sec. 2, Sec. 3.1);
 *   sizes[g]  number of members of the group labelled g, 0 where g is not a
 *             label (the paper's group_size indexed by the root, Sec. 3.4.1);
 *   catalogue (label, size) of every group with size >= max(min_size, 1),
 *             ascending label ("groups of length > 20", Sec. 4.1, is one
 *             such threshold).
 *
 * Conventions for every entry point:
 *   - Pointers named *_dev are device pointers (cudaMalloc, torch tensors on
 *     the GPU); *_host are host pointers (pinned memory is fastest).  The
 *     caller owns all of them.  Arrays are contiguous, int32 or float32,
 *     positions are [n][3] float32 (x, y, z per particle, AoS).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 *   - Functions return FOF_OK (0) or a FOF_ERR_* code; fof_strerror() names
 *     it.  No entry point throws, aborts or prints.
 *   - A handle must not be used from two host threads at once.
 */
#ifndef FOF_GB300_H
#define FOF_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    FOF_OK = 0,
    FOF_ERR_ARG = 1,       /* invalid argument (see each function)          */
    FOF_ERR_RANGE = 2,     /* a position is NaN, infinite or outside [0, L)  */
    FOF_ERR_CAPACITY = 3,  /* catalogue larger than its capacity             */
    FOF_ERR_STATE = 4,     /* fof_groups before fof_link, or similar order   */
    FOF_ERR_OOM = 5,       /* device or pinned-host allocation failed        */
    FOF_ERR_CUDA = 6,      /* a CUDA runtime call failed                     */
    FOF_ERR_TIMEOUT = 7,   /* a bounded retry loop ran out (union CAS)       */
    FOF_ERR_INTERNAL = 8,  /* a device-side consistency check failed         */
    FOF_ERR_TOO_LARGE = 9  /* problem exceeds fof_run_noalloc's fixed scratch */
};

typedef struct fof_plan *fof_handle;    /* opaque, owned by the library */

typedef struct {
    int32_t label;   /* smallest particle index of the group (box-local) */
    int32_t size;    /* number of members                                */
} fof_group;

/* Tuning knobs and method variants; a zero field selects the library's
 * default.  The variant fields exist to measure the paper's alternatives
 * against the default; every variant gives the same partition (exactly),
 * except tie_rule, which changes the graph at distance exactly l_x. */
typedef struct {
    int32_t cells_per_axis;  /* cells per box side; must keep side >= l_x   */
    int32_t brick_cells;     /* cells per brick side: 1, 2, 4, 8 or 16      */
    double occupancy;        /* target mean particles per cell (default 0.30) */
    int32_t dense_min;       /* cell occupancy from which a cell is split
                                into sub-cells and linked in shared memory
                                (default 256)                                */
    int32_t retry_cap;       /* max CAS attempts per union (default 2^20)    */
    int32_t team_min;        /* cell occupancy from which one warp links the
                                cell's particles as a team (default 10, >= 2) */
    int32_t tie_rule;        /* FOF_TIE_LE (0, default): linked iff the
                                distance is <= l_x (graph definition, Sec. 1
                                footnote; "at most", abstract); FOF_TIE_LT:
                                < l_x (the naive listing, Sec. 3.1)          */
    int32_t find_variant;    /* FOF_FIND_*: path compression of Find
                                (Sec. 3.4.3); default FOF_FIND_HALVE_DEEP    */
    int32_t size_count;      /* FOF_SIZE_*: how group sizes are counted
                                (Sec. 3.4.1); default FOF_SIZE_WARP          */
    int32_t link_order;      /* FOF_LINK_*: which root a Union hooks
                                (Sec. 3.1; Sec. 3.2); default FOF_LINK_MIN   */
    int32_t debug_flags;     /* FOF_DEBUG_* bits; 0 in production            */
    int32_t reserved[2];     /* must be 0                                    */
} fof_options;

/* tie_rule */
enum { FOF_TIE_LE = 0, FOF_TIE_LT = 1 };
/* find_variant: path compression during Find (Sec. 3.4.3) */
enum {
    FOF_FIND_HALVE_DEEP = 0, /* path halving, writing only where the path is at
                                least 2 deep (the paper's choice)            */
    FOF_FIND_HALVE_ALL = 1,  /* path halving at every depth (also rewrites the
                                parent of a depth-1 node with its own value) */
    FOF_FIND_FULL = 2,       /* full compression: a second pass points every
                                node of the path at the root                 */
    FOF_FIND_NONE = 3        /* no compression                               */
};
/* size_count: group sizes (Sec. 3.4.1, 3.4.2; roots never counted) */
enum {
    FOF_SIZE_WARP = 0,       /* equal roots aggregated per warp, one atomic each */
    FOF_SIZE_HASH = 1        /* per-block shared-memory hash table of (root,
                                count), flushed with one atomic per entry    */
};
/* link_order: which root Union hooks onto which */
enum {
    FOF_LINK_MIN = 0,        /* the larger root onto the smaller (union by root
                                onto the lower offset, Sec. 3.1)             */
    FOF_LINK_RANDOM = 1      /* randomised linking: the root of lower random
                                priority onto the other (Jayanti and Tarjan,
                                discussed in Sec. 3.2); the min-index labels
                                are then set by the label pass               */
};
/* debug_flags */
enum {
    FOF_DEBUG_UNION_NO_RETRY = 1, /* every Union gives up before its first
                                     attempt and reports FOF_ERR_TIMEOUT: a
                                     deterministic test of the retry cap     */
    FOF_DEBUG_VARIANT_KERNELS = 2 /* run the variant-capable kernels even with
                                     the default variants (the control when
                                     timing the variants)                    */
};

/* ---------------------------------------------------------------------- */
/* single box                                                              */
/* ---------------------------------------------------------------------- */

/* Plan for one periodic box of side `box` with linking length `l_x` and `n`
 * particles.  Allocates the device workspace (fof_workspace_bytes) and a
 * small pinned host block.  Errors: FOF_ERR_ARG if box is not finite and
 * > 0, l_x is not finite and > 0, l_x >= box/2, n < 0, n > 2^31 - 2, or out
 * is NULL; FOF_ERR_OOM; FOF_ERR_CUDA. */
int fof_create(double box, double l_x, int64_t n, fof_handle *out);

/* As fof_create with options (may be NULL).  If `workspace_dev` is not
 * NULL the plan uses that caller-owned device block of `workspace_bytes`
 * (at least fof_workspace_bytes(...), 256-byte aligned) and allocates no
 * device memory itself; the block must outlive the handle. */
int fof_create_ex(double box, double l_x, int64_t n, const fof_options *opt,
                  void *workspace_dev, size_t workspace_bytes, fof_handle *out);

/* Device bytes a plan needs (0 if the arguments are invalid). */
size_t fof_workspace_bytes(double box, double l_x, int64_t n, const fof_options *opt);

/* ---------------------------------------------------------------------- */
/* batch of independent boxes (the single box is the batch of one)         */
/* ---------------------------------------------------------------------- */

/* Plan for `nbox` boxes; box b has side box[b], linking length l_x[b] and
 * n[b] particles (same rules as fof_create for each; total particles must
 * stay <= 2^31 - 2).  Positions, ids and sizes of the boxes are
 * concatenated in box order; ids and labels are local to their box. */
int fof_batch_create(int32_t nbox, const double *box, const double *l_x,
                     const int64_t *n, const fof_options *opt,
                     void *workspace_dev, size_t workspace_bytes, fof_handle *out);

size_t fof_batch_workspace_bytes(int32_t nbox, const double *box, const double *l_x,
                                 const int64_t *n, const fof_options *opt);

/* ---------------------------------------------------------------------- */
/* running                                                                 */
/* ---------------------------------------------------------------------- */

/* Enqueue binning and linking of pos_dev ([sum n][3] float32, device) on
 * `stream`.  Asynchronous: returns once the kernels are enqueued; pos_dev
 * must stay valid until they finish.  Out-of-range positions are reported
 * by the next fof_groups (FOF_ERR_RANGE).  Errors: FOF_ERR_ARG (NULL
 * handle, NULL pos_dev with n > 0), FOF_ERR_CUDA. */
int fof_link(fof_handle h, const float *pos_dev, void *stream);

/* fof_link for particles that moved since the last fof_link or fof_relink
 * of this plan (the paper runs the group finder on-the-fly at fixed
 * intervals of a simulation, Sec. 1, and suggests re-using the existing
 * data structures): same arguments, results and errors as fof_link, with
 * pos_dev holding the SAME particles (same count and order) at new
 * positions.  The previous binned order is kept where it still holds:
 *   path 0: no particle left its cell -- positions are updated in place and
 *           the cells, cell starts and cell lists are re-used;
 *   path 1: particles changed cells but none left its brick (16^3 cells)
 *           -- only the per-brick cell sort runs again;
 *   path 2: otherwise (or with no previous binning) -- fof_link.
 * *path_out (may be NULL) receives the path taken.  Unlike fof_link it
 * waits once for `stream` (to read which path applies), so it cannot be
 * captured in a CUDA graph. */
int fof_relink(fof_handle h, const float *pos_dev, int32_t *path_out, void *stream);

/* Enqueue finalisation and outputs of the last fof_link, then wait for the
 * stream and report.  ids_dev and sizes_dev hold sum(n) int32 each;
 * catalogue_dev holds cat_capacity fof_group entries; NULL (with
 * cat_capacity 0) asks for no catalogue, whose counts are still reported
 * and never raise FOF_ERR_CAPACITY.  For a batch, the catalogue is concatenated in box
 * order, min_size applies to every box, and n_groups_out / n_cat_out
 * (host, may be NULL) receive one count per box.  If the catalogue has more
 * than cat_capacity entries in total, the first cat_capacity are written,
 * the counts are still reported and FOF_ERR_CAPACITY is returned.  Errors:
 * FOF_ERR_STATE (no fof_link yet), FOF_ERR_RANGE, FOF_ERR_TIMEOUT,
 * FOF_ERR_CAPACITY, FOF_ERR_ARG, FOF_ERR_CUDA. */
int fof_groups(fof_handle h, int32_t *ids_dev, int32_t *sizes_dev,
               fof_group *catalogue_dev, int64_t cat_capacity, int32_t min_size,
               int64_t *n_groups_out, int64_t *n_cat_out, void *stream);

/* fof_groups without the wait: counts and status stay on the device until
 * fof_result().  Together with fof_link this sequence can be captured in a
 * CUDA graph (it performs no host synchronisation and no allocation). */
int fof_groups_async(fof_handle h, int32_t *ids_dev, int32_t *sizes_dev,
                     fof_group *catalogue_dev, int64_t cat_capacity, int32_t min_size,
                     void *stream);

/* Wait for `stream` and report the status and counts of the last
 * fof_groups_async (same meaning and errors as fof_groups). */
int fof_result(fof_handle h, int64_t *n_groups_out, int64_t *n_cat_out, void *stream);

/* Whole pipeline from HOST buffers: copies pos_host to the device, runs
 * fof_link and fof_groups, and copies ids, sizes and the catalogue back
 * into ids_host, sizes_host and catalogue_host.  Device staging buffers
 * are allocated on the first call and kept by the handle.  Same errors as
 * fof_groups, plus FOF_ERR_OOM. */
int fof_run_host(fof_handle h, const float *pos_host, int32_t *ids_host, int32_t *sizes_host,
                 fof_group *catalogue_host, int64_t cat_capacity, int32_t min_size,
                 int64_t *n_groups_out, int64_t *n_cat_out, void *stream);

/* fof_run_host over `nsteps` inputs (for example the snapshots of a
 * simulation, each with this plan's particle count), pipelined: the
 * positions of step k+1 are copied in, on a copy stream, while step k
 * runs on `stream`, and the results of step k are copied out, on a second
 * copy stream, while step k+1 runs.  pos_host[k], ids_host[k],
 * sizes_host[k] and catalogue_host[k] are step k's host buffers (pinned
 * memory overlaps best); n_groups_out / n_cat_out (may be NULL) receive
 * nsteps x nbox counts, step-major.  Returns after every result is in host
 * memory.  Two device staging sets, the copy streams and their events are
 * made on the first call and kept by the handle.  Same errors as
 * fof_run_host; FOF_ERR_CAPACITY if any step's catalogue was cut. */
int fof_run_host_many(fof_handle h, int32_t nsteps, const float *const *pos_host,
                      int32_t *const *ids_host, int32_t *const *sizes_host,
                      fof_group *const *catalogue_host, int64_t cat_capacity, int32_t min_size,
                      int64_t *n_groups_out, int64_t *n_cat_out, void *stream);

/* ---------------------------------------------------------------------- */
/* CUDA graph of the whole pipeline                                        */
/* ---------------------------------------------------------------------- */

/* Capture fof_link + fof_groups_async with these buffers into a graph kept
 * by the handle (replacing any previous one).  `stream` must not be the
 * legacy default stream. */
int fof_graph_build(fof_handle h, const float *pos_dev, int32_t *ids_dev, int32_t *sizes_dev,
                    fof_group *catalogue_dev, int64_t cat_capacity, int32_t min_size,
                    void *stream);

/* Launch the captured graph on `stream`; read results with fof_result. */
int fof_graph_launch(fof_handle h, void *stream);

/* ---------------------------------------------------------------------- */
/* introspection                                                           */
/* ---------------------------------------------------------------------- */

/* Geometry the library derives for one box (host only, no device call).
 * Cells per axis nc, cells per brick side, bricks per axis; sub-cells per
 * cell side q (1 = cells are never split) and fine cells per axis nc*q;
 * inv_fine = float32(nc*q / box), so a coordinate's fine index is
 * min(nc*q - 1, (int)(x * inv_fine)) with a float32 multiply and its cell
 * index is the fine one divided by q; xmax = largest valid coordinate;
 * t_lo / t_hi = float32 squared-distance bounds of the pre-test; bb_reach2
 * bounds the float32 squared gap between a particle and the bounding box of
 * particles it can link to.
 * Returns FOF_OK or FOF_ERR_ARG (same rules as fof_create_ex). */
typedef struct {
    int32_t cells_per_axis, brick_cells, bricks_per_axis, sub_cells, fine_per_axis;
    float inv_fine, xmax, t_lo, t_hi;
    float bb_reach2;   /* squared float32 gap from a bounding box of particles
                          beyond which no particle has a partner */
} fof_geometry;

int fof_box_geometry(double box, double l_x, int64_t n, const fof_options *opt, fof_geometry *out);

/* Plan geometry of box b: cells per axis, cells per brick side, number of
 * bricks per axis.  Any pointer may be NULL. */
int fof_plan_info(fof_handle h, int32_t b, int32_t *cells_per_axis, int32_t *brick_cells,
                  int32_t *bricks_per_axis);

/* Per-phase device timing.  When enabled, every kernel phase is bracketed
 * by CUDA events on the launching stream; fof_phase_times() then returns,
 * for up to `max` phases, the summed milliseconds and launch counts since
 * the last reset, and names[k] (static strings).  Returns the number of
 * phases, or a negative FOF_ERR_* code. */
int fof_set_timing(fof_handle h, int enable);
int fof_phase_times(fof_handle h, double *ms, int64_t *launches, const char **names, int max);
int fof_reset_times(fof_handle h);

/* Number of kernel launches the handle has enqueued since creation. */
int64_t fof_kernel_launches(fof_handle h);

void fof_destroy(fof_handle h);
const char *fof_strerror(int code);

/* ---------------------------------------------------------------------- */
/* groups spanning several domains (one GPU per domain)                    */
/* ---------------------------------------------------------------------- */

/* The merge step of the distributed group finder (paper Sec. 3.3, Fig.
 * "Distributed Union-Find", steps 3-4; hash table of group ids, Sec. 3.4.1).
 * Every domain first finds the groups of its own particles plus a ghost
 * layer of width l_x, labels each local group with a globally unique id,
 * and lists links (a[k], b[k]) between ids that name the same group (for
 * example a ghost particle's id and the id of the local group holding it).
 * The links of all domains are gathered (all-gather), and this function runs
 * the union-find over the whole list, following indirect links through
 * third domains.  Sets are joined by size (Sec. 3.3); `weights` (may be
 * NULL with nweights 0) give the size of the ids in weight_ids, other ids
 * weigh 1 per first appearance.
 * For each query[k], label_out[k] receives the SMALLEST id of its merged
 * set (the id itself when it appears in no link or weight), and
 * weight_out[k] (may be NULL) the set's total weight (0 for such ids).
 * Host pointers, int64; nothing is kept between calls.  Host code only:
 * needs no GPU.  Errors: FOF_ERR_ARG (negative counts, NULL arrays with
 * non-zero counts), FOF_ERR_OOM. */
int fof_merge_links(int64_t npairs, const int64_t *a, const int64_t *b, int64_t nweights,
                    const int64_t *weight_ids, const int64_t *weights, int64_t nq,
                    const int64_t *query, int64_t *label_out, int64_t *weight_out);

/* ---------------------------------------------------------------------- */
/* allocation-free single-box run                                          */
/* ---------------------------------------------------------------------- */

/* The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory: a host application that owns, and has
 * already handed out, all GPU memory (N-body codes typically leave little
 * free for an on-the-fly group finder), or a time-step loop that must not
 * call cudaMalloc/cudaFree because they synchronise the whole device.
 *
 * Runs fof_link + fof_groups for ONE box with the same arguments, outputs
 * and errors as fof_create + fof_link + fof_groups, but allocates nothing:
 * no cudaMalloc/cudaFree, no pinned memory, no events, no plan.  The
 * workspace is a fixed 32 MiB array in the library's own device memory,
 * which every GPU that loads the library holds until the process exits.
 *   - Problems whose workspace (fof_workspace_bytes with NULL options)
 *     exceeds 32 MiB are rejected with FOF_ERR_TOO_LARGE, checked before any
 *     pointer; that is about 580,000 particles at the default occupancy.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current, and later calls in
 *     the same context reuse it; a call after the context was re-created
 *     (cudaDeviceReset) looks it up again.  Make the first call on a device,
 *     and the first after a reset, before any stream capture.
 *   - Every call on a device shares the one array and overwrites it (the
 *     call clears what must start at zero).  Calls whose GPU work overlaps,
 *     from several host threads or on several streams, race and give wrong
 *     results: serialise them.
 *   - Blocking: returns after the stream has finished the work. */
int fof_run_noalloc(double box, double l_x, int64_t n, const float *pos_dev,
                    int32_t *ids_dev, int32_t *sizes_dev, fof_group *catalogue_dev,
                    int64_t cat_capacity, int32_t min_size, int64_t *n_groups_out,
                    int64_t *n_cat_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* FOF_GB300_H */
