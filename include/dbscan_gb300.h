/*
 * dbscan_gb300.h -- C ABI of a GB300-native (sm_103a) exact Euclidean DBSCAN.
 *
 * The library implements the grid method of Wang, Gu and Shun, "Theoretically-
 * Efficient and Practical Parallel DBSCAN" (SIGMOD 2020): points go into cells
 * of side eps/sqrt(d) (Sec. 3, Algorithm 1; Sec. 4.1), core points are marked
 * by range counts over neighbouring cells (Sec. 4.3, Algorithm 2), core cells
 * are joined by bichromatic-closest-pair tests with early exit and a lock-free
 * union-find (Sec. 4.4, Algorithm 3), and border points collect the clusters of
 * the core points within eps (Sec. 4.5, Algorithm 4).  The result is the one
 * fixed by the DBSCAN definition of Sec. 2, with these conventions:
 *
 *   - within(p, q) is  sum_i (p_i - q_i)^2 <= fl(eps*eps)  evaluated in IEEE
 *     FP64, left to right, without fused multiply-add.  FP32 inputs are widened
 *     exactly.  In the FP32 precision mode the library first decides each pair
 *     in FP32 and recomputes in FP64 any pair whose FP32 value lies inside a
 *     forward-error band around eps^2, so the decisions are those of the FP64
 *     predicate in both modes.
 *   - a point is core iff at least min_pts points (itself included) are
 *     within eps of it;
 *   - a cluster is named by the smallest input index of its core points;
 *   - labels[p] is the cluster of a core point, the smallest cluster of a
 *     border point, and -1 for noise;
 *   - the full cluster set of each non-core point is returned as CSR, sorted
 *     ascending (core points have an empty entry there; their one cluster is
 *     labels[p]).
 *
 * Conventions for every call:
 *   - pointers named d_* are device pointers, h_* are host pointers;
 *   - the caller owns all input and output buffers; the context owns its
 *     device workspace, which it allocates in dbscan_create();
 *   - all device work is ordered on the caller's CUDA stream (a cudaStream_t
 *     passed as void*; NULL = legacy default stream);
 *   - errors are returned as dbscan_status codes; no C++ exception crosses
 *     the ABI; a context stays usable after any error it returns;
 *   - a context is not thread-safe: one call at a time per context.
 */
#ifndef DBSCAN_GB300_H
#define DBSCAN_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DBSCAN_OK = 0,
    DBSCAN_ERR_INVALID_ARG = 1,     /* bad size, pointer, eps, min_pts or non-finite coordinate */
    DBSCAN_ERR_UNSUPPORTED_DIM = 2, /* d outside the supported range */
    DBSCAN_ERR_OOM = 3,             /* device or pinned allocation failed */
    DBSCAN_ERR_KEY_OVERFLOW = 4,    /* the grid needs more cells per dimension than the key holds */
    DBSCAN_ERR_CAPACITY = 5,        /* a data-dependent buffer of the context is too small */
    DBSCAN_ERR_CUDA = 6,            /* a CUDA runtime call failed */
    DBSCAN_ERR_DEVICE_TIMEOUT = 7,  /* a bounded device retry loop gave up */
    DBSCAN_ERR_STATE = 8            /* call out of order (e.g. border ids before a run) */
} dbscan_status;

/* Element type of the input coordinates. */
enum { DBSCAN_F32 = 0, DBSCAN_F64 = 1 };

/* Options for dbscan_set_option(). */
enum {
    /* value: DBSCAN_PREC_FP32_RECHECK (default) or DBSCAN_PREC_FP64 */
    DBSCAN_OPT_PRECISION = 0,
    /* value: DBSCAN_SCHED_SIZE (default), DBSCAN_SCHED_NONE */
    DBSCAN_OPT_SCHEDULE = 1,
    /* value: 0 (default) or 1: count distance evaluations in dbscan_stats */
    DBSCAN_OPT_COLLECT_STATS = 2,
    /* value: iteration limit of every bounded device retry loop (default 1<<22) */
    DBSCAN_OPT_MAX_ITERS = 3,
    /* value: 0 (default) or 1: record CUDA events around each phase and report
       the phase durations in dbscan_stats.phase_ms */
    DBSCAN_OPT_PHASE_TIMING = 4,
    /* value: 1 (default) or 0: in the FP32-band mode, decide whole cells by
       the bounding boxes of their points where the boxes settle the question
       (all pairs within eps, or none), as the quadtree range counts of
       Sec. 5.2 do; 0 tests every pair point by point */
    DBSCAN_OPT_CELL_BOUNDS = 5,
    /* value: 1 (default) or 0: dbscan_run_batch captures its sequence as a CUDA
       graph and replays it; 0 enqueues the kernels directly every call */
    DBSCAN_OPT_BATCH_GRAPH = 6,
    /* value: capacity (records) of the pair log, 0 (default) = off.  While on,
       runs use the learned schedule's pair list in logging mode: every pair
       the core-point boxes do not settle gets an exact BCP test (no union-find
       skipping) and its features and outcome are recorded, for
       dbscan_train_scheduler() */
    DBSCAN_OPT_PAIR_LOG = 7,
    /* value: 1, 2, 4 (default) or 8: core cells a warp of the connectivity
       kernel takes from the work counter at once (their pair lists are
       flattened across the warp's lanes) */
    DBSCAN_OPT_CONNECT_CELLS = 8,
    /* value: 2 (default) or 1: with SIZE or NONE, test the adjacent-cell pairs
       first, compress the union-find, then the farther pairs (2); or all pairs
       in one wave (1) */
    DBSCAN_OPT_CONNECT_WAVES = 9,
    /* value: 0 (default: as many as fit) or 1..32: resident blocks per SM of
       the persistent (grid-stride, work-counter) kernels */
    DBSCAN_OPT_BLOCKS_PER_SM = 10,
    /* value: 0 (default: off) or a limit L: MarkCore counts for the points of
       sparse cells with fewer than 8 points and at most L points in their
       neighbouring cells with one thread per point instead of one warp per
       cell, and ClusterBorder assigns their non-core points the same way
       (faster on sparse inputs); L >= 2^30 takes every such cell */
    DBSCAN_OPT_SMALL_CELLS = 11,
    /* value: 1 (default) or 0: in the FP32-band mode with cell bounds, the
       bounding boxes of two cells' core points settle whole pairs in
       ClusterCore and whole cells in ClusterBorder; 0 leaves those to the
       point tests (saves the core boxes where they rarely decide) */
    DBSCAN_OPT_PAIR_BOXES = 12,
    /* value: 0 (default) or 1: record a link witness for every union of two
       clusters during the run (for dbscan_link_witnesses; a checking aid, the
       result does not change) */
    DBSCAN_OPT_WITNESS = 13,
    /* value: 0 (default) or L = 1..3: for 5 <= d <= 8 in the FP32-band mode
       with cell bounds, MarkCore counts the points of a neighbouring cell of
       at least 32 points by descending a quadtree of L levels below the cell
       (the range counting of Sec. 5.2): nodes whose points are all within eps
       count whole, nodes with none are skipped, only the leaves in between
       are scanned.  Ignored below 5 dimensions and in the FP64 mode. */
    DBSCAN_OPT_QUADTREE = 14,
    /* value: 1 (default) or 0: dbscan_run_slabs copies host input into device
       memory once when it fits (free memory above its size plus 4 GiB) and
       reads every pass from there; 0 reads pinned host input in place and
       stages pageable input chunk by chunk in every pass */
    DBSCAN_OPT_SLAB_STAGE = 15,
    /* value: 0 (default) or 1: open an NVTX range per phase of every run (the
       phases of dbscan_stats.phase_ms, named "dbscan:<phase>") and per step of
       dbscan_run_slabs, for profilers that filter or group by NVTX ranges; host
       calls only, no effect on the result */
    DBSCAN_OPT_NVTX = 16
};
enum { DBSCAN_PREC_FP64 = 0, DBSCAN_PREC_FP32_RECHECK = 1 };
/* SIZE: core-cell pairs are tested in order of non-increasing core count of the
 * owning cell (Sec. 4.4, "Reducing Cell Connectivity Queries"), adjacent cells
 * first, then (after path compression) the farther ones.
 * NONE: pairs are tested in cell order (ablation).
 * LEARNED: the pairs the core-point boxes do not settle are scored by the
 * context's network and tested likeliest-connected first (extends the size
 * heuristic of Sec. 4.4; exact BCP decides every pair as before). */
enum { DBSCAN_SCHED_SIZE = 0, DBSCAN_SCHED_NONE = 1, DBSCAN_SCHED_LEARNED = 2 };

typedef struct dbscan_ctx dbscan_ctx;

/* Counters of the last run (filled by dbscan_get_stats). */
typedef struct {
    int64_t n;                      /* points */
    int32_t d;                      /* dimension */
    int32_t precision;              /* mode actually used (FP32 mode falls back to FP64
                                       when eps^2 lies outside [2^-60, 2^60]) */
    int32_t key_bits;               /* bits of the packed cell key */
    int32_t radix_passes;           /* 8-bit passes of the key sort */
    int64_t num_cells;              /* non-empty cells */
    int64_t num_core_cells;         /* cells with at least one core point */
    int64_t num_neighbor_entries;   /* cached neighbour-cell list length */
    int64_t num_candidate_pairs;    /* core-cell pairs, each unordered pair once */
    int64_t num_pairs_tested;       /* BCP tests run */
    int64_t num_pairs_skipped;      /* pairs skipped because union-find had joined them */
    int64_t num_pairs_connected;    /* pairs found connected (by BCP or by their boxes) */
    int64_t num_pairs_box_decided;  /* pairs settled by the core-point bounding boxes alone */
    int64_t num_pairs_listed;       /* learned schedule: pairs left for BCP after the boxes */
    int64_t num_core_points;
    int64_t num_border_points;
    int64_t num_noise_points;
    int64_t num_border_memberships; /* total length of the border sets */
    int64_t band_rechecks;          /* FP32 decisions recomputed in FP64 */
    int64_t distance_evals;         /* pair distances evaluated (only with COLLECT_STATS) */
    int64_t distance_evals_phase[3];/* of which in MarkCore, BCP tests, border assignment */
    float band_lo, band_hi;         /* FP32 band around eps^2 (FP32 mode) */
    int64_t kernel_launches;        /* CUDA kernels the run launched */
    /* Phase durations in ms (only with PHASE_TIMING), from CUDA events on the
       run's stream: 0 bounding box, 1 host read of the box, 2 cell keys, sort
       and grouping, 3 cell boxes and the lookup structure of the neighbour
       search (supercell hash, or the tree for d >= 5), 4 the neighbour-list
       kernel, 5 MarkCore, 6 core compaction and pair schedule, 7 BCP
       connectivity with union-find, 8 labels and border counts. */
    float phase_ms[9];
    /* Algorithmic work of MarkCore (only with COLLECT_STATS): the sum over the
       cells with fewer than minPts points of |g| times the points of all their
       neighbouring cells, the distance tests a scan without early exit makes. */
    int64_t markcore_pair_bound;
    /* Pair schedule the run used: the context's, or DBSCAN_SCHED_SIZE when the
       learned schedule's pair list would exceed 2^31 pairs (its fallback). */
    int32_t schedule_used;
    int32_t reserved;
    /* rho of the run's connectivity rule: 0 = exact DBSCAN (dbscan_set_approx) */
    double rho;
} dbscan_stats;

/*
 * Create a context able to cluster up to max_points points of dimension up to
 * max_dim.  Allocates the device workspace on the current device (its size
 * grows linearly with max_points and with the number of candidate
 * neighbouring cells of min(max_dim, 4)).  1 <= max_dim <= 8;
 * 0 <= max_points < 2^31-1.  Runs of d >= 5 find neighbouring cells with a
 * tree over the non-empty cells (Sec. 5.1) instead of offset enumeration;
 * their tree and neighbour-list buffers are allocated at the first such run
 * (OOM there if the device is full).
 * Returns OK, INVALID_ARG, UNSUPPORTED_DIM, OOM or CUDA.  *ctx is NULL on error.
 */
dbscan_status dbscan_create(dbscan_ctx **ctx, int64_t max_points, int max_dim);

/* Free the context and its workspace (synchronises the device). NULL is a no-op. */
void dbscan_destroy(dbscan_ctx *ctx);

/* Set one DBSCAN_OPT_* option; INVALID_ARG for unknown options or values. */
dbscan_status dbscan_set_option(dbscan_ctx *ctx, int option, int64_t value);

/*
 * Exact DBSCAN (Algorithm 1) of d_points [n, d], row-major, element type dtype
 * (DBSCAN_F32 or DBSCAN_F64), on the given stream.
 *   eps      > 0 and finite;  min_pts >= 1;  0 <= n <= max_points;
 *   1 <= d <= max_dim; every coordinate finite.
 * Outputs (device, caller-allocated, indexed like the input):
 *   d_core   [n] uint8:  1 iff core (Algorithm 2);
 *   d_labels [n] int32:  cluster name as described above;
 *   d_border_offsets [n+1] int64 or NULL: CSR offsets of the border sets.
 * *num_border_memberships (host, may be NULL) receives the total set length,
 * which is the capacity dbscan_border_ids() needs.
 * The call synchronises the stream twice: once after the bounding-box
 * reduction (its result sizes the cell key) and once at the end to read the
 * device status; for d >= 5 once more after the neighbour counts (their total
 * sizes the neighbour lists).  Returns OK, INVALID_ARG, UNSUPPORTED_DIM,
 * KEY_OVERFLOW (d <= 4: more than 2^30 cells in a dimension or more than 63
 * key bits; d >= 5: more than 2^15 cells in a dimension), CAPACITY,
 * DEVICE_TIMEOUT or CUDA; outputs are undefined unless OK.
 */
dbscan_status dbscan_run(dbscan_ctx *ctx, const void *d_points, int64_t n, int d, int dtype,
                         double eps, int64_t min_pts, uint8_t *d_core, int32_t *d_labels,
                         int64_t *d_border_offsets, int64_t *num_border_memberships,
                         void *stream);

/*
 * Fill d_ids with the border sets of the last successful dbscan_run() on this
 * context (Algorithm 4), in the CSR layout of its d_border_offsets: the entry of
 * point p is d_ids[off[p] .. off[p+1]), ascending cluster names.  capacity is
 * the length of d_ids and must be >= the run's num_border_memberships.
 * The input points of that run must still be unchanged in device memory.
 * Returns OK, STATE (no run), CAPACITY, INVALID_ARG or CUDA.  Synchronises.
 */
dbscan_status dbscan_border_ids(dbscan_ctx *ctx, int32_t *d_ids, int64_t capacity, void *stream);

/*
 * Link witnesses of the last successful run (dbscan_run or dbscan_run_batch)
 * made with DBSCAN_OPT_WITNESS = 1: a certificate that each cluster is
 * connected through steps of at most eps between core points (Sec. 2), which
 * a checker can verify pair by pair without rerunning the method.
 *   d_rep [n] int32 (the run's n rows): for a core point, the input index of
 *     the first core point of its cell (cells have side eps/sqrt(d), so any two
 *     of their points are within eps, Sec. 3); -1 for other points;
 *   d_links [2 * capacity] int32: pair i = (d_links[2i], d_links[2i+1]), input
 *     indices of two core points within eps that joined two clusters of the
 *     union-find (Algorithm 3): one pair per successful union;
 *   *count (host) receives the number of pairs; capacity must be at least that
 *     (CAPACITY otherwise; the number is at most the number of cells, and
 *     exactly the number of core cells minus the number of clusters).
 * For a batch the indices are rows of the whole batch.  The run's workspace
 * must be untouched since (no other run on the context).  Returns OK, STATE
 * (no run, or the run had the option off), CAPACITY, INVALID_ARG or CUDA.
 * Synchronises the stream.
 */
dbscan_status dbscan_link_witnesses(dbscan_ctx *ctx, int32_t *d_rep, int32_t *d_links, int64_t capacity,
                                    int64_t *count, void *stream);

/* One problem of a batch: rows [row0, row0 + n) of the batch's point array,
 * using the first d of its ld columns. */
typedef struct {
    int64_t row0;     /* first row; instance i+1 starts where instance i ends (row0 of 0 is 0) */
    int64_t n;        /* rows of this instance (0 allowed) */
    int32_t d;        /* dimension of this instance, 1 <= d <= ld */
    int32_t reserved; /* set to 0 */
    double eps;       /* > 0, finite */
    int64_t min_pts;  /* >= 1 */
} dbscan_instance;

/*
 * Exact DBSCAN of count independent instances at once (the batched use of
 * Algorithm 1): d_points [N, ld] row-major (N = sum of the instances' n, at
 * most the context's max_points; ld <= max_dim, ld <= 3), element type dtype.
 * Each instance is clustered on its own, with its own eps and min_pts; the
 * outputs are indexed by row like the input:
 *   d_core [N], d_labels [N]: as in dbscan_run(), with cluster names local to
 *     the instance (the smallest core index counted from the instance's row0);
 *   d_border_offsets [N+1] or NULL: border-set CSR over all rows (the names in
 *     it are instance-local too); dbscan_border_ids() fills it afterwards.
 * All instances go through the same kernels in one pass: each gets its own
 * grid and thresholds built on the device from its own bounding box.  The
 * whole sequence is captured as one CUDA graph on the first call and replayed
 * by later calls with the same count, sizes, pointers, dtype and options (the
 * coordinates, eps and min_pts may change between calls).  Precision: the FP32
 * band with FP64 recheck for FP32 input when every eps^2 lies in
 * [2^-60, 2^60], otherwise FP64.  Synchronises the stream once at the end.
 * Returns OK, INVALID_ARG, UNSUPPORTED_DIM, KEY_OVERFLOW (an instance's grid
 * exceeds its share of the 63-bit cell key), CAPACITY, DEVICE_TIMEOUT, OOM or
 * CUDA.
 */
dbscan_status dbscan_run_batch(dbscan_ctx *ctx, const dbscan_instance *h_instances, int count,
                               const void *d_points, int ld, int dtype, uint8_t *d_core, int32_t *d_labels,
                               int64_t *d_border_offsets, int64_t *num_border_memberships, void *stream);

/*
 * Same as dbscan_run() but with host buffers: copies h_points to the device,
 * runs, and copies core flags, labels and (when h_border_offsets is not NULL)
 * the border-set offsets [n+1] back; with h_border_ids also the border ids,
 * which need ids_capacity >= the run's set length (*num_border_memberships
 * receives it; CAPACITY if the buffer is too small, and the caller may retry
 * with a larger one).  Pinned host memory gives asynchronous copies; pageable
 * memory works but is staged by the driver.  The device copies live in the
 * context (allocated at the first call, the ids buffer grown as needed).
 * Synchronises the stream.
 */
dbscan_status dbscan_run_host(dbscan_ctx *ctx, const void *h_points, int64_t n, int d, int dtype,
                              double eps, int64_t min_pts, uint8_t *h_core, int32_t *h_labels,
                              int64_t *h_border_offsets, int32_t *h_border_ids, int64_t ids_capacity,
                              int64_t *num_border_memberships, void *stream);

/* dbscan_run_batch() with host buffers, like dbscan_run_host(): h_points [N,
 * ld], outputs indexed by row (N = the instances' total). */
dbscan_status dbscan_run_batch_host(dbscan_ctx *ctx, const dbscan_instance *h_instances, int count,
                                    const void *h_points, int ld, int dtype, uint8_t *h_core, int32_t *h_labels,
                                    int64_t *h_border_offsets, int32_t *h_border_ids, int64_t ids_capacity,
                                    int64_t *num_border_memberships, void *stream);

/* What a dbscan_run_slabs() call did. */
typedef struct {
    int32_t slabs;            /* slabs run (cuts that coincide are merged) */
    int32_t axis;             /* partition dimension: the widest of the bounding box */
    int64_t max_slab_points;  /* largest slab with its halo */
    int64_t halo_points;      /* points run as halo, summed over slabs */
    int64_t border_pairs;     /* (border point, cluster) pairs merged before deduplication */
    int64_t kernel_launches;  /* kernels this call launched, the slab runs' included */
    double ms[5];             /* host-timed: extremes and histogram passes, slab selection,
                                 slab runs (with their border sets), merges, names and copies out */
} dbscan_slab_stats;

/*
 * Exact DBSCAN of one instance larger than the context's workspace, as the
 * paper's billion-point runs (Sec. 7) need: the points are split into slabs
 * along the widest dimension of their bounding box, each slab is run through
 * dbscan_run() with every point within a halo of 2 eps (plus rounding margin)
 * on either side, and the runs are merged on the device into the result of
 * dbscan_run() on the whole input (same core flags, names and border sets):
 * owned points' core flags are exact in their slab, a point a slab calls core
 * is core, and each edge between core points lies inside the run of the slab
 * that owns one of its ends (Sec. 2, Algorithm 1).
 *   points   [n, d] row-major, DBSCAN_F32 or DBSCAN_F64; device memory, or
 *            host memory, copied to the device once if it fits there (see
 *            DBSCAN_OPT_SLAB_STAGE), else read in place when pinned or staged
 *            in 256 MiB chunks when pageable;  0 <= n < 2^31 - 1 (no bound
 *            from max_points);  d <= max_dim;  eps, min_pts as in dbscan_run();
 *   num_slabs  1..4096 slabs cut at equal point counts, or 0: the fewest
 *            whose slab-with-halo counts (bounded from an 8192-bin histogram
 *            of the axis coordinate) fit max_points;
 *   core [n] uint8, labels [n] int32, border_offsets [n+1] int64 (or NULL):
 *            the outputs of dbscan_run(), in host or device memory;
 *            *num_border_memberships receives the border sets' total length,
 *            the capacity dbscan_slab_border_ids() needs;
 *   stats    may be NULL.
 * Device memory beyond the context's workspace, kept for later calls: 17n
 * bytes of global state, one slab-sized input copy with its outputs
 * (max_points x (row + 17) bytes), 16 bytes per border pair, and the staged
 * input (n x row bytes) when host input is staged.  The input is read once
 * per slab plus two passes (extremes, histogram).  Returns
 * INVALID_ARG (also for a non-finite coordinate), CAPACITY (a slab with its
 * halo exceeds max_points: too many points share one histogram bin, or the
 * halo is wider than the slabs), OOM, DEVICE_TIMEOUT, CUDA, or what a slab's
 * dbscan_run() returns.  Synchronises the stream.  Afterwards the context
 * holds no run for dbscan_border_ids() or dbscan_link_witnesses().
 */
dbscan_status dbscan_run_slabs(dbscan_ctx *ctx, const void *points, int64_t n, int d, int dtype, double eps,
                               int64_t min_pts, int32_t num_slabs, uint8_t *core, int32_t *labels,
                               int64_t *border_offsets, int64_t *num_border_memberships, dbscan_slab_stats *stats,
                               void *stream);

/*
 * The border sets of the last successful dbscan_run_slabs() on this context
 * (Algorithm 4), in the CSR layout of its border_offsets: ascending cluster
 * names.  border_ids (host or device) holds capacity entries, at least the
 * call's num_border_memberships (CAPACITY otherwise; NULL is allowed when that
 * is 0).  Returns OK, STATE (no such call, or a later one failed), CAPACITY,
 * INVALID_ARG or CUDA.  Synchronises the stream.
 */
dbscan_status dbscan_slab_border_ids(dbscan_ctx *ctx, int32_t *border_ids, int64_t capacity, void *stream);

/*
 * Exact DBSCAN like dbscan_run(), without any allocation, for callers that
 * cannot allocate device memory (code running inside another framework's
 * memory pool, plugins whose host forbids device allocation after start-up,
 * callers that must avoid the implicit synchronisation of cudaMalloc/cudaFree).
 * The paper has no counterpart: this is a packaging of the same run.
 *
 * Working memory is one fixed __device__ array of the library (20 MiB), held by
 * every GPU that loads the library until the process exits.  Limits:
 * n <= 16384 points and d <= 3; larger n returns DBSCAN_ERR_CAPACITY, larger d
 * DBSCAN_ERR_UNSUPPORTED_DIM.  The caller passes the input d_points [n, d]
 * (DBSCAN_F32 or DBSCAN_F64) and the outputs d_core [n] and d_labels [n], with
 * the meaning they have in dbscan_run(); border sets are not returned.
 * Precision is the FP32 band with FP64 recheck, schedule SIZE.
 *
 * No cudaMalloc, cudaFree, pinned allocation or allocating library routine is
 * called.  Every call resolves the array's device address
 * (cudaGetSymbolAddress); the first call on a device, and any call after the
 * address has changed (a device reset), sets the array up: it copies the
 * neighbour-offset tables into it, clears the cell hash and synchronises the
 * device, so make that first call before any stream capture.  The array is
 * shared by every call on a device and keeps the last call's contents (each
 * call clears what must start at zero): calls that overlap on the GPU, from
 * any thread or stream, race and corrupt each other.  Synchronises the stream
 * like dbscan_run().
 */
dbscan_status dbscan_run_static(const void *d_points, int64_t n, int d, int dtype, double eps,
                                int64_t min_pts, uint8_t *d_core, int32_t *d_labels, void *stream);

/*
 * Learned pair scheduler (an extension of the priority order of Sec. 4.4; the
 * paper trains nothing).  The context holds a network of 6 inputs, two hidden
 * layers of 32 ReLU units and one logit output (1313 FP32 parameters,
 * initialised deterministically at dbscan_create).  Its inputs per pair of
 * core cells: log2(1 + larger core count), log2(1 + smaller core count), the
 * distance between the core centroids, the minimum and maximum distance
 * between the core-point boxes (all three divided by eps), and smaller over
 * larger core count.
 *
 * dbscan_train_scheduler: re-initialise the network from seed and fit it with
 * Adam (learning rate lr, mini-batches of `batch` records, `epochs` passes) to
 * the binary cross-entropy of the records logged by the last run made with
 * DBSCAN_OPT_PAIR_LOG; h_losses (host, `epochs` floats, may be NULL) receives
 * the mean loss of each epoch.  Returns STATE if nothing is logged.
 * Synchronises the device.
 */
dbscan_status dbscan_train_scheduler(dbscan_ctx *ctx, int epochs, int batch, float lr, uint64_t seed,
                                     float *h_losses);

/* Copy the network's 1313 parameters to (set = 0) or from (set = 1) h_weights.
 * Layout: W1[32][6], b1[32], W2[32][32], b2[32], w3[32], b3. */
dbscan_status dbscan_scheduler_weights(dbscan_ctx *ctx, float *h_weights, int count, int set);

/* Mean binary cross-entropy (with logits) of the network on n records
 * d_features [n][6], d_labels [n] (0/1) and its gradient, h_grad [1313]
 * (same layout as the parameters).  Synchronises the device. */
dbscan_status dbscan_scheduler_loss_grad(dbscan_ctx *ctx, const float *d_features, const uint8_t *d_labels,
                                         int64_t n, float *h_loss, float *h_grad);

/* Copy the pair log of the last logging run to d_features [capacity][6] and
 * d_labels [capacity]; *count receives the number of records.  CAPACITY if
 * capacity is too small.  Synchronises the device. */
dbscan_status dbscan_get_pair_log(dbscan_ctx *ctx, float *d_features, uint8_t *d_labels, int64_t capacity,
                                  int64_t *count);

/* Read back one DBSCAN_OPT_* option (INVALID_ARG for unknown options). */
dbscan_status dbscan_get_option(const dbscan_ctx *ctx, int option, int64_t *value);

/* The configuration an autotuner run chose, and what it measured. */
typedef struct {
    int32_t schedule;       /* DBSCAN_OPT_SCHEDULE */
    int32_t cell_bounds;    /* DBSCAN_OPT_CELL_BOUNDS */
    int32_t connect_waves;  /* DBSCAN_OPT_CONNECT_WAVES */
    int32_t connect_cells;  /* DBSCAN_OPT_CONNECT_CELLS */
    int32_t blocks_per_sm;  /* DBSCAN_OPT_BLOCKS_PER_SM */
    int32_t small_cells;    /* DBSCAN_OPT_SMALL_CELLS */
    int32_t pair_boxes;     /* DBSCAN_OPT_PAIR_BOXES */
    int32_t quadtree;       /* DBSCAN_OPT_QUADTREE */
    int32_t trials;         /* configurations timed */
    float best_ms;          /* wall time of one call with the chosen configuration (best of reps) */
    float default_ms;       /* the same for the configuration the context had before */
} dbscan_tuning;

/*
 * Autotuner (the tile and schedule choice of the batched persistent kernels):
 * time dbscan_run on this input for candidate settings of the pair schedule,
 * the cell-box decisions (FP32 mode only), one or two connectivity waves, the
 * core cells per work item of the connectivity kernel, the resident blocks
 * per SM of the persistent kernels and MarkCore's thread-per-point limit, by coordinate descent from the context's
 * current setting (one warm-up and `reps` timed calls per candidate, the
 * fastest kept), and leave the fastest setting in the context.  None of the
 * settings changes the result.  Arguments as for dbscan_run; the outputs go
 * to scratch buffers the call allocates and frees.  out (host, may be NULL)
 * receives the choice.  Returns the first failing run's status, OOM, or OK.
 */
dbscan_status dbscan_autotune(dbscan_ctx *ctx, const void *d_points, int64_t n, int d, int dtype, double eps,
                              int64_t min_pts, int reps, dbscan_tuning *out, void *stream);

/* The same for dbscan_run_batch (arguments as there; the graph is recaptured
 * for every candidate). */
dbscan_status dbscan_autotune_batch(dbscan_ctx *ctx, const dbscan_instance *host_desc, int count,
                                    const void *d_points, int ld, int dtype, int reps, dbscan_tuning *out,
                                    void *stream);

/*
 * rho-approximate DBSCAN (the relaxed problem of Gan and Tao, Sec. 2): rho > 0
 * lets core points farther apart than eps but within eps(1 + rho) connect, so
 * several clusterings are valid; rho = 0 (the default) is exact DBSCAN.  The
 * following runs and batches of the context keep the core rule and the
 * border rule at eps and decide the connectivity of neighbouring core cells
 * (Algorithm 3) with the threshold r = fl(eps * fl(1 + rho)): a pair of core
 * points joins two cells iff sum_i (p_i - q_i)^2 <= fl(r * r) in FP64 (the
 * FP32 band with recheck applies to r as it does to eps), and the core-point
 * boxes settle a pair when all of their pairs are within r, or none is.
 * Every pair of core points within eps lies in one cell or in neighbouring
 * cells, so it is always joined, and no join is longer than r: the result is
 * a valid rho-approximate clustering (Sec. 5.2 answers the same problem with
 * approximate range counts on a quadtree).  Cluster names and border sets
 * follow the exact conventions.  0 <= rho <= 1e6, else INVALID_ARG.
 */
dbscan_status dbscan_set_approx(dbscan_ctx *ctx, double rho);

/* Counters of the last run (host copy; no device work). */
dbscan_status dbscan_get_stats(const dbscan_ctx *ctx, dbscan_stats *out);

/* Static English text for a status code. */
const char *dbscan_status_string(int status);

/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int dbscan_version(void);

#ifdef __cplusplus
}
#endif
#endif /* DBSCAN_GB300_H */
