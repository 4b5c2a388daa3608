// Host-side launchers of the phase kernels (one stream, no host sync inside).
#pragma once

#include "internal.cuh"

namespace gbdb {

// ---- cells (grid.cu)
// out: [2*kMaxDim + 1] int64: order-preserving keys of the per-dimension
// minima and maxima (see bbox_key_to_double) and a non-finite flag.
void launch_bbox(const void *X, int dtype, int n, int d, int nb, long long *out, cudaStream_t s);
inline double bbox_key_to_double(long long k) {
    const long long b = k >= 0 ? k : (k ^ 0x7fffffffffffffffll);
    double x;
    __builtin_memcpy(&x, &b, sizeof x);
    return x;
}
// Buffers of the cell grouping (semisort) of one run.
struct Semisort {
    const void *unused;
    ulonglong2 *ht;       // cell hash, hcap slots {key, point count, then cell id}; empty between runs
    uint64_t hcap;        // power of two >= 2 * max points
    uint32_t *slot_of, *rank_of;  // [n] slot of each point, its position in the cell
    uint32_t *slots;      // [m] slots of the non-empty cells, in insertion order
    uint64_t *k0, *k1;    // sort of the m cell keys
    uint32_t *v0, *v1;
    void *sort_scratch;
    size_t sort_scratch_size;
    long long *part;
    uint64_t *cell_key;   // [m] keys in Z order
    int *count;           // [m+1] points per cell (scratch for the scan)
    int *cell_start;      // [m+1]
    float *pf;
    double *pd;           // null unless FP64 input
    int *orig, *cell_of;
    int *cell_inst;       // [m] instance of each cell (several instances only)
    int key_lo, key_bits; // key bits the cell sort orders by
    unsigned *bloom;      // 2^bloom_lg bits: Bloom filter of the run's cell keys (cleared per run), or null
    int bloom_lg;
    bool super;           // d = 2, 3: a dense grid keeps the offset enumeration, a sparse one
                          // takes supercells (decided on the device from n and m)
    int n;                // points of the run
    unsigned *bloom_all;  // the Bloom filter's storage (supercell keys)
};
// Group the points by cell: fills cell_key, cell_start, pf/pd, orig, cell_of,
// ctr->m, and the slots' cell ids.
void launch_semisort(const void *X, int dtype, const RunParams &P, int SD, const Semisort &S, DevCounters *ctr,
                     cudaStream_t s);
// Empty every slot of the cell hash (first use, or after a failed run).
void launch_table_clear(ulonglong2 *ht, uint64_t cap, cudaStream_t s);
// Empty the slots the run used (keeps the table clean for the next run): the
// cells' slots, or at the end of a supercell run the supercells' slots.
void launch_table_reset(const Semisort &S, DevCounters *ctr, cudaStream_t s, bool end_of_run = true);
// The supercell table of d = 2, 3 (empties the cells' slots of the hash
// first), then the neighbour lists through it (fixed stride per cell, as
// launch_neighbors).
void launch_super_table(const Semisort &S, const RunParams &P, DevCounters *ctr, cudaStream_t s);
void launch_neighbors_super(const Semisort &S, const RunParams &P, int stride, const float4 *blo,
                            const float4 *bhi, const int *cell_start, int *nbr_cnt, int *nbr_near, int *nbr_pts,
                            int *nbr, DevCounters *ctr, cudaStream_t s);
void launch_neighbors(const uint64_t *cell_key, const ulonglong2 *ht, uint64_t hcap, const unsigned *bloom,
                      int bloom_lg, const RunParams &P, const signed char *offs, int noff, int n_near,
                      const float4 *blo, const float4 *bhi, const int *cell_start, int *nbr_cnt, int *nbr_near,
                      int *nbr_pts, int *nbr, DevCounters *ctr, cudaStream_t s, bool only_dense = false);
// log2 of the Bloom filter's bit count for max_points points (4 to 8 bits per point)
inline int bloom_log2(long long max_points) {
    int lg = 10;
    while ((1ll << lg) < 4 * max_points) ++lg;
    return lg;
}
// per-cell FP32 bounding boxes of pts[start[c] .. start[c+1]) (and the
// centroids when cent is not null)
void launch_boxes(int SD, const float *pts, const int *start, const DevCounters *ctr, float4 *lo, float4 *hi,
                  cudaStream_t s, float4 *cent = nullptr);

// The quadtree below the cells (d >= 5), read by MarkCore: per level l =
// 1..levels, qpos[l-1][t] nodes start before point t, qstart[l-1][k] is the
// first point of node k, qlo/qhi[l-1] its FP32 box (two float4 per node).
struct QtView {
    int levels;
    const int *qpos[3];
    const int *qstart[3];
    const float4 *qlo[3], *qhi[3];
};

// Device arrays of one run, shared by the cluster phases.
struct Bufs {
    // sorted points and cell table
    const float *pf;
    const double *pd;  // null unless FP64 input
    const int *orig, *cell_of, *cell_start;
    const int *nbr_cnt;  // [m] neighbours of cell c: nbr[c*nbr_stride .. + nbr_cnt[c])
    const int *nbr_near; // [m] how many of them are at |delta|_inf <= 1 (listed first)
    const int *nbr;
    int nbr_stride;
    const long long *nbr_off;  // [m] CSR offsets of the lists (d >= 5); null: fixed stride
    const int *nbr_pts;        // [m] points in all neighbouring cells of c
    // MarkCore / compaction
    int *core_s;        // [n] 0/1 in cell order
    int *core_pos;      // [n+1] exclusive scan of core_s
    int *ccs;           // [m+1] core points of cell c: [ccs[c], ccs[c+1]) of the compacted arrays
    float *cpf;         // compacted core points
    double *cpd;
    int *core_orig;     // input index of compacted core point
    int *core_cell;     // cell of compacted core point
    const float4 *blo, *bhi;  // per-cell bounding box of all points
    float4 *cblo, *cbhi;      // per-cell bounding box of the core points
    float4 *ccent;            // per-cell centroid of the core points (learned schedule)
    // schedule
    uint64_t *sk0, *sk1;
    uint32_t *sv0, *sv1;
    void *sort_scratch;
    size_t sort_scratch_size;
    int max_iters;
    int *rank;          // [m] position of the cell in test order
    // union-find and labels
    int *parent, *compmin, *cell_label;
    // border
    int *noncore;       // [n_noncore] cell-order indices of the non-core points
    long long *bcount, *boff;
    unsigned char *bbig;  // [N] by input index: the point's border set outgrew k_border_small's
    int2 *bcache;         // [N] by input index: a border set of at most 2 names from the count pass
    int *bheavy;          // [N] non-core list positions whose sets have more than 2 names
    long long *part;
    int64_t n_max;
    QtView qt;
};

// ---- clusters (cluster.cu)
void launch_markcore(int D, int mode, const RunParams &P, const Bufs &B, DevCounters *ctr, cudaStream_t s);
void launch_core_compact(int SD, const RunParams &P, const Bufs &B, DevCounters *ctr, cudaStream_t s);
// returns the test order of the cells (null: cell order)
const uint32_t *launch_schedule(int sched, const RunParams &P, const Bufs &B, DevCounters *ctr, cudaStream_t s);
void launch_connect(int D, int mode, const uint32_t *order, const RunParams &P, const Bufs &B, DevCounters *ctr,
                    cudaStream_t s);
// ---- cells and neighbour lists for 5 <= d <= 8 (hd.cu)
struct HdBufs {
    uint64_t *klo, *khi;          // [n] 128-bit Morton key of each point's cell (low, high word)
    uint64_t *ckey_lo, *ckey_hi;  // [m] cell keys, Z order
    int4 *ccoord;                 // [m] cell coordinates, 8 x 16 bits
    int2 *child;                  // [m-1] children of the internal tree nodes (leaf of cell c: m-1+c)
    int *parent;                  // [2m-1] parent of each node (-1 at the root)
    int *flag;                    // [m-1] arrival counters of the bottom-up pass
    int4 *nlo, *nhi;              // [m-1] node bounds in cell coordinates, 8 x 16 bits
    float4 *nblo, *nbhi;          // [m-1] x 2: node bounding boxes of the points (FP32-band mode)
    long long *nbr_off;           // [m+1] offset of each cell's neighbour list
    int *scratch;                 // per-warp leaf scratch of the neighbour kernel
    int *nmax;                    // [m-1] last cell (leaf) under each internal node
    long long *fwd_off;           // [m] offset of each cell's forward list (cells after it only)
    int *fn, *ff;                 // [m] forward adjacent / farther counts
    int *bn, *bf;                 // [m] backward adjacent / farther counts (zero before the transpose)
    // quadtree below the cells (MarkCore's range counts), allocated when used
    unsigned *qsub_in, *qsub;     // [n] sub-cell key of each point, by input index / in cell order
    int *qpos[3];                 // per level: [n+1] nodes starting before each point
    int *qstart[3];               // per level: [n+1] first point of each node (then n)
    float4 *qlo[3], *qhi[3];      // per level: [n][2] FP32 box of each node's points
};
// Cells of the sorted points (key_bits = d * bits), then their boxes and tree.
void hd_cells(const void *X, int dtype, const RunParams &P, int key_bits, const HdBufs &H, const Bufs &B,
              DevCounters *ctr, cudaStream_t s);
void hd_tree(const RunParams &P, const HdBufs &H, const Bufs &B, DevCounters *ctr, cudaStream_t s);
// The forward neighbour lists (each unordered pair once, from its lower cell)
// into fwd (cap entries), one walk per 32 cells; ctr->E (zero before)
// receives their total, which exceeds cap if fwd was too small.
void hd_neighbors(const RunParams &P, const HdBufs &H, const Bufs &B, int *fwd, long long cap, DevCounters *ctr,
                  cudaStream_t s);
// The full lists from the forward ones (rank: as many entries as fwd; nbr:
// twice as many; H.bn, H.bf and, when used, B.nbr_pts zero before).
void hd_transpose(const RunParams &P, const HdBufs &H, const Bufs &B, const int *fwd, int *rank, int *nbr,
                  DevCounters *ctr, cudaStream_t s);
long long hd_scratch_ints();  // size of HdBufs::scratch

// full path compression of the cell union-find
void launch_uf_compress(int *parent, DevCounters *ctr, int max_iters, cudaStream_t s);
void launch_labels(const RunParams &P, const Bufs &B, uint8_t *core_out, int32_t *labels_out,
                   DevCounters *ctr, cudaStream_t s);
// count pass (fill = false; with the CSR offsets if offsets) or fill pass
// (fill = true, ids != null)
void launch_border(int D, int mode, bool fill, const RunParams &P, const Bufs &B, int32_t *labels_out,
                   int32_t *ids, long long ids_cap, DevCounters *ctr, cudaStream_t s, bool offsets = true);
void launch_border_offsets(const RunParams &P, const Bufs &B, cudaStream_t s);
// link witnesses of the last run in input indices (see k_witness_export)
void launch_witness_export(const Bufs &B, int n_core, const int2 *wit, long long nwit, int32_t *rep,
                           int32_t *links, cudaStream_t s);

}  // namespace gbdb
