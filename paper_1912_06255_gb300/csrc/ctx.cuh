// Host-side state of a dbscan_ctx (shared by the C-ABI translation units).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "internal.cuh"
#include "learned.cuh"

namespace gbdb {
struct SlabState;  // dbscan_run_slabs buffers (slab.cu)
// Neighbour-offset table of dimension d (<= kMaxEnumDim), kMaxEnumDim bytes per
// offset, nearest first; and its number of offsets.
std::vector<signed char> offset_table(int d);
int num_offsets(int d);
}  // namespace gbdb

constexpr int kPhases = 9;  // dbscan_stats.phase_ms

struct dbscan_ctx {
    int device = 0;
    int64_t max_points = 0;
    int max_dim = 0;
    int sd_max = 2;
    int noff_max = 0;
    // options
    int precision = DBSCAN_PREC_FP32_RECHECK;
    int sched = DBSCAN_SCHED_SIZE;
    int collect_stats = 0;
    int max_iters = 1 << 22;
    int phase_timing = 0;
    int cell_bounds = 1;
    int use_graph = 1;
    int cn_cells = 4;       // DBSCAN_OPT_CONNECT_CELLS
    int waves = 2;          // DBSCAN_OPT_CONNECT_WAVES
    int blocks_per_sm = 0;  // DBSCAN_OPT_BLOCKS_PER_SM
    int mc_small_nbr = 0;   // DBSCAN_OPT_SMALL_CELLS
    int pair_box = 1;       // DBSCAN_OPT_PAIR_BOXES
    double rho = 0.0;       // dbscan_set_approx: 0 = exact DBSCAN
    int witness = 0;        // DBSCAN_OPT_WITNESS
    int qt_levels = 0;      // DBSCAN_OPT_QUADTREE
    int slab_stage = 1;     // DBSCAN_OPT_SLAB_STAGE
    int nvtx = 0;           // DBSCAN_OPT_NVTX
    mutable int nvtx_open = 0;  // a phase range is open (closed by the next phase or an early return)
    int2 *wit = nullptr;    // [max_points] link witnesses (allocated while the option is on)
    long long wit_count = 0;
    bool have_wit = false;  // the last run recorded link witnesses
    cudaEvent_t ev[kPhases + 1] = {};
    // workspace
    void *arena = nullptr;
    size_t arena_bytes = 0;
    uint64_t *k0 = nullptr, *k1 = nullptr;
    uint32_t *v0 = nullptr, *v1 = nullptr;
    void *sort_scratch = nullptr;
    size_t sort_scratch_size = 0;
    long long *part = nullptr;
    uint32_t *slot_of = nullptr, *rank_of = nullptr, *slots = nullptr;  // cell grouping
    uint64_t hcap = 0;
    bool table_clean = false;  // every slot of ht empty ({kEmptyKey, 0})
    float *pf = nullptr, *cpf = nullptr;
    double *pd = nullptr, *cpd = nullptr;
    int *orig = nullptr, *cell_of = nullptr, *cell_start = nullptr;
    uint64_t *cell_key = nullptr;
    ulonglong2 *ht = nullptr;  // cell hash: 16-byte slots {key, cell id}
    int *nbr_cnt = nullptr;  // neighbours per cell; ids at nbr[c * noff(d)]
    int *nbr_near = nullptr; // of which adjacent (|delta|_inf <= 1), listed first
    int *nbr = nullptr;
    long long nbr_cap = 0;
    int *core_s = nullptr, *core_pos = nullptr, *ccs = nullptr, *core_orig = nullptr, *core_cell = nullptr;
    int *rank = nullptr;
    int *cell_inst = nullptr;      // [N] instance of each cell (batches)
    gbdb::Inst *d_inst = nullptr;  // instance table (device), one entry for single runs
    gbdb::Inst *h_inst = nullptr;  // pinned host copy
    int last_mode_sel = 0;
    // batches
    int batch_cap = 0;
    dbscan_instance *d_bdesc = nullptr, *h_bdesc = nullptr;
    gbdb::Inst *d_binst = nullptr;
    long long *d_bbox = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    cudaStream_t cap_stream = nullptr;
    long long graph_launches = 0;  // kernel nodes of the captured graph
    unsigned long long graph_key[14] = {0};
    float4 *blo = nullptr, *bhi = nullptr, *cblo = nullptr, *cbhi = nullptr;  // cell / core-point boxes
    float4 *ccent = nullptr;  // core-point centroids (learned schedule)
    // learned schedule: network (device), its Adam state, pair list, pair log
    float *mlp = nullptr;     // [4 * kMlpParams + 1]: weights, grad, m1, m2, loss
    int2 *lpairs = nullptr;
    void *lscratch = nullptr;
    size_t lscratch_size = 0;
    uint64_t *lk0 = nullptr, *lk1 = nullptr;
    long long lcap = 0;
    float *log_feat = nullptr;
    unsigned char *log_lab = nullptr;
    long long log_cap = 0, log_count = 0;
    int *parent = nullptr, *compmin = nullptr;
    int *noncore = nullptr;
    long long *bcount = nullptr, *boff = nullptr;
    unsigned char *bbig = nullptr;
    int2 *bcache = nullptr;
    int *bheavy = nullptr;
    long long *bbox_out = nullptr;  // [2*kMaxDim + 1], see launch_bbox
    signed char *offs = nullptr;  // [kMaxEnumDim][kMaxOffsets][kMaxEnumDim]
    int noff[gbdb::kMaxEnumDim + 1] = {0};
    int *nbr_pts = nullptr;     // points in all neighbouring cells, per cell
    unsigned *bloom = nullptr;  // Bloom filter of the cell keys of a hashed run (d <= 4)
    int bloom_lg = 10;
    // 5 <= d <= 8: cells, tree and CSR neighbour lists (allocated at the first such run)
    gbdb::HdBufs hd{};
    void *hd_arena = nullptr;
    void *qt_arena = nullptr;  // quadtree below the cells (allocated at the first run that uses it)
    int *hd_nbr = nullptr;  // lists that outgrow the arena's nbr buffer
    long long hd_nbr_cap = 0;
    int *nbr_cur = nullptr;                  // where the last run's neighbour lists live
    const long long *nbr_off_cur = nullptr;  // their CSR offsets (null: fixed stride)
    gbdb::DevCounters *ctr = nullptr;
    gbdb::SlabState *slab = nullptr;  // allocated at the first dbscan_run_slabs call
    // pinned host
    gbdb::DevCounters *h_ctr = nullptr;
    long long *h_bbox = nullptr;
    // host-buffer entry point
    void *d_in = nullptr;
    size_t d_in_bytes = 0;
    uint8_t *d_core_h = nullptr;
    int32_t *d_lab_h = nullptr;
    int64_t *d_off_h = nullptr;
    int32_t *d_ids_h = nullptr;
    int64_t d_ids_cap = 0;
    // last run
    bool have_run = false;
    bool boff_ready = false;  // the last run's border-set offsets are in boff
    gbdb::RunParams last{};
    int last_D = 0, last_mode = 0;
    const void *last_points = nullptr;
    int last_dtype = 0;
    dbscan_stats stats{};
    // DBSCAN_FAULT in the environment when the context was created (host-side
    // fault injection for the tests of the error paths): "alloc" makes every
    // allocation after dbscan_create fail like an exhausted device
    bool fault_alloc = false;
};

// NVTX range k of the run's phases (DBSCAN_OPT_NVTX): phase_range(c, k)
// closes the previous phase's range and opens phase k's; k = kPhases closes.
void phase_range(const dbscan_ctx *c, int k);
// A named range of its own (the slab steps), closed by range_pop.
void range_push(const dbscan_ctx *c, const char *name);
void range_pop(const dbscan_ctx *c);

// Device allocation of a context's lazily allocated buffers (fails with
// cudaErrorMemoryAllocation, allocating nothing, under DBSCAN_FAULT=alloc).
inline cudaError_t ctx_malloc(const dbscan_ctx *c, void **p, size_t bytes) {
    if (c->fault_alloc) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}
