// C ABI: context, workspace and the run sequence of Algorithm 1.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "ctx.cuh"
#include "geom.cuh"
#include "grid.cuh"
#include "inst.cuh"
#include "learned.cuh"

using namespace gbdb;

namespace gbdb {

// Candidate neighbour offsets of a d-dimensional cell (d <= 4): integer delta
// != 0 with sum_j max(|delta_j| - 1, 0)^2 <= d.  A pair within eps spans cells
// whose coordinates differ by delta with sum_j (|delta_j| - 1)_+^2 * s^2 < eps^2
// = d * s^2 for the exact side s = eps / sqrt(d); the side used is shrunk by
// 2^-20, which absorbs the rounding of the FP64 cell coordinates, so "<= d"
// keeps every such cell.  Sorted nearest first.
std::vector<signed char> offset_table(int d) {
    const int r = 1 + (int)std::floor(std::sqrt((double)d));
    std::vector<std::vector<int>> offs;
    std::vector<int> cur(d, -r);
    for (;;) {
        int bound = 0, nz = 0;
        for (int j = 0; j < d; ++j) {
            int a = std::abs(cur[j]) - 1;
            if (a > 0) bound += a * a;
            nz |= cur[j];
        }
        if (nz && bound <= d) offs.push_back(cur);
        int j = 0;
        while (j < d && ++cur[j] > r) cur[j++] = -r;
        if (j == d) break;
    }
    auto key = [d](const std::vector<int> &o) {
        int b = 0, e = 0;
        for (int j = 0; j < d; ++j) {
            int a = std::abs(o[j]) - 1;
            if (a > 0) b += a * a;
            e += o[j] * o[j];
        }
        return std::make_pair(b, e);
    };
    std::stable_sort(offs.begin(), offs.end(),
                     [&](const std::vector<int> &a, const std::vector<int> &b) { return key(a) < key(b); });
    std::vector<signed char> tab(offs.size() * kMaxEnumDim, 0);
    for (size_t i = 0; i < offs.size(); ++i)
        for (int j = 0; j < d; ++j) tab[i * kMaxEnumDim + j] = (signed char)offs[i][j];
    return tab;
}

int num_offsets(int d) { return (int)(offset_table(d).size() / kMaxEnumDim); }

}  // namespace gbdb

namespace {

constexpr int kVersion = 100;  // 0.1.0


size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace


static const char *const kPhaseRange[kPhases] = {
    "dbscan:bbox", "dbscan:bbox_readback", "dbscan:cells", "dbscan:boxes_lookup", "dbscan:neighbor_lists",
    "dbscan:markcore", "dbscan:compact_schedule", "dbscan:connect", "dbscan:labels_border"};

void phase_range(const dbscan_ctx *c, int k) {
    if (c->nvtx_open) {  // the previous phase's range, or one left open by a failed run
        nvtxRangePop();
        c->nvtx_open = 0;
    }
    if (c->nvtx && k >= 0 && k < kPhases) {
        nvtxRangePushA(kPhaseRange[k]);
        c->nvtx_open = 1;
    }
}
void range_push(const dbscan_ctx *c, const char *name) {
    if (c->nvtx) nvtxRangePushA(name);
}
void range_pop(const dbscan_ctx *c) {
    if (c->nvtx) nvtxRangePop();
}

static dbscan_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return DBSCAN_OK;
    if (e == cudaErrorMemoryAllocation) return DBSCAN_ERR_OOM;
    return DBSCAN_ERR_CUDA;
}

#define CK(x)                                                  \
    do {                                                       \
        cudaError_t e_ = (x);                                  \
        if (e_ != cudaSuccess) { (void)cudaGetLastError(); return cuda_status(e_); } \
    } while (0)

static Bufs make_bufs(dbscan_ctx *c, bool f64) {
    Bufs B{};
    B.pf = c->pf;
    B.pd = f64 ? c->pd : nullptr;
    B.orig = c->orig;
    B.cell_of = c->cell_of;
    B.cell_start = c->cell_start;
    B.nbr_cnt = c->nbr_cnt;
    B.nbr_near = c->nbr_near;
    B.nbr = c->nbr_cur ? c->nbr_cur : c->nbr;
    B.nbr_off = c->nbr_off_cur;
    B.nbr_pts = c->nbr_pts;
    B.core_s = c->core_s;
    B.core_pos = c->core_pos;
    B.ccs = c->ccs;
    B.cpf = c->cpf;
    B.cpd = f64 ? c->cpd : nullptr;
    B.core_orig = c->core_orig;
    B.core_cell = c->core_cell;
    B.blo = c->blo;
    B.bhi = c->bhi;
    B.cblo = c->cblo;
    B.cbhi = c->cbhi;
    B.ccent = (c->sched == DBSCAN_SCHED_LEARNED || c->log_cap > 0) ? c->ccent : nullptr;
    B.sk0 = c->k0;
    B.sk1 = c->k1;
    B.sv0 = c->v0;
    B.sv1 = c->v1;
    B.sort_scratch = c->sort_scratch;
    B.sort_scratch_size = c->sort_scratch_size;
    B.max_iters = c->max_iters;
    B.rank = c->rank;
    B.parent = c->parent;
    B.compmin = c->compmin;
    B.noncore = c->noncore;
    B.bcount = c->bcount;
    B.boff = c->boff;
    B.bbig = c->bbig;
    B.bcache = c->bcache;
    B.bheavy = c->bheavy;
    B.part = c->part;
    B.n_max = c->max_points;
    B.qt.levels = 0;
    if (c->qt_arena)
        for (int l = 0; l < 3; ++l) {
            B.qt.qpos[l] = c->hd.qpos[l];
            B.qt.qstart[l] = c->hd.qstart[l];
            B.qt.qlo[l] = c->hd.qlo[l];
            B.qt.qhi[l] = c->hd.qhi[l];
        }
    return B;
}

// Neighbour-offset table of dimension d inside the context.
static const signed char *offs_for(const dbscan_ctx *c, int d) {
    return c->offs + (size_t)(d - 1) * kMaxOffsets * kMaxEnumDim;
}

// Xavier-uniform weights, zero biases, from a splitmix64 stream of the seed;
// clears the Adam state.
static cudaError_t init_mlp(dbscan_ctx *c, uint64_t seed) {
    std::vector<float> h(4 * kMlpParams + 1, 0.f);
    uint64_t st = seed * 0x9e3779b97f4a7c15ull + 1;
    auto next = [&]() {
        uint64_t z = (st += 0x9e3779b97f4a7c15ull);
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        z ^= z >> 31;
        return (double)(z >> 11) * 0x1p-53;  // [0, 1)
    };
    auto fill = [&](int off, int fan_in, int fan_out) {
        const double a = std::sqrt(6.0 / (fan_in + fan_out));
        for (int i = 0; i < fan_in * fan_out; ++i) h[off + i] = (float)((2.0 * next() - 1.0) * a);
    };
    fill(kOW1, kMlpIn, kMlpHid);
    fill(kOW2, kMlpHid, kMlpHid);
    fill(kOW3, kMlpHid, 1);
    return cudaMemcpy(c->mlp, h.data(), sizeof(float) * h.size(), cudaMemcpyHostToDevice);
}

static Learned learned_state(dbscan_ctx *c) {
    Learned L{};
    L.w = c->mlp;
    L.pairs = c->lpairs;
    L.k0 = c->lk0;
    L.k1 = c->lk1;
    L.scratch = c->lscratch;
    L.scratch_size = c->lscratch_size;
    L.cap = c->lcap;
    L.log_feat = c->log_feat;
    L.log_lab = c->log_lab;
    L.log_cap = c->log_cap;
    return L;
}

// Pair list of the learned schedule: 16 pairs per point of capacity at first
// (grown by grow_learned when a run needs more).
static cudaError_t ensure_learned(dbscan_ctx *c, long long want = 0) {
    if (c->lpairs) return cudaSuccess;
    const long long cap = want > 0 ? want : 16 * std::max<int64_t>(c->max_points, 1);
    cudaError_t e = ctx_malloc(c, (void **)&c->lpairs, sizeof(int2) * cap);
    if (e == cudaSuccess) e = ctx_malloc(c, (void **)&c->lk0, sizeof(uint64_t) * cap);
    if (e == cudaSuccess) e = ctx_malloc(c, (void **)&c->lk1, sizeof(uint64_t) * cap);
    if (e == cudaSuccess) e = ctx_malloc(c, (void **)&c->lscratch, sort_scratch_bytes(cap));
    if (e == cudaSuccess) {
        c->lscratch_size = sort_scratch_bytes(cap);
        c->lcap = cap;
        return cudaSuccess;
    }
    cudaFree(c->lpairs);
    cudaFree(c->lk0);
    cudaFree(c->lk1);
    cudaFree(c->lscratch);
    c->lpairs = nullptr;
    c->lk0 = c->lk1 = nullptr;
    c->lscratch = nullptr;
    return e;
}

dbscan_status gbdb_enqueue_batch_prologue(dbscan_ctx *c, const void *d_points, int ld, int dtype, int count,
                                          long long n_total, int want_fp32, int key_limit, double rho,
                                          cudaStream_t s);
dbscan_status gbdb_batch_buffers(dbscan_ctx *c, const dbscan_instance *h, int count);
void gbdb_batch_free(dbscan_ctx *c);
void gbdb_slab_free(dbscan_ctx *c);

// Buffers of the tree-based neighbour search (5 <= d <= 8), one allocation.
static cudaError_t ensure_hd(dbscan_ctx *c) {
    if (c->hd_arena) return cudaSuccess;
    const size_t N = (size_t)std::max<int64_t>(c->max_points, 1);
    HdBufs &H = c->hd;
    struct Item { void **p; size_t bytes; };
    const Item items[] = {
        {(void **)&H.klo, 8 * N}, {(void **)&H.khi, 8 * N}, {(void **)&H.ckey_lo, 8 * N},
        {(void **)&H.ckey_hi, 8 * N}, {(void **)&H.ccoord, 16 * N}, {(void **)&H.child, 8 * N},
        {(void **)&H.parent, 4 * 2 * N}, {(void **)&H.flag, 4 * N}, {(void **)&H.nlo, 16 * N},
        {(void **)&H.nhi, 16 * N}, {(void **)&H.nbr_off, 8 * (N + 1)},
        {(void **)&H.scratch, sizeof(int) * (size_t)hd_scratch_ints()},
        {(void **)&H.nblo, 32 * N}, {(void **)&H.nbhi, 32 * N},
        {(void **)&H.nmax, 4 * N}, {(void **)&H.fwd_off, 8 * N},
        {(void **)&H.fn, 4 * N}, {(void **)&H.ff, 4 * N}, {(void **)&H.bn, 4 * N}, {(void **)&H.bf, 4 * N},
    };
    size_t total = 0;
    for (const auto &it : items) total += align_up(it.bytes);
    const cudaError_t e = ctx_malloc(c, (void **)&c->hd_arena, total);
    if (e != cudaSuccess) {
        c->hd_arena = nullptr;
        return e;
    }
    size_t at = 0;
    for (const auto &it : items) {
        *it.p = (char *)c->hd_arena + at;
        at += align_up(it.bytes);
    }
    return cudaSuccess;
}

// Buffers of the quadtree below the cells (5 <= d <= 8, MarkCore's range
// counts), one allocation for all three levels.
static cudaError_t ensure_qt(dbscan_ctx *c) {
    if (c->qt_arena) return cudaSuccess;
    const size_t N = (size_t)std::max<int64_t>(c->max_points, 1);
    HdBufs &H = c->hd;
    std::vector<std::pair<void **, size_t>> items = {{(void **)&H.qsub_in, 4 * N}, {(void **)&H.qsub, 4 * N}};
    for (int l = 0; l < 3; ++l) {
        items.push_back({(void **)&H.qpos[l], 4 * (N + 1)});
        items.push_back({(void **)&H.qstart[l], 4 * (N + 1)});
        items.push_back({(void **)&H.qlo[l], 32 * N});
        items.push_back({(void **)&H.qhi[l], 32 * N});
    }
    size_t total = 0;
    for (const auto &it : items) total += align_up(it.second);
    const cudaError_t e = ctx_malloc(c, &c->qt_arena, total);
    if (e != cudaSuccess) {
        c->qt_arena = nullptr;
        return e;
    }
    size_t at = 0;
    for (const auto &it : items) {
        *it.first = (char *)c->qt_arena + at;
        at += align_up(it.second);
    }
    return cudaSuccess;
}

// Steps 3-4 for 5 <= d <= 8: cells by a 128-bit key sort, the tree over the
// cells, then the neighbour lists in one walk per 32 cells into the larger of
// the arena's list buffer and the grown one.  One read-back checks the total:
// if the lists did not fit, the buffer grows and the walk runs again.
template <typename MarkFn>
static dbscan_status enqueue_hd_cells(dbscan_ctx *c, const RunParams &P, const void *d_points, int dtype,
                                      int key_bits, cudaStream_t s, MarkFn mark) {
    if (ensure_hd(c) != cudaSuccess) {
        (void)cudaGetLastError();
        return DBSCAN_ERR_OOM;
    }
    Bufs B = make_bufs(c, dtype == DBSCAN_F64);
    B.n_max = P.n;
    mark(2);
    hd_cells(d_points, dtype, P, key_bits, c->hd, B, c->ctr, s);
    mark(3);
    hd_tree(P, c->hd, B, c->ctr, s);
    mark(4);
    // one buffer of 4 F entries: the forward lists [F], their ranks in the
    // backward lists [F], the full lists [2 F]
    for (int attempt = 0; attempt < 2; ++attempt) {
        int *buf = c->hd_nbr_cap > c->nbr_cap ? c->hd_nbr : c->nbr;
        const long long capF = (c->hd_nbr_cap > c->nbr_cap ? c->hd_nbr_cap : c->nbr_cap) / 4;
        CK(cudaMemsetAsync(&c->ctr->E, 0, sizeof(long long), s));
        hd_neighbors(P, c->hd, B, buf, capF, c->ctr, s);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(c->h_ctr, c->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (c->h_ctr->err) return (dbscan_status)c->h_ctr->err;
        const long long E = c->h_ctr->E;
        if (E <= capF) {
            const size_t m = (size_t)c->h_ctr->m;
            CK(cudaMemsetAsync(c->hd.bn, 0, 4 * m, s));
            CK(cudaMemsetAsync(c->hd.bf, 0, 4 * m, s));
            if (P.mc_small_nbr > 0 && P.mc_small_nbr < (1 << 30)) CK(cudaMemsetAsync(c->nbr_pts, 0, 4 * m, s));
            hd_transpose(P, c->hd, B, buf, buf + capF, buf + 2 * capF, c->ctr, s);
            c->nbr_cur = buf + 2 * capF;
            c->nbr_off_cur = c->hd.nbr_off;
            return DBSCAN_OK;
        }
        cudaFree(c->hd_nbr);
        c->hd_nbr = nullptr;
        c->hd_nbr_cap = 0;
        const long long grown = 4 * (E + E / 4);
        if (ctx_malloc(c, (void **)&c->hd_nbr, sizeof(int) * (size_t)grown) != cudaSuccess) {
            (void)cudaGetLastError();
            c->hd_nbr = nullptr;
            return DBSCAN_ERR_OOM;
        }
        c->hd_nbr_cap = grown;
    }
    return DBSCAN_ERR_CAPACITY;
}

// Steps 3-4 for d <= 4: cells by the hash semisort, neighbour lists by
// offset enumeration through the hash (fixed stride per cell).
template <typename MarkFn>
static dbscan_status enqueue_hash_cells(dbscan_ctx *c, const RunParams &P, int SD, const void *d_points, int dtype,
                                        int d_enum, int sort_lo, int sort_bits, Semisort &S, cudaStream_t s,
                                        MarkFn mark) {
    const bool f64 = dtype == DBSCAN_F64;
    // 3. cells: group the points by cell (semisort, Sec. 4.1) through the cell hash
    mark(2);
    if (!c->table_clean) {
        launch_table_clear(c->ht, c->hcap, s);
    }
    c->table_clean = false;
    S.ht = c->ht;
    S.hcap = c->hcap;
    S.slot_of = c->slot_of;
    S.rank_of = c->rank_of;
    S.slots = c->slots;
    S.k0 = c->k0;
    S.k1 = c->k1;
    S.v0 = c->v0;
    S.v1 = c->v1;
    S.sort_scratch = c->sort_scratch;
    S.sort_scratch_size = c->sort_scratch_size;
    S.part = c->part;
    S.cell_key = c->cell_key;
    S.count = c->core_pos;  // scratch until the compaction
    S.cell_start = c->cell_start;
    S.pf = c->pf;
    S.pd = f64 ? c->pd : nullptr;
    S.orig = c->orig;
    S.cell_of = c->cell_of;
    S.cell_inst = c->cell_inst;
    // d = 2, 3: neighbours through supercells (blocks of 2^d cells), which
    // must be consecutive in the cell order: every key bit above the lowest d
    // is sorted, in whole 8-bit digits.  Otherwise whole digits only: the (at
    // most 7) lowest key bits left out of the order only shuffle cells inside a
    // block of 2^7 consecutive Z positions.
    S.super = d_enum == 2 || d_enum == 3;
    if (S.super) {
        const int top = sort_lo + sort_bits;
        const int digits = std::max(1, (sort_bits - d_enum + 7) / 8);
        S.key_lo = std::max(sort_lo, top - 8 * digits);
        S.key_bits = top - S.key_lo;
    } else {
        const int whole = sort_bits >= 8 ? sort_bits & ~7 : sort_bits;
        S.key_lo = sort_lo + (sort_bits - whole);
        S.key_bits = whole;
    }
    // the Bloom filter of the cell keys pays only when the hash table does not
    // fit in L2 (the supercell path keeps its own filter in the same storage)
    const bool use_bloom = 16 * c->hcap > ((uint64_t)96 << 20);
    S.n = P.n;
    S.bloom = use_bloom ? c->bloom : nullptr;
    S.bloom_all = c->bloom;
    S.bloom_lg = c->bloom_lg;
    if (use_bloom) CK(cudaMemsetAsync(c->bloom, 0, ((size_t)1 << c->bloom_lg) / 8, s));
    launch_semisort(d_points, dtype, P, SD, S, c->ctr, s);

    // 4. cell boxes, neighbour lists
    mark(3);
    if (P.box) launch_boxes(SD, c->pf, c->cell_start, c->ctr, c->blo, c->bhi, s);
    int *nbr_pts = P.mc_small_nbr > 0 && P.mc_small_nbr < (1 << 30) ? c->nbr_pts : nullptr;
    if (S.super) launch_super_table(S, P, c->ctr, s);  // returns at once on a dense grid
    mark(4);
    int n_near = 1;
    for (int j = 0; j < d_enum; ++j) n_near *= 3;
    // d = 2, 3: the offset enumeration runs only on a dense grid, the supercells only on a sparse one
    launch_neighbors(c->cell_key, c->ht, c->hcap, S.bloom, c->bloom_lg, P, offs_for(c, d_enum), c->noff[d_enum],
                     n_near - 1, c->blo, c->bhi, c->cell_start, c->nbr_cnt, c->nbr_near, nbr_pts, c->nbr, c->ctr,
                     s, S.super);
    if (S.super)
        launch_neighbors_super(S, P, c->noff[d_enum], c->blo, c->bhi, c->cell_start, c->nbr_cnt, c->nbr_near,
                               nbr_pts, c->nbr, c->ctr, s);
    c->nbr_cur = c->nbr;
    c->nbr_off_cur = nullptr;
    return DBSCAN_OK;
}

// Steps 3-10 of a run (cells, boxes, neighbour lists, MarkCore, compaction,
// schedule, BCP connectivity, labels, border counts), then the reset of the
// cell hash and the read-back of the device counters, all enqueued on s
// without a host synchronisation (so a batch can be captured in a graph).
template <typename MarkFn>
static dbscan_status enqueue_core(dbscan_ctx *c, const RunParams &P, int D, int SD, int mode, const void *d_points,
                                  int dtype, int d_enum, int sort_lo, int sort_bits, uint8_t *d_core,
                                  int32_t *d_labels, int64_t *d_border_offsets, cudaStream_t s, MarkFn mark) {
    const bool f64 = dtype == DBSCAN_F64;
    const int64_t n = P.n;
    const bool hashed = P.d <= kMaxEnumDim;
    Semisort S{};
    if (!hashed) {
        // 3-4. cells by key sort, neighbour lists by the tree over the cells
        const dbscan_status st = enqueue_hd_cells(c, P, d_points, dtype, sort_bits, s, mark);
        if (st != DBSCAN_OK) return st;
    } else {
        const dbscan_status st = enqueue_hash_cells(c, P, SD, d_points, dtype, d_enum, sort_lo, sort_bits, S, s, mark);
        if (st != DBSCAN_OK) return st;
    }

    // 5. MarkCore, 6. compaction, 7. schedule, 8. connect, 9. labels, 10. border
    Bufs B = make_bufs(c, f64);
    B.n_max = n;
    B.nbr_stride = hashed ? c->noff[d_enum] : 0;
    B.qt.levels = P.qt;
    mark(5);
    launch_markcore(D, mode, P, B, c->ctr, s);
    mark(6);
    launch_core_compact(SD, P, B, c->ctr, s);
    if (B.ccent) {
        // learned schedule (or a logging run for its training)
        if (ensure_learned(c) != cudaSuccess) {
            (void)cudaGetLastError();
            return DBSCAN_ERR_OOM;
        }
        mark(7);
        launch_connect_learned(D, mode, c->log_cap > 0, P, B, learned_state(c), c->ctr, s);
    } else {
        const uint32_t *order = launch_schedule(c->sched, P, B, c->ctr, s);
        mark(7);
        launch_connect(D, mode, order, P, B, c->ctr, s);
    }
    mark(8);
    launch_labels(P, B, d_core, d_labels, c->ctr, s);
    // the offsets only when the caller takes them now (else dbscan_border_ids scans them)
    launch_border(D, mode, false, P, B, d_labels, nullptr, 0, c->ctr, s, d_border_offsets != nullptr);
    c->boff_ready = d_border_offsets != nullptr;
    mark(9);
    if (hashed) launch_table_reset(S, c->ctr, s);
    if (d_border_offsets)
        CK(cudaMemcpyAsync(d_border_offsets, c->boff, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToDevice, s));
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(c->h_ctr, c->ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, s));
    return DBSCAN_OK;
}

// After the stream has been synchronised: counters into stats, state for
// dbscan_border_ids, status of the run.
static dbscan_status finish_run(dbscan_ctx *c, const RunParams &P, int D, int mode, const void *d_points, int dtype,
                                int64_t n, int64_t *num_border_memberships, long long launches0) {
    if (P.d <= kMaxEnumDim) c->table_clean = c->h_ctr->err == 0;  // runs of d >= 5 leave the hash alone
    const DevCounters &h = *c->h_ctr;
    dbscan_stats &st = c->stats;
    st.num_cells = h.m;
    st.num_core_cells = h.m_core;
    st.num_neighbor_entries = h.E;
    st.num_candidate_pairs = h.P;
    st.num_pairs_tested = (int64_t)h.pairs_tested;
    st.num_pairs_skipped = (int64_t)h.pairs_skipped;
    st.num_pairs_connected = (int64_t)h.pairs_linked;
    st.num_pairs_box_decided = (int64_t)h.pairs_box;
    st.num_core_points = h.n_core;
    st.num_border_points = h.n_border;
    st.num_noise_points = n - h.n_core - h.n_border;
    st.num_border_memberships = h.K;
    st.band_rechecks = (int64_t)h.band_rechecks;
    for (int k = 0; k < 3; ++k) st.distance_evals_phase[k] = (int64_t)h.dist_evals[k];
    st.distance_evals = st.distance_evals_phase[0] + st.distance_evals_phase[1] + st.distance_evals_phase[2];
    st.markcore_pair_bound = (int64_t)h.mc_bound;
    st.kernel_launches = g_launches - launches0;
    if (c->phase_timing) {
        for (int k = 0; k < kPhases; ++k)
            if (cudaEventElapsedTime(&st.phase_ms[k], c->ev[k], c->ev[k + 1]) != cudaSuccess) st.phase_ms[k] = 0.f;
        (void)cudaGetLastError();
    }
    if (c->log_cap > 0) c->log_count = std::min<long long>(h.P_list, c->log_cap);
    c->wit_count = (long long)h.n_wit;
    c->have_wit = P.wit != nullptr && h.err == 0;
    st.num_pairs_listed = h.P_list;
    if (h.err) return (dbscan_status)h.err;
    if (num_border_memberships) *num_border_memberships = h.K;
    c->have_run = true;
    c->last = P;
    c->last_D = D;
    c->last_mode = mode;
    c->last_points = d_points;
    c->last_dtype = dtype;
    return DBSCAN_OK;
}

extern "C" {

const char *dbscan_status_string(int s) {
    switch (s) {
    case DBSCAN_OK: return "ok";
    case DBSCAN_ERR_INVALID_ARG: return "invalid argument";
    case DBSCAN_ERR_UNSUPPORTED_DIM: return "unsupported dimension";
    case DBSCAN_ERR_OOM: return "out of memory";
    case DBSCAN_ERR_KEY_OVERFLOW: return "cell key overflow";
    case DBSCAN_ERR_CAPACITY: return "workspace capacity exceeded";
    case DBSCAN_ERR_CUDA: return "CUDA error";
    case DBSCAN_ERR_DEVICE_TIMEOUT: return "device retry limit reached";
    case DBSCAN_ERR_STATE: return "call out of order";
    default: return "unknown status";
    }
}

int dbscan_version(void) { return kVersion; }

void dbscan_destroy(dbscan_ctx *c) {
    if (!c) return;
    cudaDeviceSynchronize();
    cudaFree(c->arena);
    cudaFree(c->d_in);
    cudaFree(c->d_core_h);
    cudaFree(c->d_lab_h);
    cudaFree(c->d_off_h);
    cudaFree(c->d_ids_h);
    cudaFreeHost(c->h_ctr);
    cudaFreeHost(c->h_bbox);
    cudaFreeHost(c->h_inst);
    gbdb_batch_free(c);
    gbdb_slab_free(c);
    cudaFree(c->lpairs);
    cudaFree(c->lk0);
    cudaFree(c->lk1);
    cudaFree(c->lscratch);
    cudaFree(c->hd_arena);
    cudaFree(c->qt_arena);
    cudaFree(c->hd_nbr);
    cudaFree(c->log_feat);
    cudaFree(c->log_lab);
    cudaFree(c->wit);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    for (auto &e : c->ev)
        if (e) cudaEventDestroy(e);
    delete c;
}

dbscan_status dbscan_create(dbscan_ctx **out, int64_t max_points, int max_dim) {
    if (!out) return DBSCAN_ERR_INVALID_ARG;
    *out = nullptr;
    if (max_points < 0 || max_points >= 0x7ffffffell) return DBSCAN_ERR_INVALID_ARG;
    if (max_dim < 1 || max_dim > kMaxDim) return DBSCAN_ERR_UNSUPPORTED_DIM;
    const char *fault = std::getenv("DBSCAN_FAULT");
    if (fault && std::strstr(fault, "create")) return DBSCAN_ERR_OOM;  // injected: as if the arena did not fit
    dbscan_ctx *c = new (std::nothrow) dbscan_ctx();
    if (!c) return DBSCAN_ERR_OOM;
    c->fault_alloc = fault && std::strstr(fault, "alloc");
    cudaGetDevice(&c->device);
    const int64_t N = std::max<int64_t>(max_points, 1);
    c->max_points = max_points;
    c->max_dim = max_dim;
    c->sd_max = max_dim <= 2 ? 2 : (max_dim <= 4 ? 4 : 8);
    for (int d = 1; d <= kMaxEnumDim; ++d) c->noff[d] = num_offsets(d);
    int noff_max = 0;
    for (int d = 1; d <= std::min(max_dim, kMaxEnumDim); ++d) noff_max = std::max(noff_max, c->noff[d]);
    c->noff_max = noff_max;
    c->nbr_cap = (long long)noff_max * N + 1;
    const int64_t npart = scan_partials(N + 1) + 2;
    const uint64_t hcap = hash_capacity((int)N);
    c->sort_scratch_size = sort_scratch_bytes(N);
    c->bloom_lg = bloom_log2(N);
    const int SD = c->sd_max;
    const size_t BW = SD == 8 ? 2 : 1;  // float4 values per cell box

    // Carve one arena.
    struct Item { void **p; size_t bytes; };
    std::vector<Item> items = {
        {(void **)&c->k0, 8 * (size_t)N}, {(void **)&c->k1, 8 * (size_t)N},
        {(void **)&c->v0, 4 * (size_t)N}, {(void **)&c->v1, 4 * (size_t)N},
        {(void **)&c->sort_scratch, sort_scratch_bytes(N)}, {(void **)&c->part, 8 * (size_t)npart},
        {(void **)&c->slot_of, 4 * (size_t)N}, {(void **)&c->rank_of, 4 * (size_t)N},
        {(void **)&c->slots, 4 * (size_t)N},
        {(void **)&c->pf, 4 * (size_t)N * SD}, {(void **)&c->pd, 8 * (size_t)N * SD},
        {(void **)&c->cpf, 4 * (size_t)N * SD}, {(void **)&c->cpd, 8 * (size_t)N * SD},
        {(void **)&c->orig, 4 * (size_t)N}, {(void **)&c->cell_of, 4 * (size_t)N},
        {(void **)&c->cell_start, 4 * (size_t)(N + 1)}, {(void **)&c->cell_key, 8 * (size_t)N},
        {(void **)&c->ht, 16 * (size_t)hcap}, {(void **)&c->bloom, ((size_t)1 << bloom_log2(N)) / 8},
        {(void **)&c->nbr_cnt, 4 * (size_t)(N + 1)}, {(void **)&c->nbr_near, 4 * (size_t)(N + 1)},
        {(void **)&c->nbr_pts, 4 * (size_t)(N + 1)},
        {(void **)&c->nbr, 4 * (size_t)c->nbr_cap},
        {(void **)&c->core_s, 4 * (size_t)N}, {(void **)&c->core_pos, 4 * (size_t)(N + 1)},
        {(void **)&c->ccs, 4 * (size_t)(N + 1)}, {(void **)&c->core_orig, 4 * (size_t)N},
        {(void **)&c->core_cell, 4 * (size_t)N}, {(void **)&c->rank, 4 * (size_t)N},
        {(void **)&c->cell_inst, 4 * (size_t)N}, {(void **)&c->d_inst, sizeof(Inst)},
        {(void **)&c->ccent, BW * 16 * (size_t)N}, {(void **)&c->mlp, sizeof(float) * (4 * kMlpParams + 1)},
        {(void **)&c->blo, BW * 16 * (size_t)N}, {(void **)&c->bhi, BW * 16 * (size_t)N},
        {(void **)&c->cblo, BW * 16 * (size_t)N}, {(void **)&c->cbhi, BW * 16 * (size_t)N},
        {(void **)&c->parent, 4 * (size_t)N}, {(void **)&c->compmin, 4 * (size_t)N},
        {(void **)&c->noncore, 4 * (size_t)N},
        {(void **)&c->bcount, 8 * (size_t)N}, {(void **)&c->boff, 8 * (size_t)(N + 1)},
        {(void **)&c->bbig, (size_t)N}, {(void **)&c->bcache, 8 * (size_t)N},
        {(void **)&c->bheavy, 4 * (size_t)N},
        {(void **)&c->bbox_out, 8 * (2 * kMaxDim + 1)},
        {(void **)&c->offs, (size_t)kMaxEnumDim * kMaxOffsets * kMaxEnumDim},
        {(void **)&c->ctr, sizeof(DevCounters)},
    };
    size_t total = 0;
    for (auto &it : items) total += align_up(it.bytes);
    cudaError_t e = cudaMalloc(&c->arena, total);
    if (e != cudaSuccess) { (void)cudaGetLastError(); delete c; return cuda_status(e); }
    c->arena_bytes = total;
    size_t at = 0;
    for (auto &it : items) { *it.p = (char *)c->arena + at; at += align_up(it.bytes); }
    e = cudaMallocHost((void **)&c->h_ctr, sizeof(DevCounters));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&c->h_bbox, sizeof(long long) * (2 * kMaxDim + 1));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&c->h_inst, sizeof(Inst));
    for (int k = 0; k <= kPhases && e == cudaSuccess; ++k) e = cudaEventCreate(&c->ev[k]);
    for (int d = 1; d <= kMaxEnumDim && e == cudaSuccess; ++d) {
        std::vector<signed char> t = offset_table(d);
        e = cudaMemcpy(c->offs + (size_t)(d - 1) * kMaxOffsets * kMaxEnumDim, t.data(), t.size(),
                       cudaMemcpyHostToDevice);
    }
    c->hcap = hcap;
    if (e == cudaSuccess) e = init_mlp(c, 1);
    if (e == cudaSuccess) {
        launch_table_clear(c->ht, hcap, 0);
        e = cudaGetLastError();
    }
    // the clears and copies above run on the legacy stream: finish them before
    // a run on another (possibly non-blocking) stream reads the table
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    c->table_clean = e == cudaSuccess;
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        dbscan_destroy(c);
        return cuda_status(e);
    }
    *out = c;
    return DBSCAN_OK;
}

dbscan_status dbscan_set_option(dbscan_ctx *c, int option, int64_t value) {
    if (!c) return DBSCAN_ERR_INVALID_ARG;
    switch (option) {
    case DBSCAN_OPT_PRECISION:
        if (value != DBSCAN_PREC_FP64 && value != DBSCAN_PREC_FP32_RECHECK) return DBSCAN_ERR_INVALID_ARG;
        c->precision = (int)value;
        return DBSCAN_OK;
    case DBSCAN_OPT_SCHEDULE:
        if (value != DBSCAN_SCHED_SIZE && value != DBSCAN_SCHED_NONE && value != DBSCAN_SCHED_LEARNED)
            return DBSCAN_ERR_INVALID_ARG;
        c->sched = (int)value;
        return DBSCAN_OK;
    case DBSCAN_OPT_COLLECT_STATS:
        if (value != 0 && value != 1) return DBSCAN_ERR_INVALID_ARG;
        c->collect_stats = (int)value;
        return DBSCAN_OK;
    case DBSCAN_OPT_CELL_BOUNDS:
        if (value != 0 && value != 1) return DBSCAN_ERR_INVALID_ARG;
        c->cell_bounds = (int)value;
        return DBSCAN_OK;
    case DBSCAN_OPT_PAIR_LOG: {
        if (value < 0 || value > (1ll << 31)) return DBSCAN_ERR_INVALID_ARG;
        cudaFree(c->log_feat);
        cudaFree(c->log_lab);
        c->log_feat = nullptr;
        c->log_lab = nullptr;
        c->log_cap = 0;
        c->log_count = 0;
        if (value > 0) {
            cudaError_t e = ctx_malloc(c, (void **)&c->log_feat, sizeof(float) * kMlpIn * value);
            if (e == cudaSuccess) e = ctx_malloc(c, (void **)&c->log_lab, (size_t)value);
            if (e != cudaSuccess) {
                (void)cudaGetLastError();
                cudaFree(c->log_feat);
                c->log_feat = nullptr;
                return DBSCAN_ERR_OOM;
            }
            c->log_cap = value;
        }
        return DBSCAN_OK;
    }
    case DBSCAN_OPT_BATCH_GRAPH:
        if (value != 0 && value != 1) return DBSCAN_ERR_INVALID_ARG;
        c->use_graph = (int)value;
        return DBSCAN_OK;
    case DBSCAN_OPT_CONNECT_CELLS:
        if (value != 1 && value != 2 && value != 4 && value != 8) return DBSCAN_ERR_INVALID_ARG;
        c->cn_cells = (int)value;
        return DBSCAN_OK;
    case DBSCAN_OPT_CONNECT_WAVES:
        if (value != 1 && value != 2) return DBSCAN_ERR_INVALID_ARG;
        c->waves = (int)value;
        return DBSCAN_OK;
    case DBSCAN_OPT_BLOCKS_PER_SM:
        if (value < 0 || value > 32) return DBSCAN_ERR_INVALID_ARG;
        c->blocks_per_sm = (int)value;
        return DBSCAN_OK;
    case DBSCAN_OPT_SMALL_CELLS:
        if (value < 0 || value > (1ll << 30)) return DBSCAN_ERR_INVALID_ARG;
        c->mc_small_nbr = (int)value;
        return DBSCAN_OK;
    case DBSCAN_OPT_PAIR_BOXES:
        if (value != 0 && value != 1) return DBSCAN_ERR_INVALID_ARG;
        c->pair_box = (int)value;
        return DBSCAN_OK;
    case DBSCAN_OPT_QUADTREE:
        if (value < 0 || value > 3) return DBSCAN_ERR_INVALID_ARG;
        c->qt_levels = (int)value;
        return DBSCAN_OK;
    case DBSCAN_OPT_SLAB_STAGE:
        if (value != 0 && value != 1) return DBSCAN_ERR_INVALID_ARG;
        c->slab_stage = (int)value;
        return DBSCAN_OK;
    case DBSCAN_OPT_NVTX:
        if (value != 0 && value != 1) return DBSCAN_ERR_INVALID_ARG;
        c->nvtx = (int)value;
        return DBSCAN_OK;
    case DBSCAN_OPT_WITNESS:
        if (value != 0 && value != 1) return DBSCAN_ERR_INVALID_ARG;
        if (value && !c->wit) {
            if (ctx_malloc(c, (void **)&c->wit, sizeof(int2) * (size_t)std::max<int64_t>(c->max_points, 1)) !=
                cudaSuccess) {
                (void)cudaGetLastError();
                c->wit = nullptr;
                return DBSCAN_ERR_OOM;
            }
        }
        if (!value && c->wit) {
            cudaFree(c->wit);
            c->wit = nullptr;
        }
        c->witness = (int)value;
        c->have_wit = false;
        return DBSCAN_OK;
    case DBSCAN_OPT_PHASE_TIMING:
        if (value != 0 && value != 1) return DBSCAN_ERR_INVALID_ARG;
        c->phase_timing = (int)value;
        return DBSCAN_OK;
    case DBSCAN_OPT_MAX_ITERS:
        if (value < 1 || value > (1ll << 30)) return DBSCAN_ERR_INVALID_ARG;
        c->max_iters = (int)value;
        return DBSCAN_OK;
    default:
        return DBSCAN_ERR_INVALID_ARG;
    }
}

dbscan_status dbscan_get_option(const dbscan_ctx *c, int option, int64_t *value) {
    if (!c || !value) return DBSCAN_ERR_INVALID_ARG;
    switch (option) {
    case DBSCAN_OPT_PRECISION: *value = c->precision; return DBSCAN_OK;
    case DBSCAN_OPT_SCHEDULE: *value = c->sched; return DBSCAN_OK;
    case DBSCAN_OPT_COLLECT_STATS: *value = c->collect_stats; return DBSCAN_OK;
    case DBSCAN_OPT_MAX_ITERS: *value = c->max_iters; return DBSCAN_OK;
    case DBSCAN_OPT_PHASE_TIMING: *value = c->phase_timing; return DBSCAN_OK;
    case DBSCAN_OPT_CELL_BOUNDS: *value = c->cell_bounds; return DBSCAN_OK;
    case DBSCAN_OPT_BATCH_GRAPH: *value = c->use_graph; return DBSCAN_OK;
    case DBSCAN_OPT_PAIR_LOG: *value = c->log_cap; return DBSCAN_OK;
    case DBSCAN_OPT_CONNECT_CELLS: *value = c->cn_cells; return DBSCAN_OK;
    case DBSCAN_OPT_CONNECT_WAVES: *value = c->waves; return DBSCAN_OK;
    case DBSCAN_OPT_BLOCKS_PER_SM: *value = c->blocks_per_sm; return DBSCAN_OK;
    case DBSCAN_OPT_SMALL_CELLS: *value = c->mc_small_nbr; return DBSCAN_OK;
    case DBSCAN_OPT_PAIR_BOXES: *value = c->pair_box; return DBSCAN_OK;
    case DBSCAN_OPT_WITNESS: *value = c->witness; return DBSCAN_OK;
    case DBSCAN_OPT_QUADTREE: *value = c->qt_levels; return DBSCAN_OK;
    case DBSCAN_OPT_SLAB_STAGE: *value = c->slab_stage; return DBSCAN_OK;
    case DBSCAN_OPT_NVTX: *value = c->nvtx; return DBSCAN_OK;
    default: return DBSCAN_ERR_INVALID_ARG;
    }
}

dbscan_status dbscan_set_approx(dbscan_ctx *c, double rho) {
    if (!c || !(rho >= 0.0) || !(rho <= 1e6)) return DBSCAN_ERR_INVALID_ARG;
    c->rho = rho;
    return DBSCAN_OK;
}

dbscan_status dbscan_get_stats(const dbscan_ctx *c, dbscan_stats *out) {
    if (!c || !out) return DBSCAN_ERR_INVALID_ARG;
    *out = c->stats;
    return DBSCAN_OK;
}


static dbscan_status run_once(dbscan_ctx *c, const void *d_points, int64_t n, int d, int dtype, double eps,
                              int64_t min_pts, uint8_t *d_core, int32_t *d_labels, int64_t *d_border_offsets,
                              int64_t *num_border_memberships, void *stream) {
    if (!c) return DBSCAN_ERR_INVALID_ARG;
    c->have_run = false;
    c->have_wit = false;
    if (num_border_memberships) *num_border_memberships = 0;
    if (n < 0 || n > c->max_points) return DBSCAN_ERR_INVALID_ARG;
    if (d < 1 || d > c->max_dim) return DBSCAN_ERR_UNSUPPORTED_DIM;
    if (dtype != DBSCAN_F32 && dtype != DBSCAN_F64) return DBSCAN_ERR_INVALID_ARG;
    if (!(eps > 0.0) || !std::isfinite(eps) || min_pts < 1) return DBSCAN_ERR_INVALID_ARG;
    if (n > 0 && (!d_points || !d_core || !d_labels)) return DBSCAN_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    std::memset(&c->stats, 0, sizeof(c->stats));
    c->stats.schedule_used = c->sched;
    c->stats.rho = c->rho;
    c->stats.n = n;
    c->stats.d = d;
    if (n == 0) {
        if (d_border_offsets) CK(cudaMemsetAsync(d_border_offsets, 0, sizeof(int64_t), s));
        CK(cudaStreamSynchronize(s));
        c->have_run = true;
        c->have_wit = c->witness != 0;
        c->wit_count = 0;
        c->last = RunParams{};
        return DBSCAN_OK;
    }
    const bool f64 = dtype == DBSCAN_F64;
    const int D = d <= 2 ? 2 : (d <= 3 ? 3 : (d <= 4 ? 4 : 8));
    const long long launches0 = g_launches;
    auto mark = [&](int k) {
        if (c->phase_timing) cudaEventRecord(c->ev[k], s);
        phase_range(c, k);
    };
    mark(0);
    const int SD = D == 2 ? 2 : (D == 8 ? 8 : 4);  // storage width of Store<D>

    // 1. bounding box (one sync: it sizes the cell key)
    CK(cudaMemsetAsync(c->ctr, 0, sizeof(DevCounters), s));
    const int nbb = (int)std::min<int64_t>(4 * 152, std::max<int64_t>(1, (n + 255) / 256));
    launch_bbox(d_points, dtype, (int)n, d, nbb, c->bbox_out, s);
    mark(1);
    CK(cudaMemcpyAsync(c->h_bbox, c->bbox_out, sizeof(long long) * (2 * kMaxDim + 1), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    CK(cudaGetLastError());
    if (c->h_bbox[2 * kMaxDim] != 0) return DBSCAN_ERR_INVALID_ARG;

    // 2. grid parameters (Sec. 3), built on the host from the box
    RunParams P{};
    P.n = (int)n;
    P.d = d;
    P.max_iters = c->max_iters;
    P.cn_cells = c->cn_cells;
    P.waves = c->waves;
    P.mc_small_nbr = c->mc_small_nbr;
    P.pair_box = c->pair_box;
    P.wit = c->witness ? c->wit : nullptr;
    P.wit_cap = std::max<int64_t>(c->max_points, 1);
    set_grid_cap(c->blocks_per_sm);
    P.stats = c->collect_stats;
    P.ninst = 1;
    P.inst_shift = 64;
    {
        double lo[kMaxDim], hi[kMaxDim];
        for (int j = 0; j < d; ++j) {
            lo[j] = bbox_key_to_double(c->h_bbox[j]);
            hi[j] = bbox_key_to_double(c->h_bbox[kMaxDim + j]);
        }
        int fp32 = 0;
        Inst &I = c->h_inst[0];
        // 64-bit keys below 5 dimensions, 128-bit keys of at most 15 bits per dimension above
        const int key_limit = d <= kMaxEnumDim ? 63 : 15 * d;
        const int st = build_inst(I, eps, min_pts, (int)n, d, lo, hi, f64, c->precision == DBSCAN_PREC_FP32_RECHECK,
                                  key_limit, &fp32, c->rho);
        if (st != DBSCAN_OK) return (dbscan_status)st;
        I.row0 = 0;
        P.min_pts = I.thr.min_pts;
        P.eps2 = I.thr.eps2;
        P.lo = I.thr.lo;
        P.hi = I.thr.hi;
        c->stats.key_bits = d * I.bits;
        // d <= 4: the m cell keys, whole digits only; d >= 5: the n point keys
        c->stats.radix_passes = d <= kMaxEnumDim
                                    ? ((d == 2 || d == 3) ? std::max(1, (d * I.bits - d + 7) / 8)
                                                          : std::max(1, d * I.bits / 8))
                                    : (d * I.bits + 7) / 8;
        const int mode_sel = fp32 ? (f64 ? kF32FromF64 : kF32FromF32) : (f64 ? kF64FromF64 : kF64FromF32);
        c->last_mode_sel = mode_sel;
    }
    const int mode = c->last_mode_sel;
    CK(cudaMemcpyAsync(c->d_inst, c->h_inst, sizeof(Inst), cudaMemcpyHostToDevice, s));
    P.inst = c->d_inst;
    P.cell_inst = c->cell_inst;
    c->stats.precision = (mode == kF32FromF32 || mode == kF32FromF64) ? DBSCAN_PREC_FP32_RECHECK : DBSCAN_PREC_FP64;
    P.box = c->stats.precision == DBSCAN_PREC_FP32_RECHECK && c->cell_bounds ? 1 : 0;
    // the quadtree of the cells (Sec. 5.2) for MarkCore: d >= 5 with box bounds
    P.qt = d > kMaxEnumDim && P.box ? c->qt_levels : 0;
    if (P.qt > 0 && ensure_qt(c) != cudaSuccess) {
        (void)cudaGetLastError();
        return DBSCAN_ERR_OOM;
    }
    c->stats.band_lo = P.lo;
    c->stats.band_hi = P.hi;

    dbscan_status st = enqueue_core(c, P, D, SD, mode, d_points, dtype, d, 0, c->stats.key_bits, d_core, d_labels,
                                    d_border_offsets, s, mark);
    if (st != DBSCAN_OK) return st;
    CK(cudaStreamSynchronize(s));
    return finish_run(c, P, D, mode, d_points, dtype, n, num_border_memberships, launches0);
}

static dbscan_status run_batch_once(dbscan_ctx *c, const dbscan_instance *hi, int count, const void *d_points, int ld,
                               int dtype, uint8_t *d_core, int32_t *d_labels, int64_t *d_border_offsets,
                               int64_t *num_border_memberships, void *stream) {
    if (!c || !hi || count < 1) return DBSCAN_ERR_INVALID_ARG;
    c->have_run = false;
    c->have_wit = false;
    if (num_border_memberships) *num_border_memberships = 0;
    if (ld < 1 || ld > c->max_dim || ld > 3) return DBSCAN_ERR_UNSUPPORTED_DIM;
    if (dtype != DBSCAN_F32 && dtype != DBSCAN_F64) return DBSCAN_ERR_INVALID_ARG;
    int64_t total = 0;
    bool fp32_all = dtype == DBSCAN_F32 && c->precision == DBSCAN_PREC_FP32_RECHECK;
    for (int i = 0; i < count; ++i) {
        const dbscan_instance &I = hi[i];
        if (I.row0 != total || I.n < 0 || I.d < 1 || I.d > ld || !(I.eps > 0.0) || !std::isfinite(I.eps) ||
            I.min_pts < 1)
            return DBSCAN_ERR_INVALID_ARG;
        total += I.n;
        const double T = I.eps * I.eps;
        if (!(T >= 0x1p-60 && T <= 0x1p60)) fp32_all = false;
    }
    if (total > c->max_points) return DBSCAN_ERR_INVALID_ARG;
    if (total > 0 && (!d_points || !d_core || !d_labels)) return DBSCAN_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    std::memset(&c->stats, 0, sizeof(c->stats));
    c->stats.schedule_used = c->sched;
    c->stats.rho = c->rho;
    c->stats.n = total;
    c->stats.d = ld;
    if (total == 0) {
        if (d_border_offsets) CK(cudaMemsetAsync(d_border_offsets, 0, sizeof(int64_t), s));
        CK(cudaStreamSynchronize(s));
        c->have_run = true;
        c->have_wit = c->witness != 0;
        c->wit_count = 0;
        c->last = RunParams{};
        return DBSCAN_OK;
    }
    dbscan_status st = gbdb_batch_buffers(c, hi, count);
    if (st != DBSCAN_OK) return st;
    const bool f64 = dtype == DBSCAN_F64;
    const int D = ld <= 2 ? 2 : 3;
    const int SD = D == 2 ? 2 : 4;
    const int mode = fp32_all ? kF32FromF32 : (f64 ? kF64FromF64 : kF64FromF32);
    int inst_bits = 1;
    while ((1 << inst_bits) < count) ++inst_bits;
    RunParams P{};
    P.n = (int)total;
    P.d = ld;
    P.max_iters = c->max_iters;
    P.cn_cells = c->cn_cells;
    P.waves = c->waves;
    P.mc_small_nbr = c->mc_small_nbr;
    P.pair_box = c->pair_box;
    P.wit = c->witness ? c->wit : nullptr;
    P.wit_cap = std::max<int64_t>(c->max_points, 1);
    set_grid_cap(c->blocks_per_sm);
    P.stats = c->collect_stats;
    P.box = fp32_all && c->cell_bounds ? 1 : 0;
    P.ninst = count;
    P.inst_shift = 63 - inst_bits;
    P.inst = c->d_binst;
    P.cell_inst = c->cell_inst;
    c->stats.precision = fp32_all ? DBSCAN_PREC_FP32_RECHECK : DBSCAN_PREC_FP64;
    c->stats.key_bits = 63;
    c->stats.radix_passes = ld >= 2 ? 8 : 7;
    const long long launches0 = g_launches;
    if (!c->table_clean) {
        launch_table_clear(c->ht, c->hcap, s);
        c->table_clean = true;
    }
    // The cell sort orders by all 63 key bits: instance, then Z order inside
    // it.  (An instance's Morton code occupies only the low d * bits, so a sort
    // of the top bits alone would leave each instance's cells unordered.)
    auto enqueue = [&]() -> dbscan_status {
        if (c->phase_timing) cudaEventRecord(c->ev[0], s);
        if (c->phase_timing) cudaEventRecord(c->ev[1], s);
        dbscan_status e = gbdb_enqueue_batch_prologue(c, d_points, ld, dtype, count, total, fp32_all ? 1 : 0,
                                                      P.inst_shift, c->rho, s);
        if (e != DBSCAN_OK) return e;
        return enqueue_core(c, P, D, SD, mode, d_points, dtype, ld, 0, 63, d_core, d_labels, d_border_offsets, s,
                            [&](int k) {
                                if (c->phase_timing) cudaEventRecord(c->ev[k], s);
                            });
    };
    unsigned long long rho_bits = 0;
    std::memcpy(&rho_bits, &c->rho, sizeof rho_bits);
    const unsigned long long key[14] = {(unsigned long long)count, (unsigned long long)total,
                                        (unsigned long long)(uintptr_t)d_points, (unsigned long long)ld,
                                        (unsigned long long)dtype, (unsigned long long)(uintptr_t)d_core,
                                        (unsigned long long)(uintptr_t)d_labels,
                                        (unsigned long long)(uintptr_t)d_border_offsets,
                                        (unsigned long long)(mode | (c->sched << 4) | (P.box << 8) | (P.stats << 9) |
                                                             ((c->log_cap > 0) << 10) | (c->pair_box << 11) | (c->cn_cells << 12) |
                                                             (c->waves << 20) | (c->blocks_per_sm << 24)),
                                        (unsigned long long)c->mc_small_nbr ^ ((unsigned long long)c->lcap << 31),
                                        (unsigned long long)c->phase_timing, (unsigned long long)c->max_iters,
                                        1ull | ((unsigned long long)c->witness << 1), rho_bits};
    // phase timing records events between the steps: that run is enqueued
    // directly instead of replaying the graph
    if (!c->use_graph || c->phase_timing) {
        st = enqueue();
        if (st != DBSCAN_OK) return st;
    } else {
        if (!c->graph_exec || std::memcmp(key, c->graph_key, sizeof key) != 0) {
            if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
            c->graph_exec = nullptr;
            // capture on a private stream (the legacy default stream cannot be
            // captured); the graph then runs on the caller's stream
            if (!c->cap_stream) CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
            cudaGraph_t graph = nullptr;
            const cudaStream_t user = s;
            s = c->cap_stream;
            CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
            const long long l0 = g_launches;
            st = enqueue();
            c->graph_launches = g_launches - l0;
            cudaError_t e = cudaStreamEndCapture(s, &graph);
            s = user;
            if (st != DBSCAN_OK) {
                if (graph) cudaGraphDestroy(graph);
                (void)cudaGetLastError();
                return st;
            }
            CK(e);
            e = cudaGraphInstantiate(&c->graph_exec, graph, 0);
            cudaGraphDestroy(graph);
            CK(e);
            std::memcpy(c->graph_key, key, sizeof key);
        }
        c->table_clean = false;
        CK(cudaGraphLaunch(c->graph_exec, s));
        g_launches += c->graph_launches;  // kernels the replay runs
    }
    CK(cudaStreamSynchronize(s));
    return finish_run(c, P, D, mode, d_points, dtype, total, num_border_memberships, launches0);
}

// The learned schedule's pair list starts at 16 pairs per point; a run that
// needs more reports CAPACITY with the demand, the list grows, and the run is
// repeated once.  A demand beyond 2^31 pairs (the pair sort's limit), or one
// the device cannot hold, falls back to the size schedule for that call.
static bool pair_list_full(const dbscan_ctx *c) {
    return c->h_ctr->err == DBSCAN_ERR_CAPACITY && c->h_ctr->err_info == 50;
}

static bool grow_learned(dbscan_ctx *c) {
    const unsigned long long demand = c->h_ctr->P_demand;
    if (demand >= (1ull << 31) - 1024) return false;
    const long long want = std::min<long long>(std::max<long long>(2 * c->lcap, (long long)(demand * 5 / 4) + 1024),
                                               (1ll << 31) - 1);
    cudaFree(c->lpairs);
    cudaFree(c->lk0);
    cudaFree(c->lk1);
    cudaFree(c->lscratch);
    c->lpairs = nullptr;
    c->lk0 = c->lk1 = nullptr;
    c->lscratch = nullptr;
    c->lcap = 0;
    if (ensure_learned(c, want) == cudaSuccess) return true;
    (void)cudaGetLastError();
    return false;
}

// Runs fn; on a full pair list, grows it and runs again, else runs once more
// with the size schedule.
extern "C++" {
template <typename Fn> dbscan_status with_pair_list_retry(dbscan_ctx *c, Fn fn) {
    dbscan_status st = fn();
    if (st != DBSCAN_ERR_CAPACITY || !pair_list_full(c)) return st;
    if (grow_learned(c)) {
        st = fn();
        if (st != DBSCAN_ERR_CAPACITY || !pair_list_full(c)) return st;
    }
    const int sched = c->sched;
    const long long log_cap = c->log_cap;
    c->sched = DBSCAN_SCHED_SIZE;
    c->log_cap = 0;  // a logging run needs the full list: this call logs nothing
    st = fn();
    c->sched = sched;
    c->log_cap = log_cap;
    c->stats.schedule_used = DBSCAN_SCHED_SIZE;
    return st;
}
}  // extern "C++"

dbscan_status dbscan_run(dbscan_ctx *c, const void *d_points, int64_t n, int d, int dtype, double eps,
                         int64_t min_pts, uint8_t *d_core, int32_t *d_labels, int64_t *d_border_offsets,
                         int64_t *num_border_memberships, void *stream) {
    if (!c) return DBSCAN_ERR_INVALID_ARG;
    return with_pair_list_retry(c, [&]() {
        return run_once(c, d_points, n, d, dtype, eps, min_pts, d_core, d_labels, d_border_offsets,
                        num_border_memberships, stream);
    });
}

dbscan_status dbscan_run_batch(dbscan_ctx *c, const dbscan_instance *hi, int count, const void *d_points, int ld,
                               int dtype, uint8_t *d_core, int32_t *d_labels, int64_t *d_border_offsets,
                               int64_t *num_border_memberships, void *stream) {
    if (!c) return DBSCAN_ERR_INVALID_ARG;
    return with_pair_list_retry(c, [&]() {
        return run_batch_once(c, hi, count, d_points, ld, dtype, d_core, d_labels, d_border_offsets,
                              num_border_memberships, stream);
    });
}

dbscan_status dbscan_train_scheduler(dbscan_ctx *c, int epochs, int batch, float lr, uint64_t seed, float *h_losses) {
    if (!c || epochs < 1 || batch < 1 || !(lr > 0.f)) return DBSCAN_ERR_INVALID_ARG;
    const long long n = c->log_count;
    if (n <= 0) return DBSCAN_ERR_STATE;
    CK(init_mlp(c, seed));
    float *w = c->mlp, *g = c->mlp + kMlpParams, *m1 = g + kMlpParams, *m2 = m1 + kMlpParams, *loss = m2 + kMlpParams;
    const long long nb = std::min<long long>(batch, n);
    const long long steps = (n + nb - 1) / nb;
    int t = 0;
    uint64_t st = seed ^ 0x5bd1e995ull;
    for (int ep = 0; ep < epochs; ++ep) {
        CK(cudaMemset(loss, 0, sizeof(float)));
        st = st * 6364136223846793005ull + 1442695040888963407ull;
        const long long start = (long long)((st >> 17) % (uint64_t)n);
        for (long long k = 0; k < steps; ++k) {
            CK(cudaMemsetAsync(g, 0, sizeof(float) * kMlpParams, 0));
            mlp_loss_grad(w, c->log_feat, c->log_lab, (start + k * nb) % n, nb, n, g, loss, 0);
            mlp_adam(w, g, m1, m2, lr, ++t, 0);
        }
        float l = 0.f;
        CK(cudaMemcpy(&l, loss, sizeof(float), cudaMemcpyDeviceToHost));
        if (h_losses) h_losses[ep] = l / (float)steps;
    }
    CK(cudaGetLastError());
    return DBSCAN_OK;
}

dbscan_status dbscan_scheduler_weights(dbscan_ctx *c, float *h_weights, int count, int set) {
    if (!c || !h_weights || count != kMlpParams) return DBSCAN_ERR_INVALID_ARG;
    CK(cudaMemcpy(set ? (void *)c->mlp : (void *)h_weights, set ? (const void *)h_weights : (const void *)c->mlp,
                  sizeof(float) * kMlpParams, set ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost));
    return DBSCAN_OK;
}

dbscan_status dbscan_scheduler_loss_grad(dbscan_ctx *c, const float *d_features, const uint8_t *d_labels,
                                         int64_t n, float *h_loss, float *h_grad) {
    if (!c || !d_features || !d_labels || n < 1 || !h_loss || !h_grad) return DBSCAN_ERR_INVALID_ARG;
    float *g = c->mlp + kMlpParams, *loss = c->mlp + 4 * kMlpParams;
    CK(cudaMemset(g, 0, sizeof(float) * kMlpParams));
    CK(cudaMemset(loss, 0, sizeof(float)));
    mlp_loss_grad(c->mlp, d_features, d_labels, 0, n, n, g, loss, 0);
    CK(cudaGetLastError());
    CK(cudaMemcpy(h_grad, g, sizeof(float) * kMlpParams, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(h_loss, loss, sizeof(float), cudaMemcpyDeviceToHost));
    return DBSCAN_OK;
}

dbscan_status dbscan_get_pair_log(dbscan_ctx *c, float *d_features, uint8_t *d_labels, int64_t capacity,
                                  int64_t *count) {
    if (!c || !count) return DBSCAN_ERR_INVALID_ARG;
    *count = c->log_count;
    if (c->log_count == 0) return DBSCAN_OK;
    if (capacity < c->log_count || !d_features || !d_labels) return DBSCAN_ERR_CAPACITY;
    CK(cudaMemcpy(d_features, c->log_feat, sizeof(float) * kMlpIn * c->log_count, cudaMemcpyDeviceToDevice));
    CK(cudaMemcpy(d_labels, c->log_lab, (size_t)c->log_count, cudaMemcpyDeviceToDevice));
    return DBSCAN_OK;
}

dbscan_status dbscan_border_ids(dbscan_ctx *c, int32_t *d_ids, int64_t capacity, void *stream) {
    if (!c || capacity < 0) return DBSCAN_ERR_INVALID_ARG;
    if (!c->have_run) return DBSCAN_ERR_STATE;
    if (capacity < c->stats.num_border_memberships) return DBSCAN_ERR_CAPACITY;
    if (c->stats.num_border_memberships == 0) return DBSCAN_OK;
    if (!d_ids) return DBSCAN_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const bool f64 = c->last_dtype == DBSCAN_F64;
    Bufs B = make_bufs(c, f64);
    B.n_max = c->last.n;
    B.nbr_stride = c->last.d <= kMaxEnumDim ? c->noff[c->last.d] : 0;
    CK(cudaMemsetAsync(&c->ctr->err, 0, sizeof(int), s));
    const long long l0 = g_launches;
    if (!c->boff_ready) {
        launch_border_offsets(c->last, B, s);
        c->boff_ready = true;
    }
    launch_border(c->last_D, c->last_mode, true, c->last, B, nullptr, d_ids, capacity, c->ctr, s);
    c->stats.kernel_launches += g_launches - l0;  // the run's count includes its border fill
    CK(cudaGetLastError());
    int err = 0;
    CK(cudaMemcpyAsync(&c->h_ctr->err, &c->ctr->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    err = c->h_ctr->err;
    return err ? (dbscan_status)err : DBSCAN_OK;
}

dbscan_status dbscan_link_witnesses(dbscan_ctx *c, int32_t *d_rep, int32_t *d_links, int64_t capacity,
                                    int64_t *count, void *stream) {
    if (!c || !count || capacity < 0) return DBSCAN_ERR_INVALID_ARG;
    *count = 0;
    if (!c->have_run || !c->have_wit) return DBSCAN_ERR_STATE;
    *count = c->wit_count;
    if (capacity < c->wit_count) return DBSCAN_ERR_CAPACITY;
    const int64_t n = c->stats.n;
    if (n == 0) return DBSCAN_OK;
    if (!d_rep || (c->wit_count > 0 && !d_links)) return DBSCAN_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    Bufs B = make_bufs(c, c->last_dtype == DBSCAN_F64);
    CK(cudaMemsetAsync(d_rep, 0xff, sizeof(int32_t) * (size_t)n, s));
    launch_witness_export(B, (int)c->stats.num_core_points, c->wit, c->wit_count, d_rep, d_links, s);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));
    return DBSCAN_OK;
}

// Device buffers of the host-buffer entry points: input (max_points x
// max_dim doubles), core flags, labels, border offsets (allocated at the first
// call) and border ids (grown to the largest set length seen).
static dbscan_status ensure_host_bufs(dbscan_ctx *c, int64_t ids_need) {
    if (!c->d_in) {
        const size_t need = std::max<size_t>((size_t)c->max_points * c->max_dim * 8, 8);
        const int64_t N = std::max<int64_t>(c->max_points, 1);
        cudaError_t e = ctx_malloc(c, (void **)&c->d_in, need);
        if (e == cudaSuccess) e = ctx_malloc(c, (void **)&c->d_core_h, (size_t)N);
        if (e == cudaSuccess) e = ctx_malloc(c, (void **)&c->d_lab_h, 4 * (size_t)N);
        if (e == cudaSuccess) e = ctx_malloc(c, (void **)&c->d_off_h, 8 * (size_t)(N + 1));
        if (e != cudaSuccess) {  // all or nothing: a later call allocates again
            (void)cudaGetLastError();
            cudaFree(c->d_in);
            cudaFree(c->d_core_h);
            cudaFree(c->d_lab_h);
            cudaFree(c->d_off_h);
            c->d_in = nullptr;
            c->d_core_h = nullptr;
            c->d_lab_h = nullptr;
            c->d_off_h = nullptr;
            return cuda_status(e);
        }
        c->d_in_bytes = need;
    }
    if (ids_need > c->d_ids_cap) {
        cudaFree(c->d_ids_h);
        c->d_ids_h = nullptr;
        c->d_ids_cap = 0;
        const int64_t cap = std::max<int64_t>(ids_need + ids_need / 4, 1024);
        CK(ctx_malloc(c, (void **)&c->d_ids_h, 4 * (size_t)cap));
        c->d_ids_cap = cap;
    }
    return DBSCAN_OK;
}

// After a run on the context's device buffers: core flags, labels and, when
// asked for, the border CSR back to the host.
static dbscan_status host_outputs(dbscan_ctx *c, int64_t n, uint8_t *h_core, int32_t *h_labels,
                                  int64_t *h_border_offsets, int32_t *h_border_ids, int64_t ids_capacity, int64_t K,
                                  cudaStream_t s) {
    if (n > 0) {
        CK(cudaMemcpyAsync(h_core, c->d_core_h, (size_t)n, cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(h_labels, c->d_lab_h, 4 * (size_t)n, cudaMemcpyDeviceToHost, s));
        if (h_border_offsets)
            CK(cudaMemcpyAsync(h_border_offsets, c->d_off_h, 8 * (size_t)(n + 1), cudaMemcpyDeviceToHost, s));
    } else if (h_border_offsets) {
        h_border_offsets[0] = 0;
    }
    if (h_border_ids && K > 0) {
        if (K > ids_capacity) return DBSCAN_ERR_CAPACITY;
        const dbscan_status st = ensure_host_bufs(c, K);
        if (st != DBSCAN_OK) return st;
        const dbscan_status sb = dbscan_border_ids(c, c->d_ids_h, c->d_ids_cap, s);
        if (sb != DBSCAN_OK) return sb;
        CK(cudaMemcpyAsync(h_border_ids, c->d_ids_h, 4 * (size_t)K, cudaMemcpyDeviceToHost, s));
    }
    CK(cudaStreamSynchronize(s));
    return DBSCAN_OK;
}

dbscan_status dbscan_run_host(dbscan_ctx *c, const void *h_points, int64_t n, int d, int dtype, double eps,
                              int64_t min_pts, uint8_t *h_core, int32_t *h_labels, int64_t *h_border_offsets,
                              int32_t *h_border_ids, int64_t ids_capacity, int64_t *num_border_memberships,
                              void *stream) {
    if (!c) return DBSCAN_ERR_INVALID_ARG;
    if (num_border_memberships) *num_border_memberships = 0;
    if (n < 0 || n > c->max_points || d < 1 || d > c->max_dim) return DBSCAN_ERR_INVALID_ARG;
    if (dtype != DBSCAN_F32 && dtype != DBSCAN_F64) return DBSCAN_ERR_INVALID_ARG;
    if (n > 0 && (!h_points || !h_core || !h_labels)) return DBSCAN_ERR_INVALID_ARG;
    if (h_border_ids && (!h_border_offsets || ids_capacity < 0)) return DBSCAN_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = (size_t)n * d * (dtype == DBSCAN_F64 ? 8 : 4);
    dbscan_status st = ensure_host_bufs(c, 0);
    if (st != DBSCAN_OK) return st;
    if (n > 0) CK(cudaMemcpyAsync(c->d_in, h_points, bytes, cudaMemcpyHostToDevice, s));
    int64_t K = 0;
    st = dbscan_run(c, c->d_in, n, d, dtype, eps, min_pts, c->d_core_h, c->d_lab_h,
                    h_border_offsets ? c->d_off_h : nullptr, &K, stream);
    if (st != DBSCAN_OK) return st;
    if (num_border_memberships) *num_border_memberships = K;
    return host_outputs(c, n, h_core, h_labels, h_border_offsets, h_border_ids, ids_capacity, K, s);
}

dbscan_status dbscan_run_batch_host(dbscan_ctx *c, const dbscan_instance *h_instances, int count,
                                    const void *h_points, int ld, int dtype, uint8_t *h_core, int32_t *h_labels,
                                    int64_t *h_border_offsets, int32_t *h_border_ids, int64_t ids_capacity,
                                    int64_t *num_border_memberships, void *stream) {
    if (!c || !h_instances || count < 1) return DBSCAN_ERR_INVALID_ARG;
    if (num_border_memberships) *num_border_memberships = 0;
    if (ld < 1 || ld > c->max_dim) return DBSCAN_ERR_UNSUPPORTED_DIM;
    if (dtype != DBSCAN_F32 && dtype != DBSCAN_F64) return DBSCAN_ERR_INVALID_ARG;
    int64_t N = 0;
    for (int i = 0; i < count; ++i) {
        if (h_instances[i].n < 0) return DBSCAN_ERR_INVALID_ARG;
        N += h_instances[i].n;
    }
    if (N > c->max_points) return DBSCAN_ERR_INVALID_ARG;
    if (N > 0 && (!h_points || !h_core || !h_labels)) return DBSCAN_ERR_INVALID_ARG;
    if (h_border_ids && (!h_border_offsets || ids_capacity < 0)) return DBSCAN_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    dbscan_status st = ensure_host_bufs(c, 0);
    if (st != DBSCAN_OK) return st;
    if (N > 0)
        CK(cudaMemcpyAsync(c->d_in, h_points, (size_t)N * ld * (dtype == DBSCAN_F64 ? 8 : 4), cudaMemcpyHostToDevice,
                           s));
    int64_t K = 0;
    st = dbscan_run_batch(c, h_instances, count, c->d_in, ld, dtype, c->d_core_h, c->d_lab_h,
                          h_border_offsets ? c->d_off_h : nullptr, &K, stream);
    if (st != DBSCAN_OK) return st;
    if (num_border_memberships) *num_border_memberships = K;
    return host_outputs(c, N, h_core, h_labels, h_border_offsets, h_border_ids, ids_capacity, K, s);
}

}  // extern "C"
