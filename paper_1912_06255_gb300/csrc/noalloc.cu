// dbscan_run_static: the same exact DBSCAN as dbscan_run, for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework's memory pool or allocator, plugins whose host forbids device
// allocation after start-up, and callers that must not trigger the
// synchronisation a cudaMalloc/cudaFree may imply.  For them this entry point
// takes its working memory from one file-scope __device__ array of fixed size
// instead of a context workspace.  The caller still passes the input points
// and the output arrays.
//
// Limits: at most kStaticMaxPoints points, dimension at most kStaticMaxDim.
// The array (kStaticScratchBytes) is part of the library's device image, so
// every GPU that loads the library holds it until the process exits.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <vector>

#include "ctx.cuh"
#include "geom.cuh"

using namespace gbdb;

namespace {

constexpr int64_t kStaticMaxPoints = 16384;
constexpr int kStaticMaxDim = 3;
constexpr size_t kStaticScratchBytes = 20u << 20;  // 20 MiB, layout below needs ~19.6 MiB
constexpr int kMaxDevices = 64;

}  // namespace

// The scratch array.  In host code its name is only a host-side stand-in:
// the device address comes from cudaGetSymbolAddress in setup_device().
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

namespace {

struct StaticState {
    bool ready = false;
    unsigned char *base = nullptr;  // device address of g_static_scratch when set up
    dbscan_ctx ctx;                // views into g_static_scratch of this device
    gbdb::DevCounters h_ctr;       // host copies read back by the run
    long long h_bbox[2 * kMaxDim + 1];
    gbdb::Inst h_inst;
};

StaticState g_state[kMaxDevices];
std::mutex g_setup_mu;

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Lay the workspace of a context for kStaticMaxPoints x kStaticMaxDim out over
// the scratch array (same buffers as dbscan_create).  Returns the bytes used,
// or 0 if they do not fit.
size_t carve(dbscan_ctx *c, unsigned char *base) {
    const int64_t N = kStaticMaxPoints;
    const int SD = 4;
    c->max_points = N;
    c->max_dim = kStaticMaxDim;
    c->sd_max = SD;
    for (int d = 1; d <= kMaxEnumDim; ++d) c->noff[d] = num_offsets(d);
    int noff_max = 0;
    for (int d = 1; d <= kStaticMaxDim; ++d) noff_max = noff_max > c->noff[d] ? noff_max : c->noff[d];
    c->noff_max = noff_max;
    c->nbr_cap = (long long)noff_max * N + 1;
    const int64_t npart = scan_partials(N + 1) + 2;
    const uint64_t hcap = hash_capacity((int)N);
    c->sort_scratch_size = sort_scratch_bytes(N);
    c->bloom_lg = bloom_log2(N);
    struct Item { void **p; size_t bytes; };
    const Item items[] = {
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
        {(void **)&c->blo, 16 * (size_t)N}, {(void **)&c->bhi, 16 * (size_t)N},
        {(void **)&c->cblo, 16 * (size_t)N}, {(void **)&c->cbhi, 16 * (size_t)N},
        {(void **)&c->parent, 4 * (size_t)N}, {(void **)&c->compmin, 4 * (size_t)N},
        {(void **)&c->noncore, 4 * (size_t)N},
        {(void **)&c->bcount, 8 * (size_t)N}, {(void **)&c->boff, 8 * (size_t)(N + 1)},
        {(void **)&c->bbig, (size_t)N}, {(void **)&c->bcache, 8 * (size_t)N},
        {(void **)&c->bheavy, 4 * (size_t)N},
        {(void **)&c->bbox_out, 8 * (2 * kMaxDim + 1)},
        {(void **)&c->offs, (size_t)kMaxEnumDim * kMaxOffsets * kMaxEnumDim},
        {(void **)&c->ctr, sizeof(DevCounters)},
    };
    size_t at = 0;
    for (const Item &it : items) {
        *it.p = base + at;
        at += align256(it.bytes);
    }
    return at <= kStaticScratchBytes ? at : 0;
}

// With the device current: resolve the device address of the scratch array
// (every call: after a device reset or in another context the module is
// loaded again, possibly at another address) and, the first time or when
// the address moved, lay the workspace out over it and upload the neighbour
// offset tables (plain copies into the array; nothing is allocated).  The
// set-up ends with a device synchronisation, so its copies and clears are
// complete before any stream of the caller (blocking or not) uses the array.
dbscan_status setup_device(int dev) {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    StaticState &st = g_state[dev];
    unsigned char *base = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void **)&base, g_static_scratch);
    if (e != cudaSuccess || base == nullptr) {
        (void)cudaGetLastError();
        return DBSCAN_ERR_CUDA;
    }
    if (st.ready && st.base == base) return DBSCAN_OK;
    st.ready = false;
    st.ctx = dbscan_ctx();
    dbscan_ctx &c = st.ctx;
    c.device = dev;
    if (carve(&c, base) == 0) return DBSCAN_ERR_CAPACITY;
    for (int d = 1; d <= kMaxEnumDim; ++d) {
        std::vector<signed char> t = offset_table(d);
        e = cudaMemcpy(c.offs + (size_t)(d - 1) * kMaxOffsets * kMaxEnumDim, t.data(), t.size(),
                       cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return DBSCAN_ERR_CUDA;
        }
    }
    c.hcap = hash_capacity((int)kStaticMaxPoints);
    launch_table_clear(c.ht, c.hcap, 0);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return DBSCAN_ERR_CUDA;
    }
    c.table_clean = true;
    c.h_ctr = &st.h_ctr;
    c.h_bbox = st.h_bbox;
    c.h_inst = &st.h_inst;
    st.base = base;
    st.ready = true;
    return DBSCAN_OK;
}

}  // namespace

extern "C" dbscan_status dbscan_run_static(const void *d_points, int64_t n, int d, int dtype, double eps,
                                           int64_t min_pts, uint8_t *d_core, int32_t *d_labels,
                                           void *stream) {
    if (n < 0 || n > kStaticMaxPoints) return DBSCAN_ERR_CAPACITY;
    if (d < 1 || d > kStaticMaxDim) return DBSCAN_ERR_UNSUPPORTED_DIM;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return DBSCAN_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) return DBSCAN_ERR_CUDA;
    dbscan_status s = setup_device(dev);
    if (s != DBSCAN_OK) return s;
    // The run clears every counter and buffer that has to start at zero; the
    // rest of the array is overwritten before it is read.
    return dbscan_run(&g_state[dev].ctx, d_points, n, d, dtype, eps, min_pts, d_core, d_labels, nullptr,
                      nullptr, stream);
}
