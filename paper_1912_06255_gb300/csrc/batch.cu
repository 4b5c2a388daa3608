// dbscan_run_batch: many independent problem instances in one pass of the
// same persistent kernels, captured once as a CUDA graph and replayed.
//
// Every instance gets its own grid (origin, cell side eps/sqrt(d), key bits)
// and thresholds (eps^2, FP32 band, minPts), built on the device from its own
// bounding box; its id sits in the top bits of its cell keys, so cells,
// neighbour lists, BCP pairs and union-find sets never mix instances.  The
// kernels take cells and cell pairs from global work counters, so uneven
// instance sizes balance out across the GPU.  Nothing in the sequence waits
// for the host, which is what lets it be captured.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "ctx.cuh"
#include "geom.cuh"
#include "grid.cuh"
#include "inst.cuh"

using namespace gbdb;

namespace {

constexpr int BB_CHUNK = 4096;  // rows per warp work item of the box reduction
constexpr int BB_SLOTS = 2 * kMaxDim + 1;

__device__ __forceinline__ long long okey(double x) {
    const long long b = __double_as_longlong(x);
    return b >= 0 ? b : (b ^ 0x7fffffffffffffffll);
}
__device__ __forceinline__ double okey_to_double(long long k) {
    return __longlong_as_double(k >= 0 ? k : (k ^ 0x7fffffffffffffffll));
}

__device__ __forceinline__ int find_inst(const dbscan_instance *desc, int count, long long row) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (desc[mid].row0 <= row) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void k_bb_init(long long *bb, int count) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count * BB_SLOTS; i += gridDim.x * blockDim.x) {
        const int j = i % BB_SLOTS;
        bb[i] = j < kMaxDim ? 0x7fffffffffffffffll : (j < 2 * kMaxDim ? (long long)0x8000000000000000ull : 0);
    }
}

// Extremes kept per lane in the input's own type (FP32 min/max, or the
// order-preserving integer keys of FP64 values), merged as FP64 keys.
template <typename T> struct BbAcc;
template <> struct BbAcc<float> {
    float mn[kMaxDim], mx[kMaxDim];
    bool bad;
    __device__ void reset() {
        for (int j = 0; j < kMaxDim; ++j) { mn[j] = __int_as_float(0x7f800000); mx[j] = __int_as_float(0xff800000); }
        bad = false;
    }
    __device__ void add(float x, int j) {
        bad |= (__float_as_uint(x) & 0x7f800000u) == 0x7f800000u;
        mn[j] = fminf(mn[j], x);
        mx[j] = fmaxf(mx[j], x);
    }
    __device__ long long lo(int j) const { return okey((double)mn[j]); }
    __device__ long long hi(int j) const { return okey((double)mx[j]); }
};
template <> struct BbAcc<double> {
    long long mn[kMaxDim], mx[kMaxDim];
    bool bad;
    __device__ void reset() {
        for (int j = 0; j < kMaxDim; ++j) { mn[j] = 0x7fffffffffffffffll; mx[j] = (long long)0x8000000000000000ull; }
        bad = false;
    }
    __device__ void add(double x, int j) {
        const long long b = __double_as_longlong(x);
        bad |= ((b >> 52) & 0x7ff) == 0x7ff;
        const long long k = b >= 0 ? b : (b ^ 0x7fffffffffffffffll);
        mn[j] = k < mn[j] ? k : mn[j];
        mx[j] = k > mx[j] ? k : mx[j];
    }
    __device__ long long lo(int j) const { return mn[j]; }
    __device__ long long hi(int j) const { return mx[j]; }
};

template <typename T>
__device__ __forceinline__ void bb_flush(long long *bb, int inst, int d, const BbAcc<T> &a) {
    long long *b = bb + (long long)inst * BB_SLOTS;
    for (int j = 0; j < d; ++j) {
        atomicMin(b + j, a.lo(j));
        atomicMax(b + kMaxDim + j, a.hi(j));
    }
    if (a.bad) atomicOr((unsigned long long *)(b + 2 * kMaxDim), 1ull);
}

// Per-instance bounding boxes: a warp takes BB_CHUNK consecutive rows, keeps
// per-lane extremes while its rows stay in one instance, and merges them into
// that instance's slots with atomics.
template <typename T>
__global__ void __launch_bounds__(256)
k_batch_bbox(const T *__restrict__ X, int ld, long long n_total, const dbscan_instance *__restrict__ desc, int count,
             long long *__restrict__ bb) {
    const int lane = threadIdx.x & 31;
    for (long long r0 = (long long)warp_id_global() * BB_CHUNK; r0 < n_total;
         r0 += (long long)warps_global() * BB_CHUNK) {
        const long long r1 = r0 + BB_CHUNK < n_total ? r0 + BB_CHUNK : n_total;
        int cur = -1, d = 0;
        long long lo = 0, hi = 0;
        BbAcc<T> acc;
        acc.reset();
        for (long long r = r0 + lane; r < r1; r += 32) {
            if (cur < 0 || r < lo || r >= hi) {
                if (cur >= 0) bb_flush(bb, cur, d, acc);
                cur = find_inst(desc, count, r);
                lo = desc[cur].row0;
                hi = lo + desc[cur].n;
                d = desc[cur].d;
                acc.reset();
            }
            for (int j = 0; j < d; ++j) acc.add(X[r * ld + j], j);
        }
        if (cur >= 0) bb_flush(bb, cur, d, acc);
    }
}

// One thread per instance: its grid and thresholds from its box.
__global__ void k_batch_inst(const dbscan_instance *__restrict__ desc, int count, const long long *__restrict__ bb,
                             int want_fp32, int f64, int key_limit, double rho, int ld, Inst *__restrict__ inst,
                             DevCounters *ctr) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const dbscan_instance D = desc[i];
    Inst I;
    double lo[kMaxDim], hi[kMaxDim];
    const long long *b = bb + (long long)i * BB_SLOTS;
    for (int j = 0; j < kMaxDim; ++j) {
        lo[j] = D.n > 0 ? okey_to_double(b[j]) : 0.0;
        hi[j] = D.n > 0 ? okey_to_double(b[kMaxDim + j]) : 0.0;
    }
    if (D.n > 0 && b[2 * kMaxDim] != 0) set_error(ctr, DBSCAN_ERR_INVALID_ARG, i);
    int fp32 = 0;
    const int st =
        build_inst(I, D.eps, D.min_pts, (int)D.n, D.d, lo, hi, f64 != 0, want_fp32 != 0, key_limit, &fp32, rho);
    if (st != DBSCAN_OK) set_error(ctr, st, i);
    // the key interleaves all ld stored coordinates (the unused ones are zero),
    // so an instance of lower dimension still needs ld * bits key bits
    else if (ld * I.bits > key_limit) set_error(ctr, DBSCAN_ERR_KEY_OVERFLOW, i);
    else if (want_fp32 && !fp32) set_error(ctr, DBSCAN_ERR_INVALID_ARG, i);
    I.row0 = (int)D.row0;
    inst[i] = I;
}

cudaError_t ensure_batch(dbscan_ctx *c, int count) {
    if (c->batch_cap >= count) return cudaSuccess;
    cudaFree(c->d_bdesc);
    cudaFree(c->d_binst);
    cudaFree(c->d_bbox);
    cudaFreeHost(c->h_bdesc);
    c->d_bdesc = nullptr;
    c->d_binst = nullptr;
    c->d_bbox = nullptr;
    c->h_bdesc = nullptr;
    c->batch_cap = 0;
    cudaError_t e = ctx_malloc(c, (void **)&c->d_bdesc, sizeof(dbscan_instance) * count);
    if (e == cudaSuccess) e = ctx_malloc(c, (void **)&c->d_binst, sizeof(Inst) * count);
    if (e == cudaSuccess) e = ctx_malloc(c, (void **)&c->d_bbox, sizeof(long long) * BB_SLOTS * count);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&c->h_bdesc, sizeof(dbscan_instance) * count);
    if (e == cudaSuccess) c->batch_cap = count;
    return e;
}

}  // namespace

// Run-wide pieces shared with capi.cu.
dbscan_status gbdb_enqueue_batch_prologue(dbscan_ctx *c, const void *d_points, int ld, int dtype, int count,
                                          long long n_total, int want_fp32, int key_limit, double rho,
                                          cudaStream_t s) {
    if (cudaMemsetAsync(c->ctr, 0, sizeof(DevCounters), s) != cudaSuccess) return DBSCAN_ERR_CUDA;
    if (cudaMemcpyAsync(c->d_bdesc, c->h_bdesc, sizeof(dbscan_instance) * count, cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
        return DBSCAN_ERR_CUDA;
    k_bb_init<<<(count * BB_SLOTS + 255) / 256, 256, 0, s>>>(c->d_bbox, count);
    count_launch();
    if (dtype == DBSCAN_F32) {
        const int g = grid_for((const void *)k_batch_bbox<float>, 256);
        k_batch_bbox<float><<<g, 256, 0, s>>>((const float *)d_points, ld, n_total, c->d_bdesc, count, c->d_bbox);
    } else {
        const int g = grid_for((const void *)k_batch_bbox<double>, 256);
        k_batch_bbox<double><<<g, 256, 0, s>>>((const double *)d_points, ld, n_total, c->d_bdesc, count, c->d_bbox);
    }
    count_launch();
    k_batch_inst<<<(count + 127) / 128, 128, 0, s>>>(c->d_bdesc, count, c->d_bbox, want_fp32,
                                                     dtype == DBSCAN_F64 ? 1 : 0, key_limit, rho, ld, c->d_binst,
                                                     c->ctr);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? DBSCAN_OK : DBSCAN_ERR_CUDA;
}

dbscan_status gbdb_batch_buffers(dbscan_ctx *c, const dbscan_instance *h, int count) {
    if (ensure_batch(c, count) != cudaSuccess) {
        (void)cudaGetLastError();
        return DBSCAN_ERR_OOM;
    }
    std::memcpy(c->h_bdesc, h, sizeof(dbscan_instance) * count);
    return DBSCAN_OK;
}

void gbdb_batch_free(dbscan_ctx *c) {
    cudaFree(c->d_bdesc);
    cudaFree(c->d_binst);
    cudaFree(c->d_bbox);
    cudaFreeHost(c->h_bdesc);
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    c->graph_exec = nullptr;
}
