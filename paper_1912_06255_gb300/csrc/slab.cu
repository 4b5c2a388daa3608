// dbscan_run_slabs: one instance too large for a context's workspace (the
// paper's billion-point runs, Sec. 7, keep the whole input in one shared
// memory) clustered as a sequence of slabs along its widest dimension, each
// run with a halo through the ordinary single-instance path, and merged into
// the one exact result.
//
// Why the merge is exact.  Slab s owns the points whose coordinate x on the
// partition axis lies in [c_s, c_{s+1}) and its run sees every point with x in
// [L_s, U_s], where L_s <= c_s - 2 eps' and U_s >= c_{s+1} + 2 eps', eps' being
// the largest |x_p - x_q| of a pair the FP64 predicate accepts (below).
//  (1) Core flags.  An owned point sees its whole eps-neighbourhood, so its
//      flag is exact; so is the flag of every point within eps of an owned
//      point, whose neighbourhood lies within 2 eps' of the owned range.
//      Farther points may miss part of their neighbourhood: their counts can
//      only be too small, so every point a slab run calls core is core.
//  (2) Edges.  A slab run only joins points it calls core that pass the
//      connectivity test, so by (1) every component of a run is a connected
//      set of the core graph (Sec. 2).  Conversely an edge p-q between core
//      points, p owned by slab s, has q within eps of p: both flags are exact
//      in slab s, and its run puts p and q in one component.  The union of all
//      runs' components is therefore exactly the components of the core graph.
//  (3) Border sets.  A non-core point owned by slab s has all its core
//      neighbours within eps, with exact flags in slab s; its set is the set
//      of their merged components.
// The merge is a union-find over the global point indices that hooks the
// larger root under the smaller, so each root is the smallest core index of
// its cluster, which is the cluster's name (Sec. 2 convention of this
// library).  Each point a run calls core is united with its local cluster's
// first core point; the owned non-core points' local cluster names are mapped
// to merged names, sorted, deduplicated and written as CSR.
//
// Rounding margin.  The predicate accumulates fl((p_i - q_i)^2) left to right
// and compares with fl(eps^2); rounded sums of non-negative terms never fall
// below a term, so an accepted pair has fl(fl(p_k - q_k)^2) <= fl(eps^2) on
// the axis k.  With u = 2^-53 and gradual underflow this gives |p_k - q_k| <=
// eps (1 + 4u) + 2^-537 = eps'.  The halo width H = 2 (eps (1 + 2^-40) +
// 2^-500) exceeds 2 eps', and L_s, U_s are c_s - H, c_{s+1} + H rounded two
// ulps outward.
//
// Input and outputs may live in host memory (pinned: the kernels read it in
// place over the host link; pageable: staged through a device buffer chunk by
// chunk) or in device memory; the kernels index points with 64-bit integers.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "ctx.cuh"
#include "geom.cuh"

using namespace gbdb;

namespace gbdb {

struct SlabState {
    // global, one entry per input point
    int64_t n_cap = 0;
    int *parent = nullptr;     // union-find over core points (identity elsewhere)
    int *label = nullptr;      // merged names
    uint8_t *core = nullptr;   // owner's core flags
    long long *off = nullptr;  // [n+1] border counts, then CSR offsets
    long long *part = nullptr; // scan partials for n+1 entries
    // one slab with its halo (the context's max_points)
    int64_t s_cap = 0;
    int s_elt = 0;             // bytes per point row of the slab buffer
    void *s_pts = nullptr;
    int *s_gid = nullptr;      // global index; ~index for halo points
    uint8_t *s_core = nullptr;
    int *s_lab = nullptr;
    long long *s_off = nullptr;
    int *s_ids = nullptr;
    int64_t s_ids_cap = 0;
    // (point, cluster) pairs of owned border points
    uint64_t *pk0 = nullptr, *pk1 = nullptr;
    int64_t p_cap = 0;
    void *sort_scratch = nullptr;
    size_t sort_bytes = 0;
    long long *p_part = nullptr;
    int64_t p_part_cap = 0;
    // pageable input: one chunk at a time
    void *stage = nullptr;
    size_t stage_bytes = 0;
    // host input copied to the device once (DBSCAN_OPT_SLAB_STAGE)
    void *dev_in = nullptr;
    size_t dev_in_bytes = 0;
    // small device state
    unsigned long long *hist = nullptr;  // [kSlabBins]
    long long *bounds = nullptr;         // [2 * kMaxDim + 1] ordered keys + non-finite flag
    long long *cnt = nullptr;            // [4] selected points, pending pairs
    DevCounters *ctr = nullptr;
    long long *h_small = nullptr;        // pinned mirror of bounds / cnt
    DevCounters *h_ctr = nullptr;
    // the last call's border ids (in the free half of the pending buffers)
    const int *ids = nullptr;
    int64_t ids_total = 0;
    bool have = false;
};

}  // namespace gbdb

namespace {

constexpr int SL_THREADS = 256;
constexpr int kSlabBins = 8192;             // histogram bins along the partition axis (32 KiB of shared counts)
constexpr size_t kStageBytes = 256u << 20;  // pageable input: bytes staged per chunk
constexpr int kMaxSlabs = 4096;

__device__ __forceinline__ long long okey(double x) {
    const long long b = __double_as_longlong(x);
    return b >= 0 ? b : (b ^ 0x7fffffffffffffffll);
}
double okey_host_to_double(long long k) {
    const long long b = k >= 0 ? k : (k ^ 0x7fffffffffffffffll);
    double x;
    std::memcpy(&x, &b, 8);
    return x;
}

int grid_of(int64_t n, int per_block) {
    const int64_t b = (n + per_block - 1) / per_block;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 16));
}

// ------------------------------------------------------------ input passes
__global__ void k_sl_bounds_init(long long *b) {
    const int j = threadIdx.x;
    if (j < 2 * kMaxDim) b[j] = j < kMaxDim ? 0x7fffffffffffffffll : (long long)0x8000000000000000ull;
    if (j == 0) b[2 * kMaxDim] = 0;
}

// Per-dimension extremes of n points, merged into b as ordered FP64 keys.
// Extremes are kept in the input's type (FP32 min/max is exact and stays off
// the FP64 pipe) and widened once per warp.
template <typename T>
__global__ void __launch_bounds__(SL_THREADS) k_sl_bounds(const T *__restrict__ X, long long n, int d, long long *b) {
    T mn[kMaxDim], mx[kMaxDim];
#pragma unroll
    for (int j = 0; j < kMaxDim; ++j) { mn[j] = (T)INFINITY; mx[j] = (T)-INFINITY; }
    bool bad = false;
    const long long step = (long long)gridDim.x * SL_THREADS;
    for (long long i0 = (long long)blockIdx.x * SL_THREADS + threadIdx.x; i0 < n; i0 += 2 * step) {
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const long long i = i0 + u * step;
            if (i >= n) break;
#pragma unroll
            for (int j = 0; j < kMaxDim; ++j) {
                if (j < d) {
                    const T x = X[i * d + j];
                    bad |= !isfinite(x);
                    mn[j] = x < mn[j] ? x : mn[j];
                    mx[j] = x > mx[j] ? x : mx[j];
                }
            }
        }
    }
#pragma unroll
    for (int j = 0; j < kMaxDim; ++j) {
        if (j < d) {
            long long kn = okey((double)mn[j]), kx = okey((double)mx[j]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                kn = min(kn, __shfl_xor_sync(0xffffffffu, kn, o));
                kx = max(kx, __shfl_xor_sync(0xffffffffu, kx, o));
            }
            if ((threadIdx.x & 31) == 0) {
                atomicMin(b + j, kn);
                atomicMax(b + kMaxDim + j, kx);
            }
        }
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr((unsigned long long *)(b + 2 * kMaxDim), 1ull);
}

// Histogram of the axis coordinate: bin = floor((x - lo) * scale), clamped.
// Counts go to shared memory first; each block flushes its non-zero bins once.
// Four points per thread per step keep enough loads in flight with the few
// blocks the shared histogram allows.
// The bins only steer the cuts and bound the slab sizes (with a margin of two
// bins), so they are computed in the input's type: for FP32 input, lo is an
// input value and the binning error stays far below one bin.
template <typename T>
__global__ void __launch_bounds__(SL_THREADS) k_sl_hist(const T *__restrict__ X, long long n, int d, int axis,
                                                        T lo, T scale, unsigned long long *hist) {
    __shared__ unsigned sh[kSlabBins];
    for (int j = threadIdx.x; j < kSlabBins; j += SL_THREADS) sh[j] = 0;
    __syncthreads();
    const long long step = (long long)gridDim.x * SL_THREADS;
    for (long long i0 = (long long)blockIdx.x * SL_THREADS + threadIdx.x; i0 < n; i0 += 4 * step) {
        T x[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const long long i = i0 + u * step;
            x[u] = i < n ? X[i * d + axis] : lo;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (i0 + u * step < n) {
                const T t = (x[u] - lo) * scale;
                const int b = t <= (T)0 ? 0 : (t >= (T)(kSlabBins - 1) ? kSlabBins - 1 : (int)t);
                atomicAdd(sh + b, 1u);
            }
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < kSlabBins; j += SL_THREADS)
        if (sh[j]) atomicAdd(hist + j, (unsigned long long)sh[j]);
}

// Appends the points with L <= x <= U (x on the axis) to the slab buffer,
// comparing in the input's own type: the host rounds each FP64 bound
// outward or inward to an FP32 value that gives the same answer for every
// FP32 x (x >= t iff x >= t rounded up; x <= t iff x <= t rounded down;
// x < t iff x < t rounded up), so FP32 input needs no FP64 instruction here;
// with their global index (~index unless c_lo <= x < c_hi).  A block takes
// tiles of SEL_ITEMS x 256 points (item k of thread t is point k*256 + t of
// the tile, so the reads coalesce), ranks its selected points with a block
// scan and claims their slots with one atomic per tile.  The count keeps
// growing past cap so the host sees an overflow, but nothing is written there.
constexpr int SEL_ITEMS = 8;

template <typename T>
__global__ void __launch_bounds__(SL_THREADS)
k_sl_select(const T *__restrict__ X, long long n, int d, int axis, long long g0, T L, T U, T c_lo, T c_hi,
            T *__restrict__ out, int *__restrict__ gid, long long cap, long long *cnt) {
    constexpr int W = SL_THREADS / 32;
    __shared__ int s_warp[W];
    __shared__ long long s_base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long tile = (long long)SL_THREADS * SEL_ITEMS;
    for (long long t0 = (long long)blockIdx.x * tile; t0 < n; t0 += (long long)gridDim.x * tile) {
        unsigned selm = 0, ownm = 0;
#pragma unroll
        for (int k = 0; k < SEL_ITEMS; ++k) {
            const long long i = t0 + (long long)k * SL_THREADS + threadIdx.x;
            if (i < n) {
                const T x = X[i * d + axis];
                if (x >= L && x <= U) selm |= 1u << k;
                if (x >= c_lo && x < c_hi) ownm |= 1u << k;
            }
        }
        const int c = __popc(selm);
        int inc = c;  // inclusive scan over the warp
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += v;
        }
        if (lane == 31) s_warp[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            const int w = lane < W ? s_warp[lane] : 0;
            int winc = w;
#pragma unroll
            for (int o = 1; o < W; o <<= 1) {
                const int v = __shfl_up_sync(0xffffffffu, winc, o);
                if (lane >= o) winc += v;
            }
            const int total = __shfl_sync(0xffffffffu, winc, W - 1);
            if (lane < W) s_warp[lane] = winc - w;
            if (lane == 0) s_base = total ? (long long)atomicAdd((unsigned long long *)cnt, (unsigned long long)total) : 0;
        }
        __syncthreads();
        long long pos = s_base + s_warp[warp] + (inc - c);
#pragma unroll
        for (int k = 0; k < SEL_ITEMS; ++k) {
            if (selm & (1u << k)) {
                const long long i = t0 + (long long)k * SL_THREADS + threadIdx.x;
                if (pos < cap) {
                    for (int j = 0; j < d; ++j) out[pos * d + j] = X[i * d + j];
                    const int g = (int)(g0 + i);
                    gid[pos] = (ownm & (1u << k)) ? g : ~g;
                }
                ++pos;
            }
        }
        __syncthreads();  // s_warp and s_base are rewritten by the next tile
    }
}

// ------------------------------------------------------------ merge
__global__ void k_sl_init(int64_t n, int *parent, int *label, uint8_t *core, long long *off) {
    for (int64_t i = (int64_t)blockIdx.x * SL_THREADS + threadIdx.x; i <= n; i += (int64_t)gridDim.x * SL_THREADS) {
        if (i < n) {
            parent[i] = (int)i;
            label[i] = -1;
            core[i] = 0;
        }
        off[i] = 0;
    }
}

__device__ __forceinline__ int gid_of(int v) { return v >= 0 ? v : ~v; }

// One slab's run into the global state: unions of the points it calls core
// with their local cluster's first core point, the owned points' core flags,
// and the owned border points' (point, cluster) pairs.
__global__ void __launch_bounds__(SL_THREADS)
k_sl_merge(int ns, const int *__restrict__ gid, const uint8_t *__restrict__ s_core, const int *__restrict__ s_lab,
           const long long *__restrict__ s_off, const int *__restrict__ s_ids, int *parent, uint8_t *core,
           uint64_t *pend, long long p_cap, long long *p_cnt, int nb, int max_iters, DevCounters *ctr) {
    for (int i = blockIdx.x * SL_THREADS + threadIdx.x; i < ns; i += gridDim.x * SL_THREADS) {
        const int v = gid[i];
        const int g = gid_of(v);
        const bool c = s_core[i] != 0;
        if (c) {
            const int r = s_lab[i];
            if (r >= 0 && r < ns) {
                const int gr = gid_of(gid[r]);
                if (gr != g) uf_link(parent, g, gr, max_iters, ctr);
            } else {
                set_error(ctr, DBSCAN_ERR_CUDA, 40);
            }
        }
        if (v >= 0) {
            core[g] = c ? 1 : 0;
            if (!c) {
                const long long a = s_off[i], b = s_off[i + 1];
                if (b > a) {
                    const long long at = (long long)atomicAdd((unsigned long long *)p_cnt, (unsigned long long)(b - a));
                    for (long long j = a; j < b; ++j) {
                        const int name = s_ids[j];
                        if (at + (j - a) < p_cap && name >= 0 && name < ns)
                            pend[at + (j - a)] = ((uint64_t)g << nb) | (uint64_t)gid_of(gid[name]);
                    }
                }
            }
        }
    }
}

// Compressing finds from every core point, then (separate launch, no stores
// to parent) each core point's root as its name.
__global__ void k_sl_compress(int64_t n, int *parent, const uint8_t *core, int max_iters, DevCounters *ctr) {
    for (int64_t i = (int64_t)blockIdx.x * SL_THREADS + threadIdx.x; i < n; i += (int64_t)gridDim.x * SL_THREADS)
        if (core[i]) uf_find(parent, (int)i, max_iters, ctr);
}
__global__ void k_sl_label(int64_t n, const int *parent, const uint8_t *core, int *label, int max_iters,
                           DevCounters *ctr) {
    for (int64_t i = (int64_t)blockIdx.x * SL_THREADS + threadIdx.x; i < n; i += (int64_t)gridDim.x * SL_THREADS) {
        if (!core[i]) continue;
        int x = (int)i, it = 0;
        for (; it < max_iters; ++it) {
            const int p = parent[x];
            if (p == x) break;
            x = p;
        }
        if (it == max_iters) set_error(ctr, DBSCAN_ERR_DEVICE_TIMEOUT, 41);
        label[i] = x;
    }
}

// Pending (point, first core point) pairs -> (point, merged name).
__global__ void k_sl_pend_map(long long P, uint64_t *pend, int nb, const int *label, DevCounters *ctr) {
    const uint64_t mask = (1ull << nb) - 1;
    for (long long i = (long long)blockIdx.x * SL_THREADS + threadIdx.x; i < P; i += (long long)gridDim.x * SL_THREADS) {
        const uint64_t e = pend[i];
        const int gn = (int)(e & mask);
        int name = label[gn];
        if (name < 0) {  // a point a slab called core is core for its owner too
            set_error(ctr, DBSCAN_ERR_CUDA, 42);
            name = gn;
        }
        pend[i] = (e & ~mask) | (uint64_t)name;
    }
}

// Sorted pairs: first occurrences are the set entries; the first entry of a
// point is its smallest cluster, which is its label.
__global__ void k_sl_unique(long long P, const uint64_t *__restrict__ key, int nb, int *flag, long long *cnt,
                            int *label) {
    const uint64_t mask = (1ull << nb) - 1;
    for (long long i = (long long)blockIdx.x * SL_THREADS + threadIdx.x; i < P; i += (long long)gridDim.x * SL_THREADS) {
        const uint64_t e = key[i];
        const bool first = i == 0 || key[i - 1] != e;
        flag[i] = first ? 1 : 0;
        if (first) {
            const long long g = (long long)(e >> nb);
            atomicAdd((unsigned long long *)(cnt + g), 1ull);
            if (i == 0 || (key[i - 1] >> nb) != (e >> nb)) label[g] = (int)(e & mask);
        }
    }
}
__global__ void k_sl_fill(long long P, const uint64_t *__restrict__ key, int nb, const int *pos, int *ids) {
    const uint64_t mask = (1ull << nb) - 1;
    for (long long i = (long long)blockIdx.x * SL_THREADS + threadIdx.x; i < P; i += (long long)gridDim.x * SL_THREADS)
        if (i == 0 || key[i - 1] != key[i]) ids[pos[i]] = (int)(key[i] & mask);
}

// ------------------------------------------------------------ host side
dbscan_status cuda_st(cudaError_t e) {
    if (e == cudaSuccess) return DBSCAN_OK;
    (void)cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? DBSCAN_ERR_OOM : DBSCAN_ERR_CUDA;
}

#define SCK(x)                                               \
    do {                                                     \
        dbscan_status st_ = cuda_st(x);                      \
        if (st_ != DBSCAN_OK) return st_;                    \
    } while (0)

template <typename P> cudaError_t grow(const dbscan_ctx *c, P **p, int64_t &cap, int64_t want, size_t elt) {
    if (*p && cap >= want) return cudaSuccess;
    cudaFree(*p);
    *p = nullptr;
    cap = 0;
    cudaError_t e = ctx_malloc(c, (void **)p, (size_t)std::max<int64_t>(want, 1) * elt);
    if (e == cudaSuccess) cap = want;
    return e;
}

cudaError_t ensure_small(dbscan_ctx *c, SlabState &S) {
    if (S.hist) return cudaSuccess;
    cudaError_t e = ctx_malloc(c, (void **)&S.hist, sizeof(unsigned long long) * kSlabBins);
    if (e == cudaSuccess) e = ctx_malloc(c, (void **)&S.bounds, sizeof(long long) * (2 * kMaxDim + 1));
    if (e == cudaSuccess) e = ctx_malloc(c, (void **)&S.cnt, sizeof(long long) * 4);
    if (e == cudaSuccess) e = ctx_malloc(c, (void **)&S.ctr, sizeof(DevCounters));
    if (e == cudaSuccess && !c->fault_alloc) e = cudaMallocHost((void **)&S.h_small, sizeof(long long) * (2 * kMaxDim + 5));
    if (e == cudaSuccess && !c->fault_alloc) e = cudaMallocHost((void **)&S.h_ctr, sizeof(DevCounters));
    if (c->fault_alloc) e = cudaErrorMemoryAllocation;
    if (e != cudaSuccess) {
        cudaFree(S.hist); cudaFree(S.bounds); cudaFree(S.cnt); cudaFree(S.ctr);
        cudaFreeHost(S.h_small); cudaFreeHost(S.h_ctr);
        S.hist = nullptr; S.bounds = nullptr; S.cnt = nullptr; S.ctr = nullptr;
        S.h_small = nullptr; S.h_ctr = nullptr;
    }
    return e;
}

cudaError_t ensure_global(dbscan_ctx *c, SlabState &S, int64_t n) {
    if (S.parent && S.n_cap >= n) return cudaSuccess;
    cudaFree(S.parent); cudaFree(S.label); cudaFree(S.core); cudaFree(S.off); cudaFree(S.part);
    S.parent = nullptr; S.label = nullptr; S.core = nullptr; S.off = nullptr; S.part = nullptr;
    S.n_cap = 0;
    const int64_t N = std::max<int64_t>(n, 1);
    cudaError_t e = ctx_malloc(c, (void **)&S.parent, 4 * (size_t)N);
    if (e == cudaSuccess) e = ctx_malloc(c, (void **)&S.label, 4 * (size_t)N);
    if (e == cudaSuccess) e = ctx_malloc(c, (void **)&S.core, (size_t)N);
    if (e == cudaSuccess) e = ctx_malloc(c, (void **)&S.off, 8 * (size_t)(N + 1));
    if (e == cudaSuccess) e = ctx_malloc(c, (void **)&S.part, 8 * (size_t)(scan_partials(N + 1) + 2));
    if (e == cudaSuccess) S.n_cap = N;
    return e;
}

cudaError_t ensure_slab(dbscan_ctx *c, SlabState &S, int elt_row) {
    const int64_t cap = std::max<int64_t>(c->max_points, 1);
    if (S.s_pts && S.s_cap >= cap && S.s_elt >= elt_row) return cudaSuccess;
    cudaFree(S.s_pts); cudaFree(S.s_gid); cudaFree(S.s_core); cudaFree(S.s_lab); cudaFree(S.s_off);
    S.s_pts = nullptr; S.s_gid = nullptr; S.s_core = nullptr; S.s_lab = nullptr; S.s_off = nullptr;
    S.s_cap = 0;
    const int row = std::max(elt_row, S.s_elt);
    cudaError_t e = ctx_malloc(c, &S.s_pts, (size_t)cap * row);
    if (e == cudaSuccess) e = ctx_malloc(c, (void **)&S.s_gid, 4 * (size_t)cap);
    if (e == cudaSuccess) e = ctx_malloc(c, (void **)&S.s_core, (size_t)cap);
    if (e == cudaSuccess) e = ctx_malloc(c, (void **)&S.s_lab, 4 * (size_t)cap);
    if (e == cudaSuccess) e = ctx_malloc(c, (void **)&S.s_off, 8 * (size_t)(cap + 1));
    if (e == cudaSuccess) { S.s_cap = cap; S.s_elt = row; }
    return e;
}

// Pending pair buffers (two, for the sort) holding at least want entries;
// keeps the first `keep` entries of pk0.
cudaError_t ensure_pend(dbscan_ctx *c, SlabState &S, int64_t want, int64_t keep, cudaStream_t s) {
    if (S.pk0 && S.p_cap >= want) return cudaSuccess;
    const int64_t cap = std::max<int64_t>(want, std::max<int64_t>(2 * S.p_cap, 1 << 20));
    uint64_t *a = nullptr, *b = nullptr;
    cudaError_t e = ctx_malloc(c, (void **)&a, 8 * (size_t)cap);
    if (e == cudaSuccess) e = ctx_malloc(c, (void **)&b, 8 * (size_t)cap);
    if (e == cudaSuccess && keep > 0) e = cudaMemcpyAsync(a, S.pk0, 8 * (size_t)keep, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaFree(a);
        cudaFree(b);
        return e;
    }
    cudaFree(S.pk0);
    cudaFree(S.pk1);
    S.pk0 = a;
    S.pk1 = b;
    S.p_cap = cap;
    return cudaSuccess;
}

// Where the kernels read chunk [i0, i0 + cnt): in place (device memory or
// pinned host memory mapped into the device's address space) or from the
// staging buffer after a copy.
struct Source {
    const char *direct = nullptr;  // device-readable base, or null (pageable: staged)
    const char *host = nullptr;
    size_t row = 0;
};

const void *chunk_ptr(const Source &src, SlabState &S, int64_t i0, int64_t cnt, cudaStream_t s, cudaError_t &e) {
    if (src.direct) return src.direct + (size_t)i0 * src.row;
    e = cudaMemcpyAsync(S.stage, src.host + (size_t)i0 * src.row, (size_t)cnt * src.row, cudaMemcpyHostToDevice, s);
    return S.stage;
}

template <typename T>
void launch_bounds_pass(const T *X, long long n, int d, long long *b, cudaStream_t s) {
    k_sl_bounds<T><<<grid_of(n, SL_THREADS * 8), SL_THREADS, 0, s>>>(X, n, d, b); count_launch();
}
template <typename T>
void launch_hist(const T *X, long long n, int d, int axis, double lo, double scale, unsigned long long *h,
                 cudaStream_t s) {
    const int g = (int)std::max<long long>(1, std::min<long long>((n + 65535) / 65536, 152 * 4));
    k_sl_hist<T><<<g, SL_THREADS, 0, s>>>(X, n, d, axis, (T)lo, (T)scale, h); count_launch();
}
// FP32 bounds equivalent to FP64 ones for every FP32 x (see k_sl_select).
float f32_up(double t) {
    float f = (float)t;
    if ((double)f < t) f = std::nextafter(f, INFINITY);
    return f;
}
float f32_down(double t) {
    float f = (float)t;
    if ((double)f > t) f = std::nextafter(f, -INFINITY);
    return f;
}

template <typename T>
void launch_select(const T *X, long long n, int d, int axis, long long g0, double L, double U, double clo,
                   double chi, void *out, int *gid, long long cap, long long *cnt, cudaStream_t s) {
    T l, u, a, b;
    if constexpr (sizeof(T) == 4) {
        l = f32_up(L);
        u = f32_down(U);
        a = f32_up(clo);
        b = f32_up(chi);
    } else {
        l = L;
        u = U;
        a = clo;
        b = chi;
    }
    k_sl_select<T><<<grid_of(n, SL_THREADS * SEL_ITEMS), SL_THREADS, 0, s>>>(X, n, d, axis, g0, l, u, a, b,
                                                                          (T *)out, gid, cap, cnt);
    count_launch();
}

struct Cuts {
    std::vector<double> c;  // c[0] = -inf, c[S] = +inf
    int64_t max_est = 0;    // largest slab-with-halo count bound from the histogram
};

// Cuts at bin edges balancing the owned counts over S slabs (consecutive equal
// cuts dropped), with an upper bound of each slab's count with its halo: the
// points of every bin that meets [L_s - w, U_s + w], w one bin width (the
// binning rounds).  pre[b] = points in bins [0, b).
Cuts choose_cuts(const std::vector<int64_t> &pre, int64_t n, int S, double lo, double hi, double H) {
    Cuts C;
    C.c.push_back(-INFINITY);
    const double w = (hi - lo) / kSlabBins;
    if (hi > lo) {
        int b = 0, last = -1;
        for (int j = 1; j < S; ++j) {
            const long double target = (long double)n * j / S;
            while (b < kSlabBins && (long double)pre[b] < target) ++b;
            if (b <= 0 || b >= kSlabBins || b == last) continue;
            last = b;
            C.c.push_back(lo + (hi - lo) * ((double)b / kSlabBins));
        }
    }
    C.c.push_back(INFINITY);
    const int Se = (int)C.c.size() - 1;
    for (int s = 0; s < Se; ++s) {
        // first and last bin meeting the widened range
        int b0 = 0, b1 = kSlabBins - 1;
        if (s > 0 && w > 0) {
            const double t = std::floor((C.c[s] - H - 2 * w - lo) / w);
            b0 = t <= 0 ? 0 : (t >= kSlabBins - 1 ? kSlabBins - 1 : (int)t);
        }
        if (s < Se - 1 && w > 0) {
            const double t = std::ceil((C.c[s + 1] + H + 2 * w - lo) / w);
            b1 = t <= 0 ? 0 : (t >= kSlabBins - 1 ? kSlabBins - 1 : (int)t);
        }
        C.max_est = std::max<int64_t>(C.max_est, b1 >= b0 ? pre[b1 + 1] - pre[b0] : 0);
    }
    return C;
}

double down2(double x) { return std::nextafter(std::nextafter(x, -INFINITY), -INFINITY); }
double up2(double x) { return std::nextafter(std::nextafter(x, INFINITY), INFINITY); }

struct Timer {
    cudaStream_t s;
    std::chrono::steady_clock::time_point t0;
    explicit Timer(cudaStream_t st) : s(st) { t0 = std::chrono::steady_clock::now(); }
    double lap() {  // ms since the last lap, after the stream drained
        cudaStreamSynchronize(s);
        const auto t = std::chrono::steady_clock::now();
        const double ms = std::chrono::duration<double, std::milli>(t - t0).count();
        t0 = t;
        return ms;
    }
};

template <typename T>
dbscan_status run_slabs(dbscan_ctx *c, SlabState &S, const Source &src, int64_t n, int d, int dtype, double eps,
                        int64_t min_pts, int num_slabs, uint8_t *core, int32_t *labels, int64_t *border_offsets,
                        int64_t *num_border_memberships, dbscan_slab_stats *st, cudaStream_t s) {
    // one launch per pass over device-readable input; staged chunks otherwise
    const int64_t chunk = src.direct ? n : std::max<int64_t>(1, (int64_t)(kStageBytes / src.row));
    Timer tm(s);
    // -------- pass 1: extremes per dimension
    k_sl_bounds_init<<<1, 32, 0, s>>>(S.bounds); count_launch();
    for (int64_t i0 = 0; i0 < n; i0 += chunk) {
        const int64_t cn = std::min(chunk, n - i0);
        cudaError_t e = cudaSuccess;
        const T *X = (const T *)chunk_ptr(src, S, i0, cn, s, e);
        SCK(e);
        launch_bounds_pass<T>(X, cn, d, S.bounds, s);
    }
    SCK(cudaMemcpyAsync(S.h_small, S.bounds, sizeof(long long) * (2 * kMaxDim + 1), cudaMemcpyDeviceToHost, s));
    SCK(cudaStreamSynchronize(s));
    if (S.h_small[2 * kMaxDim]) return DBSCAN_ERR_INVALID_ARG;  // a coordinate is not finite
    int axis = 0;
    double lo = 0, hi = 0, widest = -1;
    for (int j = 0; j < d; ++j) {
        const double a = okey_host_to_double(S.h_small[j]), b = okey_host_to_double(S.h_small[kMaxDim + j]);
        if (b - a > widest) { widest = b - a; axis = j; lo = a; hi = b; }
    }
    // -------- pass 2: histogram of the axis coordinate
    SCK(cudaMemsetAsync(S.hist, 0, sizeof(unsigned long long) * kSlabBins, s));
    const double scale = hi > lo ? kSlabBins / (hi - lo) : 0.0;
    for (int64_t i0 = 0; i0 < n; i0 += chunk) {
        const int64_t cn = std::min(chunk, n - i0);
        cudaError_t e = cudaSuccess;
        const T *X = (const T *)chunk_ptr(src, S, i0, cn, s, e);
        SCK(e);
        launch_hist<T>(X, cn, d, axis, lo, scale, S.hist, s);
    }
    std::vector<unsigned long long> hist(kSlabBins);
    SCK(cudaMemcpyAsync(hist.data(), S.hist, sizeof(unsigned long long) * kSlabBins, cudaMemcpyDeviceToHost, s));
    SCK(cudaStreamSynchronize(s));
    std::vector<int64_t> pre(kSlabBins + 1, 0);
    for (int b = 0; b < kSlabBins; ++b) pre[b + 1] = pre[b] + (int64_t)hist[b];
    const double H = 2.0 * (eps * (1.0 + std::ldexp(1.0, -40)) + std::ldexp(1.0, -500));
    const int64_t cap = c->max_points;
    Cuts C;
    if (num_slabs > 0) {
        C = choose_cuts(pre, n, num_slabs, lo, hi, H);
    } else {
        int Sg = (int)std::max<int64_t>(1, (n + cap - 1) / std::max<int64_t>(cap, 1));
        for (;; ++Sg) {
            if (Sg > kMaxSlabs) return DBSCAN_ERR_CAPACITY;
            C = choose_cuts(pre, n, Sg, lo, hi, H);
            if (C.max_est <= cap) break;
        }
    }
    const int Se = (int)C.c.size() - 1;
    if (st) { st->slabs = Se; st->axis = axis; st->ms[0] = tm.lap(); }

    // -------- global state
    k_sl_init<<<grid_of(n + 1, SL_THREADS * 8), SL_THREADS, 0, s>>>(n, S.parent, S.label, S.core, S.off); count_launch();
    SCK(cudaMemsetAsync(S.ctr, 0, sizeof(DevCounters), s));
    SCK(cudaMemsetAsync(S.cnt, 0, sizeof(long long) * 4, s));
    int nb = 1;
    while (nb < 31 && (1ll << nb) < n) ++nb;
    long long pending = 0, halo = 0, biggest = 0;
    double ms_sel = 0, ms_run = 0, ms_merge = 0;
    for (int sl = 0; sl < Se; ++sl) {
        // -------- pass 3: the slab's points with their halo
        range_push(c, "dbscan_slabs:select");
        const double clo = C.c[sl], chi = C.c[sl + 1];
        const double L = sl == 0 ? -INFINITY : down2(clo - H);
        const double U = sl == Se - 1 ? INFINITY : up2(chi + H);
        SCK(cudaMemsetAsync(S.cnt, 0, sizeof(long long), s));
        for (int64_t i0 = 0; i0 < n; i0 += chunk) {
            const int64_t cn = std::min(chunk, n - i0);
            cudaError_t e = cudaSuccess;
            const T *X = (const T *)chunk_ptr(src, S, i0, cn, s, e);
            SCK(e);
            launch_select<T>(X, cn, d, axis, i0, L, U, clo, chi, S.s_pts, S.s_gid, cap, S.cnt, s);
        }
        SCK(cudaMemcpyAsync(S.h_small, S.cnt, sizeof(long long), cudaMemcpyDeviceToHost, s));
        SCK(cudaStreamSynchronize(s));
        const int64_t ns = S.h_small[0];
        if (ns > cap) return DBSCAN_ERR_CAPACITY;  // this slab with its halo does not fit the context
        biggest = std::max<long long>(biggest, ns);
        halo += ns;
        ms_sel += tm.lap();
        range_pop(c);
        // -------- the slab's run (Algorithm 1 on the slab)
        int64_t K = 0;
        dbscan_status r = dbscan_run(c, S.s_pts, ns, d, dtype, eps, min_pts, S.s_core, S.s_lab, (int64_t *)S.s_off, &K, s);
        if (r != DBSCAN_OK) return r;
        if (K > 0) {
            SCK(grow(c, &S.s_ids, S.s_ids_cap, K, sizeof(int)));
            r = dbscan_border_ids(c, S.s_ids, S.s_ids_cap, s);
            if (r != DBSCAN_OK) return r;
        }
        ms_run += tm.lap();
        // -------- merge into the global state
        range_push(c, "dbscan_slabs:merge");
        SCK(ensure_pend(c, S, pending + K, pending, s));
        S.h_small[3] = pending;
        SCK(cudaMemcpyAsync(S.cnt + 1, S.h_small + 3, sizeof(long long), cudaMemcpyHostToDevice, s));
        k_sl_merge<<<grid_of(ns, SL_THREADS * 4), SL_THREADS, 0, s>>>((int)ns, S.s_gid, S.s_core, S.s_lab, S.s_off,
                                                                     S.s_ids, S.parent, S.core, S.pk0, S.p_cap,
                                                                     S.cnt + 1, nb, c->max_iters, S.ctr);
        count_launch();
        SCK(cudaGetLastError());
        SCK(cudaMemcpyAsync(S.h_small + 1, S.cnt + 1, sizeof(long long), cudaMemcpyDeviceToHost, s));
        SCK(cudaMemcpyAsync(S.h_ctr, S.ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, s));
        SCK(cudaStreamSynchronize(s));
        if (S.h_ctr->err) return (dbscan_status)S.h_ctr->err;
        pending = S.h_small[1];
        ms_merge += tm.lap();
        range_pop(c);
    }
    // -------- names: roots of the core points, then the border sets
    const int gm = grid_of(n, SL_THREADS * 8);
    k_sl_compress<<<gm, SL_THREADS, 0, s>>>(n, S.parent, S.core, c->max_iters, S.ctr); count_launch();
    k_sl_label<<<gm, SL_THREADS, 0, s>>>(n, S.parent, S.core, S.label, c->max_iters, S.ctr); count_launch();
    int64_t total = 0;
    const int *ids_dev = nullptr;
    if (pending > 0) {
        if (pending >= 0x7fffffffll) return DBSCAN_ERR_CAPACITY;
        const int gp = grid_of(pending, SL_THREADS * 8);
        k_sl_pend_map<<<gp, SL_THREADS, 0, s>>>(pending, S.pk0, nb, S.label, S.ctr); count_launch();
        const size_t need = sort_scratch_bytes(pending);
        if (!S.sort_scratch || S.sort_bytes < need) {
            cudaFree(S.sort_scratch);
            S.sort_scratch = nullptr;
            S.sort_bytes = 0;
            SCK(ctx_malloc(c, &S.sort_scratch, need));
            S.sort_bytes = need;
        }
        SCK(grow(c, &S.p_part, S.p_part_cap, scan_partials(pending + 1) + 2, sizeof(long long)));
        const int which = radix_sort_u64(S.pk0, nullptr, S.pk1, nullptr, (int)pending, nullptr, pending, 0, 2 * nb,
                                         S.sort_scratch, S.sort_bytes, S.ctr, c->max_iters, s);
        uint64_t *sorted = which ? S.pk1 : S.pk0;
        int *flag = (int *)(which ? S.pk0 : S.pk1);
        int *ids = flag + pending;  // the second half of the free buffer
        k_sl_unique<<<gp, SL_THREADS, 0, s>>>(pending, sorted, nb, flag, S.off, S.label); count_launch();
        scan_i32_to_i32(flag, flag, pending, nullptr, pending, S.p_part, s);  // entry -> its place in the ids
        k_sl_fill<<<gp, SL_THREADS, 0, s>>>(pending, sorted, nb, flag, ids); count_launch();
        ids_dev = ids;
    }
    scan_i64_to_i64(S.off, S.off, n, nullptr, n, S.part, s);
    SCK(cudaGetLastError());
    SCK(cudaMemcpyAsync(S.h_ctr, S.ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, s));
    SCK(cudaMemcpyAsync(S.h_small + 2, S.off + n, sizeof(long long), cudaMemcpyDeviceToHost, s));
    SCK(cudaStreamSynchronize(s));
    if (S.h_ctr->err) return (dbscan_status)S.h_ctr->err;
    total = S.h_small[2];
    const double ms_names = tm.lap();
    if (num_border_memberships) *num_border_memberships = total;
    // -------- results out
    SCK(cudaMemcpyAsync(core, S.core, (size_t)n, cudaMemcpyDefault, s));
    SCK(cudaMemcpyAsync(labels, S.label, 4 * (size_t)n, cudaMemcpyDefault, s));
    if (border_offsets) SCK(cudaMemcpyAsync(border_offsets, S.off, 8 * (size_t)(n + 1), cudaMemcpyDefault, s));
    S.ids = ids_dev;
    S.ids_total = total;
    SCK(cudaStreamSynchronize(s));
    if (st) {
        st->max_slab_points = biggest;
        st->halo_points = halo - n;  // every point is owned by one slab
        st->border_pairs = pending;
        st->ms[1] = ms_sel;
        st->ms[2] = ms_run;
        st->ms[3] = ms_merge;
        st->ms[4] = ms_names + tm.lap();
    }
    S.have = true;
    return DBSCAN_OK;
}

}  // namespace

void gbdb_slab_free(dbscan_ctx *c) {
    SlabState *S = c->slab;
    if (!S) return;
    cudaFree(S->parent); cudaFree(S->label); cudaFree(S->core); cudaFree(S->off); cudaFree(S->part);
    cudaFree(S->s_pts); cudaFree(S->s_gid); cudaFree(S->s_core); cudaFree(S->s_lab); cudaFree(S->s_off);
    cudaFree(S->s_ids); cudaFree(S->pk0); cudaFree(S->pk1); cudaFree(S->sort_scratch); cudaFree(S->p_part);
    cudaFree(S->stage); cudaFree(S->dev_in); cudaFree(S->hist); cudaFree(S->bounds); cudaFree(S->cnt); cudaFree(S->ctr);
    cudaFreeHost(S->h_small); cudaFreeHost(S->h_ctr);
    delete S;
    c->slab = nullptr;
}

extern "C" dbscan_status dbscan_run_slabs(dbscan_ctx *c, const void *points, int64_t n, int d, int dtype, double eps,
                                          int64_t min_pts, int32_t num_slabs, uint8_t *core, int32_t *labels,
                                          int64_t *border_offsets, int64_t *num_border_memberships,
                                          dbscan_slab_stats *stats, void *stream) {
    if (!c) return DBSCAN_ERR_INVALID_ARG;
    if (num_border_memberships) *num_border_memberships = 0;
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (n < 0 || n > 0x7ffffffell - 1 || d < 1 || d > c->max_dim) return DBSCAN_ERR_INVALID_ARG;
    if (dtype != DBSCAN_F32 && dtype != DBSCAN_F64) return DBSCAN_ERR_INVALID_ARG;
    if (!(eps > 0.0) || !std::isfinite(eps) || min_pts < 1) return DBSCAN_ERR_INVALID_ARG;
    if (num_slabs < 0 || num_slabs > kMaxSlabs) return DBSCAN_ERR_INVALID_ARG;
    if (n > 0 && (!points || !core || !labels)) return DBSCAN_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (c->slab) c->slab->have = false;
    c->have_run = false;
    c->have_wit = false;
    c->boff_ready = false;
    if (n == 0 && border_offsets) {
        const int64_t zero = 0;
        SCK(cudaMemcpyAsync(border_offsets, &zero, sizeof(zero), cudaMemcpyDefault, s));
        SCK(cudaStreamSynchronize(s));
    }
    if (!c->slab) {
        c->slab = new (std::nothrow) SlabState();
        if (!c->slab) return DBSCAN_ERR_OOM;
    }
    if (n == 0) {
        c->slab->ids_total = 0;
        c->slab->have = true;
        return DBSCAN_OK;
    }
    if (c->max_points < 1) return DBSCAN_ERR_CAPACITY;
    SlabState &S = *c->slab;
    const size_t row = (size_t)d * (dtype == DBSCAN_F64 ? 8 : 4);
    SCK(ensure_small(c, S));
    SCK(ensure_global(c, S, n));
    SCK(ensure_slab(c, S, (int)row));
    Source src;
    src.host = (const char *)points;
    src.row = row;
    const size_t in_bytes = (size_t)n * row;
    cudaPointerAttributes attr{};
    const bool known = cudaPointerGetAttributes(&attr, points) == cudaSuccess;
    if (!known) (void)cudaGetLastError();
    if (known && (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged) && attr.devicePointer) {
        src.direct = (const char *)attr.devicePointer;
    } else {
        // host input: one copy into device memory when it fits with room to spare
        if (c->slab_stage && (!S.dev_in || S.dev_in_bytes < in_bytes)) {
            size_t free_b = 0, total_b = 0;
            cudaFree(S.dev_in);
            S.dev_in = nullptr;
            S.dev_in_bytes = 0;
            if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess && free_b > in_bytes + ((size_t)4 << 30)) {
                if (ctx_malloc(c, &S.dev_in, in_bytes) == cudaSuccess) S.dev_in_bytes = in_bytes;
                else { S.dev_in = nullptr; (void)cudaGetLastError(); }
            } else {
                (void)cudaGetLastError();
            }
        }
        if (c->slab_stage && S.dev_in) {
            SCK(cudaMemcpyAsync(S.dev_in, points, in_bytes, cudaMemcpyHostToDevice, s));
            src.direct = (const char *)S.dev_in;
        } else if (known && attr.type == cudaMemoryTypeHost && attr.devicePointer) {
            src.direct = (const char *)attr.devicePointer;  // pinned: read in place
        } else {
            const size_t want = std::min(kStageBytes, in_bytes);
            if (!S.stage || S.stage_bytes < want) {
                cudaFree(S.stage);
                S.stage = nullptr;
                S.stage_bytes = 0;
                SCK(ctx_malloc(c, &S.stage, want));
                S.stage_bytes = want;
            }
        }
    }
    const long long launches0 = g_launches;
    dbscan_status r;
    if (dtype == DBSCAN_F32)
        r = run_slabs<float>(c, S, src, n, d, dtype, eps, min_pts, num_slabs, core, labels, border_offsets,
                             num_border_memberships, stats, s);
    else
        r = run_slabs<double>(c, S, src, n, d, dtype, eps, min_pts, num_slabs, core, labels, border_offsets,
                              num_border_memberships, stats, s);
    if (stats) stats->kernel_launches = g_launches - launches0;
    c->have_run = false;  // the context's last single run is one slab's, not this call's
    c->have_wit = false;
    c->boff_ready = false;
    return r;
}

extern "C" dbscan_status dbscan_slab_border_ids(dbscan_ctx *c, int32_t *border_ids, int64_t capacity, void *stream) {
    if (!c || capacity < 0) return DBSCAN_ERR_INVALID_ARG;
    if (!c->slab || !c->slab->have) return DBSCAN_ERR_STATE;
    const SlabState &S = *c->slab;
    if (S.ids_total == 0) return DBSCAN_OK;
    if (!border_ids) return DBSCAN_ERR_INVALID_ARG;
    if (capacity < S.ids_total) return DBSCAN_ERR_CAPACITY;
    cudaStream_t s = (cudaStream_t)stream;
    SCK(cudaMemcpyAsync(border_ids, S.ids, 4 * (size_t)S.ids_total, cudaMemcpyDefault, s));
    SCK(cudaStreamSynchronize(s));
    return DBSCAN_OK;
}
