// Device primitives: exclusive scan (prefix sum, Sec. 2 "Prefix sum") and a
// stable LSD radix sort (the integer sort that groups points by cell, Sec. 4.1).
#include <cuda_runtime.h>

#include <mutex>
#include <unordered_map>

#include "internal.cuh"

namespace gbdb {

// ------------------------------------------------------------------ helpers
thread_local long long g_launches = 0;

static thread_local int t_grid_cap = 0;
void set_grid_cap(int blocks_per_sm) { t_grid_cap = blocks_per_sm; }
int grid_cap() { return t_grid_cap; }

int grid_for(const void *kernel, int threads, size_t smem) {
    const int cap = t_grid_cap;
    static std::mutex mu;
    static std::unordered_map<const void *, int> cache;
    static int sms = 0;
    std::lock_guard<std::mutex> lock(mu);
    if (sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    int per_sm = 0;
    auto it = cache.find(kernel);
    if (it != cache.end()) {
        per_sm = it->second;
    } else {
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess ||
            per_sm <= 0)
            per_sm = 1;
        cache[kernel] = per_sm;
    }
    if (cap > 0 && cap < per_sm) per_sm = cap;
    return per_sm * sms;
}

template <typename T> __device__ __forceinline__ T warp_incl_scan(T v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// Block-wide exclusive scan of one value per thread; returns the prefix and
// writes the block total to *total (all threads).  blockDim.x <= 1024.
template <typename T> __device__ T block_excl_scan(T v, T *sh /*[33]*/, T *total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
    T inc = warp_incl_scan(v);
    if (lane == 31) sh[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T w = lane < nwarps ? sh[lane] : T(0);
        T wi = warp_incl_scan(w);
        sh[lane] = wi - w;
        if (lane == 31) sh[32] = wi;
    }
    __syncthreads();
    T res = sh[warp] + inc - v;
    *total = sh[32];
    __syncthreads();
    return res;
}

// ------------------------------------------------------------------ scan
constexpr int SC_THREADS = 256, SC_ITEMS = 8, SC_TILE = SC_THREADS * SC_ITEMS;

int64_t scan_partials(int64_t n_max) { return (n_max + SC_TILE - 1) / SC_TILE + 1; }

template <typename TI, typename TO>
__global__ void __launch_bounds__(SC_THREADS)
k_scan_reduce(const TI *__restrict__ in, int64_t n_host, const int *n_dev, long long *part) {
    __shared__ long long sh[33];
    const int64_t n = n_dev ? (int64_t)*n_dev : n_host;
    const int64_t base = (int64_t)blockIdx.x * SC_TILE;
    long long s = 0;
#pragma unroll
    for (int j = 0; j < SC_ITEMS; ++j) {
        int64_t i = base + (int64_t)j * SC_THREADS + threadIdx.x;
        if (i < n) s += (long long)in[i];
    }
    long long tot;
    block_excl_scan<long long>(s, sh, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// Single block: exclusive scan of the tile sums in place.
__global__ void __launch_bounds__(1024) k_scan_partials(long long *part, int nb) {
    __shared__ long long sh[33];
    long long carry = 0;
    for (int base = 0; base < nb; base += 1024) {
        int i = base + threadIdx.x;
        long long v = i < nb ? part[i] : 0;
        long long tot;
        long long ex = block_excl_scan<long long>(v, sh, &tot);
        if (i < nb) part[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) part[nb] = carry;
}

template <typename TI, typename TO>
__global__ void __launch_bounds__(SC_THREADS)
k_scan_down(const TI *in, TO *out, int64_t n_host, const int *n_dev, const long long *part,
            int nb) {
    __shared__ long long sh[33];
    const int64_t n = n_dev ? (int64_t)*n_dev : n_host;
    const int64_t base = (int64_t)blockIdx.x * SC_TILE + (int64_t)threadIdx.x * SC_ITEMS;
    long long v[SC_ITEMS];
    long long s = 0;
#pragma unroll
    for (int j = 0; j < SC_ITEMS; ++j) {
        int64_t i = base + j;
        v[j] = i < n ? (long long)in[i] : 0;
        s += v[j];
    }
    long long tot;
    long long ex = block_excl_scan<long long>(s, sh, &tot) + part[blockIdx.x];
#pragma unroll
    for (int j = 0; j < SC_ITEMS; ++j) {
        int64_t i = base + j;
        if (i < n) out[i] = (TO)ex;
        ex += v[j];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = (TO)part[nb];
}

template <typename TI, typename TO>
static void scan_impl(const TI *in, TO *out, int64_t n_host, const int *n_dev, int64_t n_max,
                      long long *part, cudaStream_t s) {
    int nb = (int)((n_max + SC_TILE - 1) / SC_TILE);
    if (nb == 0) nb = 1;
    k_scan_reduce<TI, TO><<<nb, SC_THREADS, 0, s>>>(in, n_host, n_dev, part); count_launch();
    k_scan_partials<<<1, 1024, 0, s>>>(part, nb); count_launch();
    k_scan_down<TI, TO><<<nb, SC_THREADS, 0, s>>>(in, out, n_host, n_dev, part, nb); count_launch();
}

void scan_i32_to_i32(const int *in, int *out, int64_t n_host, const int *n_dev, int64_t n_max,
                     long long *part, cudaStream_t s) {
    scan_impl<int, int>(in, out, n_host, n_dev, n_max, part, s);
}
void scan_i64_to_i64(const long long *in, long long *out, int64_t n_host, const int *n_dev,
                     int64_t n_max, long long *part, cudaStream_t s) {
    scan_impl<long long, long long>(in, out, n_host, n_dev, n_max, part, s);
}

// ------------------------------------------------------------- radix sort
// Stable LSD radix sort of 64-bit keys (optionally carrying 32-bit values) on
// the key bits [lo, lo + bits), 8 bits a pass -- the integer sort that groups
// points by cell (Sec. 4.1).
//
// One-sweep layout: one kernel counts the digits of every pass at once; each
// pass is then a single scatter kernel.  A scatter block takes the next tile of
// 4096 keys from an atomic tile counter (so tiles start in order and every
// earlier tile belongs to a block that is already running), ranks its keys
// stably per digit inside the tile, publishes its per-digit count, and looks
// back over the earlier tiles' published counts to find its global offset
// (decoupled look-back).  The look-back waits on flags written by other
// blocks; each wait is bounded by max_iters and raises DEVICE_TIMEOUT instead
// of spinning on.
//
// Tile layout: 8 warps x 16 items x 32 lanes; item j of lane l of warp w sits
// at tile offset w*512 + j*32 + l, so (warp, item, lane) order is input order
// and ranks taken in that order keep the sort stable.
constexpr int RS_THREADS = 256, RS_WARPS = 8, RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
constexpr int RS_BINS = 256;
constexpr int RS_MAX_PASSES = 8;
constexpr int RS_LOOK = 16;  // look-back window (tiles read per step)
constexpr unsigned long long ST_AGG = 1ull << 62, ST_INC = 2ull << 62, ST_VAL = (1ull << 62) - 1;

static int64_t rs_tiles(int64_t n_max) {
    int64_t t = (n_max + RS_TILE - 1) / RS_TILE;
    return t > 0 ? t : 1;
}

// scratch: [passes][256] u32 digit offsets | [passes] u32 tile counters (padded
// to 256 B) | [passes][tiles][256] u64 tile status
size_t sort_scratch_bytes(int64_t n_max) {
    return (size_t)RS_MAX_PASSES * RS_BINS * 4 + 256 + (size_t)RS_MAX_PASSES * rs_tiles(n_max) * RS_BINS * 8;
}

__global__ void k_flag_error(DevCounters *ctr, int code, int info) { set_error(ctr, code, info); }

__global__ void __launch_bounds__(RS_THREADS)
k_radix_hist(const uint64_t *__restrict__ keys, int n_host, const int *n_dev, int lo, int passes,
             unsigned *__restrict__ ghist) {
    __shared__ unsigned sh[RS_MAX_PASSES][RS_BINS];
    const int n = n_dev ? *n_dev : n_host;
    for (int i = threadIdx.x; i < RS_MAX_PASSES * RS_BINS; i += RS_THREADS) (&sh[0][0])[i] = 0;
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)RS_THREADS + threadIdx.x; i < n; i += (int64_t)gridDim.x * RS_THREADS) {
        const uint64_t k = keys[i];
        for (int p = 0; p < passes; ++p) atomicAdd(&sh[p][(unsigned)(k >> (lo + 8 * p)) & 255u], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * RS_BINS; i += RS_THREADS) {
        const unsigned v = (&sh[0][0])[i];
        if (v) atomicAdd(ghist + i, v);
    }
}

// Exclusive scan of each pass's 256 digit counts (one block).
__global__ void __launch_bounds__(RS_BINS) k_radix_offsets(unsigned *ghist, int passes) {
    __shared__ long long sh[33];
    for (int p = 0; p < passes; ++p) {
        const unsigned v = ghist[p * RS_BINS + threadIdx.x];
        long long tot;
        const long long ex = block_excl_scan<long long>((long long)v, sh, &tot);
        ghist[p * RS_BINS + threadIdx.x] = (unsigned)ex;
    }
}

template <bool KV>
__global__ void __launch_bounds__(RS_THREADS)
k_radix_scatter(const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                uint64_t *__restrict__ kout, uint32_t *__restrict__ vout, int n_host, const int *n_dev,
                int shift, const unsigned *__restrict__ goff, unsigned long long *status, int *tile_ctr,
                DevCounters *ctr, int max_iters) {
    if (run_failed_block(ctr)) return;
    __shared__ int wcnt[RS_WARPS][RS_BINS];
    __shared__ int s_tile;
    const int n = n_dev ? *n_dev : n_host;
    if (threadIdx.x == 0) s_tile = atomicAdd(tile_ctr, 1);
    __syncthreads();
    const int tile = s_tile;
    const int64_t base = (int64_t)tile * RS_TILE;
    if (base >= n) return;  // uniform per block; no later tile has keys either
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < RS_WARPS * RS_BINS; i += RS_THREADS) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    const int64_t wbase = base + (int64_t)warp * (32 * RS_ITEMS);
    uint64_t k[RS_ITEMS];
    uint32_t v[RS_ITEMS];
    int r[RS_ITEMS];
    // issue every load of the tile before ranking, so they overlap
#pragma unroll
    for (int j = 0; j < RS_ITEMS; ++j) {
        const int64_t i = wbase + j * 32 + lane;
        k[j] = i < n ? kin[i] : 0;
        if (KV) v[j] = i < n ? vin[i] : 0;
    }
#pragma unroll
    for (int j = 0; j < RS_ITEMS; ++j) {
        const int64_t i = wbase + j * 32 + lane;
        const bool ok = i < n;
        const unsigned dig = ok ? (unsigned)((k[j] >> shift) & 255u) : 0xffffffffu;
        const unsigned peers = __match_any_sync(0xffffffffu, dig);
        const int before = ok ? wcnt[warp][dig] : 0;
        __syncwarp();
        if (ok && lane == __ffs(peers) - 1) wcnt[warp][dig] = before + __popc(peers);
        __syncwarp();
        r[j] = ok ? before + __popc(peers & lt) : -1;
    }
    __syncthreads();
    // One thread per digit: exclusive prefix over warps, tile total, publish,
    // look back, publish the inclusive prefix, and fold the global base into
    // the per-warp offsets.
    {
        const int dgt = threadIdx.x;
        int run = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) {
            const int c = wcnt[w][dgt];
            wcnt[w][dgt] = run;
            run += c;
        }
        volatile unsigned long long *st = status + (int64_t)tile * RS_BINS + dgt;
        long long excl = 0;
        if (tile == 0) {
            *st = ST_INC | (unsigned long long)run;
        } else {
            *st = ST_AGG | (unsigned long long)run;
            // Look back RS_LOOK tiles at a time: the window's loads are issued
            // together, then summed nearest first up to the first inclusive
            // prefix; a tile not yet published is polled (bounded).
            bool found = false;
            for (int t0 = tile - 1; t0 >= 0 && !found; t0 -= RS_LOOK) {
                unsigned long long x[RS_LOOK];
#pragma unroll
                for (int j = 0; j < RS_LOOK; ++j)
                    x[j] = t0 - j >= 0 ? *(volatile unsigned long long *)(status + (int64_t)(t0 - j) * RS_BINS + dgt)
                                       : (unsigned long long)(2ull << 62);
#pragma unroll
                for (int j = 0; j < RS_LOOK; ++j) {
                    if (!found) {
                        if ((x[j] & ~ST_VAL) == 0) {
                            volatile unsigned long long *src = status + (int64_t)(t0 - j) * RS_BINS + dgt;
                            int it = 0;
                            while ((x[j] & ~ST_VAL) == 0 && it < max_iters) { x[j] = *src; ++it; }
                            if ((x[j] & ~ST_VAL) == 0) {
                                set_error(ctr, DBSCAN_ERR_DEVICE_TIMEOUT, 40);
                                x[j] = 2ull << 62;
                            }
                        }
                        excl += (long long)(x[j] & ST_VAL);
                        found = (x[j] & ~ST_VAL) == ST_INC;
                    }
                }
            }
            *st = ST_INC | (unsigned long long)(excl + run);
        }
        const int gb = (int)(goff[dgt] + excl);
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) wcnt[w][dgt] += gb;
    }
    __syncthreads();
    // After a timed-out wait the offsets are unknown: write nothing (the run
    // reports DEVICE_TIMEOUT); positions are also checked against n.
    if (*(volatile int *)&ctr->err == DBSCAN_ERR_DEVICE_TIMEOUT) return;
#pragma unroll
    for (int j = 0; j < RS_ITEMS; ++j) {
        if (r[j] >= 0) {
            const unsigned dig = (unsigned)((k[j] >> shift) & 255u);
            const int pos = wcnt[warp][dig] + r[j];
            if (pos >= 0 && pos < n) {
                kout[pos] = k[j];
                if (KV) vout[pos] = v[j];
            }
        }
    }
}

int radix_sort_u64(uint64_t *k0, uint32_t *v0, uint64_t *k1, uint32_t *v1, int n_host, const int *n_dev,
                   int64_t n_max, int lo, int bits, void *scratch, size_t scratch_bytes, DevCounters *ctr,
                   int max_iters, cudaStream_t s) {
    const int passes = (bits + 7) / 8;
    if (passes <= 0) return 0;
    if (scratch_bytes < sort_scratch_bytes(n_max)) {
        k_flag_error<<<1, 1, 0, s>>>(ctr, DBSCAN_ERR_CAPACITY, 60);
        count_launch();
        return 0;
    }
    const int64_t tiles = rs_tiles(n_max);
    unsigned *ghist = reinterpret_cast<unsigned *>(scratch);
    int *tile_ctr = reinterpret_cast<int *>(ghist + RS_MAX_PASSES * RS_BINS);
    unsigned long long *status =
        reinterpret_cast<unsigned long long *>(reinterpret_cast<char *>(scratch) + RS_MAX_PASSES * RS_BINS * 4 + 256);
    cudaMemsetAsync(scratch, 0,
                    (size_t)RS_MAX_PASSES * RS_BINS * 4 + 256 + (size_t)passes * tiles * RS_BINS * 8, s);
    const int gh = grid_for((const void *)k_radix_hist, RS_THREADS);
    k_radix_hist<<<gh, RS_THREADS, 0, s>>>(k0, n_host, n_dev, lo, passes, ghist); count_launch();
    k_radix_offsets<<<1, RS_BINS, 0, s>>>(ghist, passes); count_launch();
    int cur = 0;
    for (int p = 0; p < passes; ++p) {
        const uint64_t *ki = cur ? k1 : k0;
        const uint32_t *vi = cur ? v1 : v0;
        uint64_t *ko = cur ? k0 : k1;
        uint32_t *vo = cur ? v0 : v1;
        unsigned long long *st = status + (size_t)p * tiles * RS_BINS;
        if (v0)
            k_radix_scatter<true><<<(int)tiles, RS_THREADS, 0, s>>>(ki, vi, ko, vo, n_host, n_dev, lo + 8 * p,
                                                                     ghist + p * RS_BINS, st, tile_ctr + p, ctr,
                                                                     max_iters);
        else
            k_radix_scatter<false><<<(int)tiles, RS_THREADS, 0, s>>>(ki, nullptr, ko, nullptr, n_host, n_dev,
                                                                      lo + 8 * p, ghist + p * RS_BINS, st,
                                                                      tile_ctr + p, ctr, max_iters);
        count_launch();
        cur ^= 1;
    }
    return cur;
}

}  // namespace gbdb
