// Device primitives: exclusive scan (prefix sum, Sec. 2 "Prefix sum") and a
// stable LSD radix sort (the integer sort that groups points by cell, Sec. 4.1).
#include <cuda_runtime.h>

#include <mutex>
#include <unordered_map>

#include "internal.cuh"

namespace gbdb {

// ------------------------------------------------------------------ helpers
thread_local long long g_launches = 0;

int grid_for(const void *kernel, int threads, size_t smem) {
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
    auto it = cache.find(kernel);
    if (it != cache.end()) return it->second;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) !=
            cudaSuccess || per_sm <= 0)
        per_sm = 1;
    int g = per_sm * sms;
    cache[kernel] = g;
    return g;
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
// One pass = histogram per tile, scan of the digit-major histogram, stable
// scatter.  A tile is 4096 keys: 8 warps x 16 items x 32 lanes, item j of lane
// l of warp w at tile offset w*512 + j*32 + l, so (warp, item, lane) order is
// input order and ranks taken in that order keep the sort stable.
constexpr int RS_THREADS = 256, RS_WARPS = 8, RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
constexpr int RS_BINS = 256;

int64_t radix_hist_size(int64_t n_max) {
    int64_t nb = (n_max + RS_TILE - 1) / RS_TILE;
    if (nb == 0) nb = 1;
    return nb * RS_BINS + 1;
}

__global__ void __launch_bounds__(RS_THREADS)
k_radix_hist(const uint64_t *__restrict__ keys, int n_host, const int *n_dev, int shift,
             unsigned *__restrict__ hist, int nblk) {
    __shared__ unsigned cnt[RS_BINS];
    const int n = n_dev ? *n_dev : n_host;
    for (int i = threadIdx.x; i < RS_BINS; i += RS_THREADS) cnt[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    if (base < n) {
#pragma unroll 4
        for (int j = 0; j < RS_ITEMS; ++j) {
            int64_t i = base + (int64_t)j * RS_THREADS + threadIdx.x;
            unsigned dig = i < n ? (unsigned)((keys[i] >> shift) & 255u) : 0xffffffffu;
            unsigned peers = __match_any_sync(0xffffffffu, dig);
            int leader = __ffs(peers) - 1;
            if (dig != 0xffffffffu && (int)(threadIdx.x & 31) == leader)
                atomicAdd(&cnt[dig], (unsigned)__popc(peers));
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < RS_BINS; i += RS_THREADS) hist[(int64_t)i * nblk + blockIdx.x] = cnt[i];
}

__global__ void __launch_bounds__(RS_THREADS)
k_radix_scatter(const uint64_t *__restrict__ kin, const uint32_t *__restrict__ vin,
                uint64_t *__restrict__ kout, uint32_t *__restrict__ vout, int n_host,
                const int *n_dev, int shift, const int *__restrict__ offs, int nblk) {
    __shared__ int wcnt[RS_WARPS][RS_BINS];
    __shared__ int gbase[RS_BINS];
    const int n = n_dev ? *n_dev : n_host;
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    if (base >= n) return;  // whole block uniform
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < RS_WARPS * RS_BINS; i += RS_THREADS) (&wcnt[0][0])[i] = 0;
    for (int i = threadIdx.x; i < RS_BINS; i += RS_THREADS) gbase[i] = offs[(int64_t)i * nblk + blockIdx.x];
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    const int64_t wbase = base + (int64_t)warp * (32 * RS_ITEMS);
    uint64_t k[RS_ITEMS];
    uint32_t v[RS_ITEMS];
    int r[RS_ITEMS];
#pragma unroll
    for (int j = 0; j < RS_ITEMS; ++j) {
        int64_t i = wbase + j * 32 + lane;
        bool ok = i < n;
        k[j] = ok ? kin[i] : 0;
        v[j] = ok ? vin[i] : 0;
        unsigned dig = ok ? (unsigned)((k[j] >> shift) & 255u) : 0xffffffffu;
        unsigned peers = __match_any_sync(0xffffffffu, dig);
        int before = ok ? wcnt[warp][dig] : 0;
        __syncwarp();
        if (ok && lane == __ffs(peers) - 1) wcnt[warp][dig] = before + __popc(peers);
        __syncwarp();
        r[j] = ok ? before + __popc(peers & lt) : -1;
    }
    __syncthreads();
    // Exclusive prefix over warps for each digit, plus the block's global base.
    for (int dgt = threadIdx.x; dgt < RS_BINS; dgt += RS_THREADS) {
        int run = gbase[dgt];
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) {
            int c = wcnt[w][dgt];
            wcnt[w][dgt] = run;
            run += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < RS_ITEMS; ++j) {
        if (r[j] >= 0) {
            unsigned dig = (unsigned)((k[j] >> shift) & 255u);
            int pos = wcnt[warp][dig] + r[j];
            kout[pos] = k[j];
            vout[pos] = v[j];
        }
    }
}

int radix_sort_u64(uint64_t *k0, uint32_t *v0, uint64_t *k1, uint32_t *v1, int n_host,
                   const int *n_dev, int64_t n_max, int bits, unsigned *hist, long long *part,
                   cudaStream_t s) {
    int nblk = (int)((n_max + RS_TILE - 1) / RS_TILE);
    if (nblk == 0 || bits <= 0) return 0;
    const int64_t hsz = (int64_t)nblk * RS_BINS;
    int *offs = reinterpret_cast<int *>(hist);  // scanned in place (counts fit in int)
    int cur = 0;
    for (int shift = 0; shift < bits; shift += 8) {
        const uint64_t *ki = cur ? k1 : k0;
        const uint32_t *vi = cur ? v1 : v0;
        uint64_t *ko = cur ? k0 : k1;
        uint32_t *vo = cur ? v0 : v1;
        k_radix_hist<<<nblk, RS_THREADS, 0, s>>>(ki, n_host, n_dev, shift, hist, nblk); count_launch();
        scan_i32_to_i32(offs, offs, hsz, nullptr, hsz, part, s);
        k_radix_scatter<<<nblk, RS_THREADS, 0, s>>>(ki, vi, ko, vo, n_host, n_dev, shift, offs, nblk); count_launch();
        cur ^= 1;
    }
    return cur;
}

}  // namespace gbdb
