// Cells (Algorithm 1 line 2; Sec. 4.1 "Grid Computation"): bounding box,
// FP64 cell keys, grouping points by cell, the hash of non-empty cells and the
// cached neighbour-cell lists (Sec. 5.1 caches them per cell as well).
#include "geom.cuh"
#include "grid.cuh"

namespace gbdb {

// ---------------------------------------------------------------- bbox
// Per-dimension minimum and maximum.  FP32 input is reduced in FP32 (exact
// min/max on the FP32 pipe); FP64 input through an order-preserving map of
// its bits to int64, so the reduction runs on the integer pipe (GB300's FP64
// rate is a small fraction of its FP32 rate).
constexpr int BB_THREADS = 256;

template <typename T> struct BBoxOps;
template <> struct BBoxOps<float> {
    using A = float;
    static __device__ __forceinline__ A key(float x) { return x; }
    static __device__ __forceinline__ A lo_init() { return __int_as_float(0x7f800000); }
    static __device__ __forceinline__ A hi_init() { return __int_as_float(0xff800000); }
    static __device__ __forceinline__ A mn(A a, A b) { return fminf(a, b); }
    static __device__ __forceinline__ A mx(A a, A b) { return fmaxf(a, b); }
    static __device__ __forceinline__ double to_d(A a) { return (double)a; }
    static __device__ __forceinline__ bool finite(float x) { return (__float_as_uint(x) & 0x7f800000u) != 0x7f800000u; }
};
template <> struct BBoxOps<double> {
    using A = long long;
    static __device__ __forceinline__ A key(double x) {
        long long b = __double_as_longlong(x);
        return b >= 0 ? b : (b ^ 0x7fffffffffffffffll);
    }
    static __device__ __forceinline__ A lo_init() { return 0x7fffffffffffffffll; }
    static __device__ __forceinline__ A hi_init() { return (long long)0x8000000000000000ull; }
    static __device__ __forceinline__ A mn(A a, A b) { return a < b ? a : b; }
    static __device__ __forceinline__ A mx(A a, A b) { return a > b ? a : b; }
    static __device__ __forceinline__ double to_d(A a) {
        return __longlong_as_double(a >= 0 ? a : (a ^ 0x7fffffffffffffffll));
    }
    static __device__ __forceinline__ bool finite(double x) {
        return ((__double_as_longlong(x) >> 52) & 0x7ff) != 0x7ff;
    }
};

__device__ __forceinline__ long long ordered_key(double x) {
    const long long b = __double_as_longlong(x);
    return b >= 0 ? b : (b ^ 0x7fffffffffffffffll);
}

// out[0..8): ordered keys of the minima, out[8..16): of the maxima, out[16]:
// non-finite flag.  The host maps the keys back to doubles.
__global__ void k_bbox_init(long long *out) {
    const int j = threadIdx.x;
    if (j < 2 * kMaxDim) out[j] = j < kMaxDim ? 0x7fffffffffffffffll : (long long)0x8000000000000000ull;
    if (j == 0) out[2 * kMaxDim] = 0;
}

template <typename T>
__global__ void __launch_bounds__(BB_THREADS)
k_bbox(const T *__restrict__ X, int n, int d, long long *__restrict__ out) {
    using O = BBoxOps<T>;
    using A = typename O::A;
    __shared__ A smn[BB_THREADS / 32][kMaxDim], smx[BB_THREADS / 32][kMaxDim];
    A mn[kMaxDim], mx[kMaxDim];
#pragma unroll
    for (int j = 0; j < kMaxDim; ++j) { mn[j] = O::lo_init(); mx[j] = O::hi_init(); }
    bool nonfinite = false;
    for (int i = blockIdx.x * BB_THREADS + threadIdx.x; i < n; i += gridDim.x * BB_THREADS) {
#pragma unroll
        for (int j = 0; j < kMaxDim; ++j) {
            if (j < d) {
                const T x = X[(int64_t)i * d + j];
                nonfinite |= !O::finite(x);
                const A k = O::key(x);
                mn[j] = O::mn(mn[j], k);
                mx[j] = O::mx(mx[j], k);
            }
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < kMaxDim; ++j) {
        if (j < d) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                mn[j] = O::mn(mn[j], __shfl_xor_sync(0xffffffffu, mn[j], o));
                mx[j] = O::mx(mx[j], __shfl_xor_sync(0xffffffffu, mx[j], o));
            }
            if (lane == 0) { smn[warp][j] = mn[j]; smx[warp][j] = mx[j]; }
        }
    }
    if (__any_sync(0xffffffffu, nonfinite) && lane == 0) atomicOr((unsigned long long *)(out + 2 * kMaxDim), 1ull);
    __syncthreads();
    if (threadIdx.x < d) {
        const int j = threadIdx.x;
        A a = smn[0][j], b = smx[0][j];
        for (int w = 1; w < BB_THREADS / 32; ++w) { a = O::mn(a, smn[w][j]); b = O::mx(b, smx[w][j]); }
        atomicMin(out + j, ordered_key(O::to_d(a)));
        atomicMax(out + kMaxDim + j, ordered_key(O::to_d(b)));
    }
}

void launch_bbox(const void *X, int dtype, int n, int d, int nb, long long *out, cudaStream_t s) {
    k_bbox_init<<<1, 32, 0, s>>>(out); count_launch();
    if (dtype == DBSCAN_F32)
        k_bbox<float><<<nb, BB_THREADS, 0, s>>>((const float *)X, n, d, out);
    else
        k_bbox<double><<<nb, BB_THREADS, 0, s>>>((const double *)X, n, d, out);
    count_launch();
}

// ---------------------------------------------------------------- keys
// Cell coordinate k_j = floor(fl(fl(x_j - origin_j) * (1/s))), then Morton
// packed.  Keys are computed in FP64 for every input type.
template <typename T>
__global__ void __launch_bounds__(256)
k_keys(const T *__restrict__ X, RunParams P, uint64_t *__restrict__ keys, uint32_t *__restrict__ vals) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
        int c[kMaxDim];
#pragma unroll
        for (int j = 0; j < kMaxDim; ++j) {
            if (j < P.d) {
                double x = (double)X[(int64_t)i * P.d + j];
                double t = __dmul_rn(__dsub_rn(x, P.origin[j]), P.inv_s);
                int k = (int)floor(t);
                c[j] = k < 0 ? 0 : (k > P.kmax[j] ? P.kmax[j] : k);
            } else {
                c[j] = 0;
            }
        }
        const uint64_t key = morton_encode(c, P.d, P.bits);
        if (P.ib) {
            keys[i] = (key << P.ib) | (uint64_t)i;
        } else {
            keys[i] = key;
            vals[i] = (uint32_t)i;
        }
    }
}

void launch_keys(const void *X, int dtype, const RunParams &P, uint64_t *keys, uint32_t *vals,
                 cudaStream_t s) {
    if (dtype == DBSCAN_F32) {
        int g = grid_for((const void *)k_keys<float>, 256);
        k_keys<float><<<g, 256, 0, s>>>((const float *)X, P, keys, vals); count_launch();
    } else {
        int g = grid_for((const void *)k_keys<double>, 256);
        k_keys<double><<<g, 256, 0, s>>>((const double *)X, P, keys, vals); count_launch();
    }
}

// ---------------------------------------------------------------- cells
__global__ void __launch_bounds__(256)
k_cell_flags(const uint64_t *__restrict__ K, int n, int ib, int *__restrict__ flags) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        flags[i] = (i == 0 || (K[i] >> ib) != (K[i - 1] >> ib)) ? 1 : 0;
}

// Gather the points into cell order, zero padded to the storage width, and
// record the cell table: cell_start[m+1], cell_key[m], cell_of[n], orig[n].
template <typename T, int SD>
__global__ void __launch_bounds__(256)
k_gather(const T *__restrict__ X, int n, int d, int ib, const uint64_t *__restrict__ K,
         const uint32_t *__restrict__ V, const int *__restrict__ flags, const int *__restrict__ cid,
         float *__restrict__ pf, double *__restrict__ pd, int *__restrict__ orig,
         int *__restrict__ cell_of, int *__restrict__ cell_start, uint64_t *__restrict__ cell_key,
         DevCounters *ctr) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint64_t key = K[i];
        const int o = ib ? (int)(key & ((1ull << ib) - 1)) : (int)V[i];
        const int c = cid[i] + flags[i] - 1;
        orig[i] = o;
        cell_of[i] = c;
        if (flags[i]) { cell_start[c] = i; cell_key[c] = key >> ib; }
        if (i == 0) {
            const int m = cid[n];
            ctr->m = m;
            cell_start[m] = n;
        }
        float f[SD];
        double x[SD];
#pragma unroll
        for (int j = 0; j < SD; ++j) {
            x[j] = j < d ? (double)X[(int64_t)o * d + j] : 0.0;
            f[j] = (float)x[j];
        }
        if constexpr (SD == 2) {
            reinterpret_cast<float2 *>(pf)[i] = make_float2(f[0], f[1]);
        } else {
#pragma unroll
            for (int j = 0; j < SD; j += 4)
                reinterpret_cast<float4 *>(pf)[(int64_t)i * (SD / 4) + j / 4] =
                    make_float4(f[j], f[j + 1], f[j + 2], f[j + 3]);
        }
        if (pd) {
#pragma unroll
            for (int j = 0; j < SD; j += 2)
                reinterpret_cast<double2 *>(pd)[(int64_t)i * (SD / 2) + j / 2] = make_double2(x[j], x[j + 1]);
        }
    }
}

template <int SD>
static void gather_sd(const void *X, int dtype, int n, int d, int ib, const uint64_t *K, const uint32_t *V,
                      const int *flags, const int *cid, float *pf, double *pd, int *orig, int *cell_of,
                      int *cell_start, uint64_t *cell_key, DevCounters *ctr, cudaStream_t s) {
    if (dtype == DBSCAN_F32) {
        int g = grid_for((const void *)k_gather<float, SD>, 256);
        k_gather<float, SD><<<g, 256, 0, s>>>((const float *)X, n, d, ib, K, V, flags, cid, pf, nullptr, orig,
                                              cell_of, cell_start, cell_key, ctr); count_launch();
    } else {
        int g = grid_for((const void *)k_gather<double, SD>, 256);
        k_gather<double, SD><<<g, 256, 0, s>>>((const double *)X, n, d, ib, K, V, flags, cid, pf, pd, orig,
                                               cell_of, cell_start, cell_key, ctr); count_launch();
    }
}

void launch_cells(const void *X, int dtype, int n, int d, int SD, int ib, const uint64_t *K, const uint32_t *V,
                  int *flags, int *cid, long long *part, float *pf, double *pd, int *orig,
                  int *cell_of, int *cell_start, uint64_t *cell_key, DevCounters *ctr, cudaStream_t s) {
    int g = grid_for((const void *)k_cell_flags, 256);
    k_cell_flags<<<g, 256, 0, s>>>(K, n, ib, flags); count_launch();
    scan_i32_to_i32(flags, cid, n, nullptr, n, part, s);
    if (SD == 2)
        gather_sd<2>(X, dtype, n, d, ib, K, V, flags, cid, pf, pd, orig, cell_of, cell_start, cell_key, ctr, s);
    else if (SD == 4)
        gather_sd<4>(X, dtype, n, d, ib, K, V, flags, cid, pf, pd, orig, cell_of, cell_start, cell_key, ctr, s);
    else
        gather_sd<8>(X, dtype, n, d, ib, K, V, flags, cid, pf, pd, orig, cell_of, cell_start, cell_key, ctr, s);
}

// ---------------------------------------------------------------- boxes
// Per-cell FP32 bounding box of the points pts[start[c] .. start[c+1]) (exact
// min/max of the stored FP32 coordinates).  One warp per cell.  Empty ranges
// get an empty box (+inf, -inf).
template <int SD>
__global__ void __launch_bounds__(256)
k_boxes(const float *__restrict__ pts, const int *__restrict__ start, const DevCounters *ctr,
        float4 *__restrict__ lo, float4 *__restrict__ hi) {
    const int m = ctr->m;
    const int lane = threadIdx.x & 31;
    for (int c = warp_id_global(); c < m; c += warps_global()) {
        const int s0 = start[c], s1 = start[c + 1];
        float l[4] = {INFINITY, INFINITY, INFINITY, INFINITY}, h[4] = {-INFINITY, -INFINITY, -INFINITY, -INFINITY};
        for (int t = s0 + lane; t < s1; t += 32) {
            float x[4] = {0.f, 0.f, 0.f, 0.f};
            if constexpr (SD == 2) {
                const float2 a = reinterpret_cast<const float2 *>(pts)[t];
                x[0] = a.x;
                x[1] = a.y;
            } else {
                const float4 a = reinterpret_cast<const float4 *>(pts)[t];
                x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) { l[j] = fminf(l[j], x[j]); h[j] = fmaxf(h[j], x[j]); }
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                l[j] = fminf(l[j], __shfl_xor_sync(0xffffffffu, l[j], o));
                h[j] = fmaxf(h[j], __shfl_xor_sync(0xffffffffu, h[j], o));
            }
        }
        if (lane == 0) {
            lo[c] = make_float4(l[0], l[1], l[2], l[3]);
            hi[c] = make_float4(h[0], h[1], h[2], h[3]);
        }
    }
}

void launch_boxes(int SD, const float *pts, const int *start, const DevCounters *ctr, float4 *lo, float4 *hi,
                  cudaStream_t s) {
    if (SD == 2) {
        int g = grid_for((const void *)k_boxes<2>, 256);
        k_boxes<2><<<g, 256, 0, s>>>(pts, start, ctr, lo, hi);
    } else {
        int g = grid_for((const void *)k_boxes<4>, 256);
        k_boxes<4><<<g, 256, 0, s>>>(pts, start, ctr, lo, hi);
    }
    count_launch();
}

// ---------------------------------------------------------------- hash
__global__ void __launch_bounds__(256) k_hash_clear(ulonglong2 *__restrict__ ht, const DevCounters *ctr) {
    const uint64_t cap = hash_capacity(ctr->m);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < cap;
         i += (uint64_t)gridDim.x * blockDim.x)
        ht[i] = make_ulonglong2(kEmptyKey, 0);
}

__global__ void __launch_bounds__(256)
k_hash_insert(ulonglong2 *__restrict__ ht, const uint64_t *__restrict__ cell_key, DevCounters *ctr) {
    const int m = ctr->m;
    const uint64_t mask = hash_capacity(m) - 1;
    const int lg = hash_log2(mask + 1);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x) {
        const uint64_t key = cell_key[c];
        uint64_t s = hash_slot(key, lg);
        bool done = false;
        for (uint64_t it = 0; it <= mask; ++it) {
            unsigned long long prev = atomicCAS(&ht[s].x, (unsigned long long)kEmptyKey, (unsigned long long)key);
            if (prev == kEmptyKey) { ht[s].y = (unsigned long long)c; done = true; break; }
            s = (s + 1) & mask;
        }
        if (!done) set_error(ctr, DBSCAN_ERR_CAPACITY, 10);
    }
}

void launch_hash(ulonglong2 *ht, const uint64_t *cell_key, DevCounters *ctr, cudaStream_t s) {
    int g = grid_for((const void *)k_hash_clear, 256);
    k_hash_clear<<<g, 256, 0, s>>>(ht, ctr); count_launch();
    g = grid_for((const void *)k_hash_insert, 256);
    k_hash_insert<<<g, 256, 0, s>>>(ht, cell_key, ctr); count_launch();
}

// ---------------------------------------------------------------- neighbours
// NeighborCells(g) (Algorithm 2): every non-empty cell h != g whose integer
// offset delta from g satisfies sum_j max(|delta_j| - 1, 0)^2 <= d, looked up
// in the hash; in the FP32-band mode cells whose point boxes are farther than
// eps apart are dropped.  One warp per cell; each lane takes NB_U offsets per
// round and issues their first probes together.  The ids go to a fixed stride
// per cell (stride = number of offsets of d), in offset-table order (nearest
// first), with their count in nbr_cnt and, in nbr_near, how many of them come
// from the first n_near offsets (|delta|_inf <= 1).
constexpr int NB_U = 4;

template <int D>
__global__ void __launch_bounds__(256)
k_neighbors(const uint64_t *__restrict__ cell_key, const ulonglong2 *__restrict__ ht, RunParams P,
            const signed char *__restrict__ offs, int noff, int n_near, const float4 *__restrict__ blo,
            const float4 *__restrict__ bhi, int *__restrict__ nbr_cnt, int *__restrict__ nbr_near,
            int *__restrict__ nbr, DevCounters *ctr) {
    const int m = ctr->m;
    const uint64_t mask = hash_capacity(m) - 1;
    const int lg = hash_log2(mask + 1);
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    long long total = 0;
    for (int c = warp_id_global(); c < m; c += warps_global()) {
        const uint64_t ckey = cell_key[c];
        int cc[D];
        {
            int tmp[kMaxDim];
            morton_decode(ckey, D, P.bits, tmp);
#pragma unroll
            for (int j = 0; j < D; ++j) cc[j] = tmp[j];
        }
        const long long base = (long long)c * noff;
        float4 clo = make_float4(0.f, 0.f, 0.f, 0.f), chi = clo;
        if (P.box) { clo = blo[c]; chi = bhi[c]; }
        int cnt = 0, near = 0;
        for (int o0 = 0; o0 < noff; o0 += 32 * NB_U) {
            uint64_t key[NB_U], slot[NB_U];
            bool act[NB_U];
#pragma unroll
            for (int u = 0; u < NB_U; ++u) {
                const int o = o0 + u * 32 + lane;
                act[u] = o < noff;
                key[u] = 0;
                slot[u] = 0;
                if (act[u]) {
                    int nc[D], dl[D];
#pragma unroll
                    for (int j = 0; j < D; ++j) {
                        dl[j] = (int)offs[o * kMaxEnumDim + j];
                        nc[j] = cc[j] + dl[j];
                        act[u] = act[u] && nc[j] >= 0 && nc[j] <= P.kmax[j];
                    }
                    if (act[u]) {
                        if constexpr (D == 2 || D == 3) key[u] = morton_offset<D>(ckey, dl);
                        else key[u] = morton_encode(nc, D, P.bits);
                        slot[u] = hash_slot(key[u], lg);
                    }
                }
            }
            ulonglong2 e[NB_U];
#pragma unroll
            for (int u = 0; u < NB_U; ++u) e[u] = act[u] ? ht[slot[u]] : make_ulonglong2(kEmptyKey, 0);
#pragma unroll
            for (int u = 0; u < NB_U; ++u) {
                int h = -1;
                if (act[u]) {
                    uint64_t s = slot[u];
                    for (uint64_t it = 0; it <= mask; ++it) {
                        if (e[u].x == key[u]) { h = (int)e[u].y; break; }
                        if (e[u].x == kEmptyKey) break;
                        s = (s + 1) & mask;
                        e[u] = ht[s];
                    }
                    // drop cells whose points are all farther than eps from all of c's
                    if (h >= 0 && P.box && boxes_min_d2<D>(clo, chi, blo[h], bhi[h]) > P.hi) h = -1;
                }
                const unsigned bal = __ballot_sync(0xffffffffu, h >= 0);
                if (h >= 0) nbr[base + cnt + __popc(bal & lt)] = h;
                cnt += __popc(bal);
                const int o_first = o0 + u * 32;
                if (o_first < n_near)
                    near += __popc(bal & (n_near - o_first >= 32 ? 0xffffffffu : ((1u << (n_near - o_first)) - 1u)));
            }
        }
        if (lane == 0) { nbr_cnt[c] = cnt; nbr_near[c] = near; }
        total += cnt;
    }
    if (lane == 0 && total) atomicAdd((unsigned long long *)&ctr->E, (unsigned long long)total);
}

void launch_neighbors(const uint64_t *cell_key, const ulonglong2 *ht, const RunParams &P,
                      const signed char *offs, int noff, int n_near, const float4 *blo, const float4 *bhi,
                      int *nbr_cnt, int *nbr_near, int *nbr, DevCounters *ctr, cudaStream_t s) {
    auto go = [&](auto k) {
        int g = grid_for((const void *)k, 256);
        k<<<g, 256, 0, s>>>(cell_key, ht, P, offs, noff, n_near, blo, bhi, nbr_cnt, nbr_near, nbr, ctr);
        count_launch();
    };
    switch (P.d) {
    case 1: go(k_neighbors<1>); break;
    case 2: go(k_neighbors<2>); break;
    case 3: go(k_neighbors<3>); break;
    default: go(k_neighbors<4>); break;
    }
}

}  // namespace gbdb
