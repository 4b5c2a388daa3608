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

// ------------------------------------------------------------ semisort
// Grouping the points by cell (Sec. 4.1): the paper semisorts (cell, point)
// pairs and keeps the non-empty cells in a hash table, since only grouping
// matters, not order.  Here each point computes its cell coordinates in FP64,
// k_j = floor(fl(fl(x_j - origin_j) * (1/s))), Morton-packs them, inserts the
// key into the cell hash (one slot per non-empty cell) and takes the next free
// position of its cell with an atomic increment.  Only the m distinct cell
// keys are then sorted, which lays the cells out along the Z-curve; the points
// are finally moved to their cell's range in one pass.  Slot = {key, cell id};
// the table is reset to empty after each run by k_table_reset, so a run only
// touches the slots it uses.
// Instance of input row i: the last instance whose first row is <= i.
__device__ __forceinline__ int inst_of_row(const RunParams &P, int i) {
    int lo = 0, hi = P.ninst - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (P.inst[mid].row0 <= i) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Cell key: Morton code of the cell coordinates, under the instance id when
// the run holds several instances.
__device__ __forceinline__ uint64_t cell_key_of(const RunParams &P, int inst, const int *c, int bits) {
    const uint64_t k = morton_encode(c, P.d, bits);
    return P.ninst > 1 ? (((uint64_t)inst << P.inst_shift) | k) : k;
}

// Grids with at least 8 points per cell on average take the offset
// enumeration of k_neighbors (nearest cells first, so MarkCore's early exit
// comes sooner); sparser ones the supercells.  Decided on the device, where m
// is known; the kernels of the other path return at once.
__device__ __forceinline__ bool grid_dense(long long n, int m) { return n >= 8ll * m; }

constexpr int INS_U = 4;  // points per thread per step (their probes overlap)

template <typename T>
__global__ void __launch_bounds__(256)
k_insert(const T *__restrict__ X, RunParams P, ulonglong2 *__restrict__ ht,
         uint64_t hmask, int hlg, uint32_t *__restrict__ slot_of, uint32_t *__restrict__ rank_of,
         uint32_t *__restrict__ slots, unsigned *__restrict__ bloom, int blg, DevCounters *ctr) {
    if (run_failed(ctr)) return;
    const int T_ = gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    // the loop bound is uniform across the warp (its first lane's index), so
    // the warp stays whole for the ballots below
    for (long long w0 = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); w0 < P.n;
         w0 += (long long)T_ * INS_U) {
        const long long i0 = w0 + lane;
        uint64_t key[INS_U], s[INS_U];
        unsigned long long cur[INS_U];
#pragma unroll
        for (int u = 0; u < INS_U; ++u) {
            const long long i = i0 + (long long)u * T_;
            key[u] = 0;
            s[u] = 0;
            // the instance of the row: lane 0 searches, the others step on from
            // its answer (a warp's 32 consecutive rows seldom cross an instance)
            int ib = 0;
            if (P.ninst > 1) {
                const long long r0 = w0 + (long long)u * T_;
                if (lane == 0 && r0 < P.n) ib = inst_of_row(P, (int)r0);
                ib = __shfl_sync(0xffffffffu, ib, 0);
            }
            if (i < P.n) {
                int ii = ib;
                while (ii + 1 < P.ninst && P.inst[ii + 1].row0 <= i) ++ii;
                const Inst &I = P.inst[ii];
                int c[kMaxDim];
#pragma unroll
                for (int j = 0; j < kMaxDim; ++j)
                    c[j] = j < I.d ? cell_coord<T>(X[i * P.d + j], I, j) : 0;
                key[u] = cell_key_of(P, ii, c, I.bits);
                s[u] = hash_slot(key[u], hlg);
            }
        }
#pragma unroll
        for (int u = 0; u < INS_U; ++u) cur[u] = i0 + (long long)u * T_ < P.n ? ht[s[u]].x : 0;
        // linear probing for the INS_U keys side by side: each step issues the
        // compare-and-swaps of all unresolved keys that see an empty slot
        // before it waits for any of them
        bool fresh[INS_U], done[INS_U];
#pragma unroll
        for (int u = 0; u < INS_U; ++u) {
            fresh[u] = false;
            done[u] = i0 + (long long)u * T_ >= P.n;
        }
        for (uint64_t it = 0;; ++it) {
            unsigned long long old[INS_U];
#pragma unroll
            for (int u = 0; u < INS_U; ++u)
                old[u] = (!done[u] && cur[u] == kEmptyKey)
                             ? atomicCAS(&ht[s[u]].x, (unsigned long long)kEmptyKey, (unsigned long long)key[u])
                             : cur[u];
            bool open = false;
#pragma unroll
            for (int u = 0; u < INS_U; ++u) {
                if (done[u]) continue;
                if (cur[u] == kEmptyKey && old[u] == kEmptyKey) {  // a new non-empty cell
                    fresh[u] = true;
                    done[u] = true;
                } else if (old[u] == key[u]) {
                    done[u] = true;
                } else if (it >= hmask) {  // the table is full
                    set_error(ctr, DBSCAN_ERR_CAPACITY, 10);
                    s[u] = ~0ull;
                    done[u] = true;
                } else {
                    s[u] = (s[u] + 1) & hmask;
                    cur[u] = ht[s[u]].x;
                    open = true;
                }
            }
            if (!open) break;
        }
        // the warp's new cells take consecutive places in the slot list with
        // one counter increment per step
        unsigned fm[INS_U];
        int nf = 0;
#pragma unroll
        for (int u = 0; u < INS_U; ++u) {
            fm[u] = __ballot_sync(0xffffffffu, fresh[u]);
            nf += __popc(fm[u]);
        }
        if (nf > 0) {
            int at = 0;
            if (lane == 0) at = atomicAdd(&ctr->m, nf);
            at = __shfl_sync(0xffffffffu, at, 0);
#pragma unroll
            for (int u = 0; u < INS_U; ++u) {
                if (fresh[u]) {
                    slots[at + __popc(fm[u] & ((1u << lane) - 1u))] = (uint32_t)s[u];
                    if (bloom) bloom_add(bloom, key[u], blg);
                }
                at += __popc(fm[u]);
            }
        }
        unsigned rk[INS_U];
#pragma unroll
        for (int u = 0; u < INS_U; ++u) {
            const long long i = i0 + (long long)u * T_;
            rk[u] = 0;
            if (i < P.n && s[u] != ~0ull) rk[u] = (unsigned)atomicAdd(&ht[s[u]].y, 1ull);  // the slot counts its points
        }
#pragma unroll
        for (int u = 0; u < INS_U; ++u) {
            const long long i = i0 + (long long)u * T_;
            if (i < P.n && s[u] != ~0ull) {
                slot_of[i] = (uint32_t)s[u];
                rank_of[i] = rk[u];
            }
        }
    }
}

// Sort input: (cell key, slot) of the m non-empty cells.
__global__ void __launch_bounds__(256)
k_cell_keys(const ulonglong2 *__restrict__ ht, const uint32_t *__restrict__ slots, uint64_t *__restrict__ keys,
            uint32_t *__restrict__ vals, const DevCounters *ctr) {
    if (run_failed(ctr)) return;
    const int m = ctr->m;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x) {
        const uint32_t s = slots[c];
        keys[c] = ht[s].x;
        vals[c] = s;
    }
}

// Cell c (in key order) owns slot vals[c]: record its key and its point count.
__global__ void __launch_bounds__(256)
k_cell_table(RunParams P, const uint64_t *__restrict__ keys, const uint32_t *__restrict__ vals,
             ulonglong2 *__restrict__ ht, uint64_t *__restrict__ cell_key,
             int *__restrict__ count, int *__restrict__ cell_inst, const DevCounters *ctr) {
    if (run_failed(ctr)) return;
    const int m = ctr->m;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x) {
        const uint32_t s = vals[c];
        count[c] = (int)ht[s].y;  // the points k_insert counted in the slot (k_slot_start rewrites it)
        cell_key[c] = keys[c];
        if (P.ninst > 1) cell_inst[c] = (int)(keys[c] >> P.inst_shift);
    }
}

// After the scan of the counts: slot value = cell id | first point << 32, so
// the scatter finds both with the one load of its slot.
__global__ void __launch_bounds__(256)
k_slot_start(const uint32_t *__restrict__ vals, const int *__restrict__ cell_start, ulonglong2 *__restrict__ ht,
             const DevCounters *ctr) {
    if (run_failed(ctr)) return;
    const int m = ctr->m;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x)
        ht[vals[c]].y = (unsigned long long)(unsigned)c | ((unsigned long long)(unsigned)cell_start[c] << 32);
}

constexpr int SC_U = 4;  // points per thread per step of the scatter (their loads overlap)

// Move every point to its cell's range: coalesced reads of the input, one
// scattered write per point.  Points are stored zero padded to SD coordinates.
template <typename T, int SD>
__global__ void __launch_bounds__(256)
k_scatter_points(const T *__restrict__ X, RunParams P, const ulonglong2 *__restrict__ ht,
                 const uint32_t *__restrict__ slot_of, const uint32_t *__restrict__ rank_of,
                 const int *__restrict__ cell_start, float *__restrict__ pf, double *__restrict__ pd,
                 int *__restrict__ orig, int *__restrict__ cell_of, const DevCounters *ctr) {
    if (run_failed(ctr)) return;
    const int n = P.n, ld = P.d;
    const int T_ = gridDim.x * blockDim.x;
    for (long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += (long long)T_ * SC_U) {
        unsigned long long e[SC_U];
#pragma unroll
        for (int u = 0; u < SC_U; ++u) {
            const long long i = i0 + (long long)u * T_;
            e[u] = i < n ? ht[slot_of[i]].y : 0ull;
        }
#pragma unroll
        for (int u = 0; u < SC_U; ++u) {
            const long long i = i0 + (long long)u * T_;
            if (i >= n) break;
            const int c = (int)(unsigned)e[u];
            const int dst = (int)(e[u] >> 32) + (int)rank_of[i];
            // coordinates beyond the instance's own dimension are stored as zero
            const int d = P.ninst > 1 ? P.inst[P.cell_inst[c]].d : ld;
            orig[dst] = (int)i;
            cell_of[dst] = c;
            float f[SD];
            double x[SD];
#pragma unroll
            for (int j = 0; j < SD; ++j) {
                x[j] = j < d ? (double)X[i * ld + j] : 0.0;
                f[j] = (float)x[j];
            }
            if constexpr (SD == 2) {
                reinterpret_cast<float2 *>(pf)[dst] = make_float2(f[0], f[1]);
            } else {
#pragma unroll
                for (int j = 0; j < SD; j += 4)
                    reinterpret_cast<float4 *>(pf)[(int64_t)dst * (SD / 4) + j / 4] =
                        make_float4(f[j], f[j + 1], f[j + 2], f[j + 3]);
            }
            if (pd) {
#pragma unroll
                for (int j = 0; j < SD; j += 2)
                    reinterpret_cast<double2 *>(pd)[(int64_t)dst * (SD / 2) + j / 2] = make_double2(x[j], x[j + 1]);
            }
        }
    }
}

// Return the slots this run used to empty.
__global__ void __launch_bounds__(256)
k_table_reset(ulonglong2 *__restrict__ ht, const uint32_t *__restrict__ slots,
              const DevCounters *ctr, int n, int cond) {
    if (run_failed(ctr)) return;
    const int m = ctr->m;
    // cond 1: only on a sparse grid (before its supercells take the table);
    // cond 2: only on a dense grid (its cells kept the table to the end)
    if (cond && (cond == 2) != grid_dense(n, m)) return;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x) {
        const uint32_t s = slots[c];
        ht[s] = make_ulonglong2(kEmptyKey, 0);
    }
}

// Every slot of the cell hash empty: {kEmptyKey, 0} (a slot's second word
// counts its points during the insert, then holds the cell id).
__global__ void __launch_bounds__(256) k_table_clear(ulonglong2 *__restrict__ ht, uint64_t cap) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < cap; i += (uint64_t)gridDim.x * blockDim.x)
        ht[i] = make_ulonglong2(kEmptyKey, 0);
}

void launch_table_clear(ulonglong2 *ht, uint64_t cap, cudaStream_t s) {
    const int g = grid_for((const void *)k_table_clear, 256);
    k_table_clear<<<g, 256, 0, s>>>(ht, cap);
    count_launch();
}

void launch_semisort(const void *X, int dtype, const RunParams &P, int SD, const Semisort &S, DevCounters *ctr,
                     cudaStream_t s) {
    const int lg = hash_log2(S.hcap);
    const uint64_t hmask = S.hcap - 1;
    if (dtype == DBSCAN_F32) {
        int g = grid_for((const void *)k_insert<float>, 256);
        k_insert<float><<<g, 256, 0, s>>>((const float *)X, P, S.ht, hmask, lg, S.slot_of, S.rank_of,
                                          S.slots, S.bloom, S.bloom_lg, ctr);
    } else {
        int g = grid_for((const void *)k_insert<double>, 256);
        k_insert<double><<<g, 256, 0, s>>>((const double *)X, P, S.ht, hmask, lg, S.slot_of, S.rank_of,
                                           S.slots, S.bloom, S.bloom_lg, ctr);
    }
    count_launch();
    int g = grid_for((const void *)k_cell_keys, 256);
    k_cell_keys<<<g, 256, 0, s>>>(S.ht, S.slots, S.k0, S.v0, ctr); count_launch();
    const int which = radix_sort_u64(S.k0, S.v0, S.k1, S.v1, 0, &ctr->m, P.n, S.key_lo, S.key_bits, S.sort_scratch,
                                     S.sort_scratch_size, ctr, P.max_iters, s);
    const uint64_t *K = which ? S.k1 : S.k0;
    const uint32_t *V = which ? S.v1 : S.v0;
    g = grid_for((const void *)k_cell_table, 256);
    k_cell_table<<<g, 256, 0, s>>>(P, K, V, S.ht, S.cell_key, S.count, S.cell_inst, ctr); count_launch();
    scan_i32_to_i32(S.count, S.cell_start, 0, &ctr->m, P.n, S.part, s);
    g = grid_for((const void *)k_slot_start, 256);
    k_slot_start<<<g, 256, 0, s>>>(V, S.cell_start, S.ht, ctr); count_launch();
    auto scat = [&](auto k, auto xp) {
        int gg = grid_for((const void *)k, 256);
        k<<<gg, 256, 0, s>>>(xp, P, S.ht, S.slot_of, S.rank_of, S.cell_start, S.pf, S.pd, S.orig, S.cell_of, ctr);
        count_launch();
    };
    const float *xf = (const float *)X;
    const double *xd = (const double *)X;
    if (dtype == DBSCAN_F32) {
        if (SD == 2) scat(k_scatter_points<float, 2>, xf);
        else if (SD == 4) scat(k_scatter_points<float, 4>, xf);
        else scat(k_scatter_points<float, 8>, xf);
    } else {
        if (SD == 2) scat(k_scatter_points<double, 2>, xd);
        else if (SD == 4) scat(k_scatter_points<double, 4>, xd);
        else scat(k_scatter_points<double, 8>, xd);
    }
}

// Empty the supercell slots (the cells' slots were emptied before).
__global__ void __launch_bounds__(256)
k_super_reset(ulonglong2 *__restrict__ ht, const uint32_t *__restrict__ sslots, const DevCounters *ctr) {
    if (run_failed(ctr)) return;
    const int ms = ctr->ms;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ms; i += gridDim.x * blockDim.x)
        ht[sslots[i]] = make_ulonglong2(kEmptyKey, 0);
}

void launch_table_reset(const Semisort &S, DevCounters *ctr, cudaStream_t s, bool end_of_run) {
    if (end_of_run && S.super) {  // the supercells' slots (none on a dense grid), or the cells' on a dense grid
        const int g = grid_for((const void *)k_super_reset, 256);
        k_super_reset<<<g, 256, 0, s>>>(S.ht, S.slots, ctr);
        count_launch();
    }
    const int cond = S.super ? (end_of_run ? 2 : 1) : 0;
    int g = grid_for((const void *)k_table_reset, 256);
    k_table_reset<<<g, 256, 0, s>>>(S.ht, S.slots, ctr, S.n, cond); count_launch();
}

// ---------------------------------------------------------------- boxes
// Per-cell FP32 bounding box of the points pts[start[c] .. start[c+1]) (exact
// min/max of the stored FP32 coordinates), and optionally their centroid.
// With many more cells than warps, a warp takes 32 consecutive cells: a lane
// reduces its own cell when it holds at most kBoxSmall points (the loads of
// neighbouring lanes are then nearly contiguous), and the warp reduces the
// larger cells together, one at a time.  With fewer cells, every cell gets a
// warp of its own.  Boxes hold BW = SD/4 float4 values per cell (at least one;
// coordinates past the stored width are zero).  Empty ranges get an empty box
// (+inf, -inf).
constexpr int kBoxSmall = 8;

template <int SD, int W>
__device__ __forceinline__ void box_point(const float *__restrict__ pts, int t, float (&x)[W]) {
    constexpr int BW = W / 4;
#pragma unroll
    for (int j = 0; j < W; ++j) x[j] = 0.f;
    if constexpr (SD == 2) {
        const float2 a = reinterpret_cast<const float2 *>(pts)[t];
        x[0] = a.x;
        x[1] = a.y;
    } else {
#pragma unroll
        for (int b = 0; b < BW; ++b) {
            const float4 a = reinterpret_cast<const float4 *>(pts)[(int64_t)t * BW + b];
            x[4 * b] = a.x; x[4 * b + 1] = a.y; x[4 * b + 2] = a.z; x[4 * b + 3] = a.w;
        }
    }
}

template <int W>
__device__ __forceinline__ void box_store(int c, int npts, const float (&l)[W], const float (&h)[W],
                                          const float (&sm)[W], int b, float4 *__restrict__ lo,
                                          float4 *__restrict__ hi, float4 *__restrict__ cent) {
    constexpr int BW = W / 4;
    lo[(int64_t)c * BW + b] = make_float4(l[4 * b], l[4 * b + 1], l[4 * b + 2], l[4 * b + 3]);
    hi[(int64_t)c * BW + b] = make_float4(h[4 * b], h[4 * b + 1], h[4 * b + 2], h[4 * b + 3]);
    if (cent) {
        const float inv = npts > 0 ? 1.f / (float)npts : 0.f;
        cent[(int64_t)c * BW + b] =
            make_float4(sm[4 * b] * inv, sm[4 * b + 1] * inv, sm[4 * b + 2] * inv, sm[4 * b + 3] * inv);
    }
}

template <int SD>
__global__ void __launch_bounds__(256)
k_boxes(const float *__restrict__ pts, const int *__restrict__ start, const DevCounters *ctr,
        float4 *__restrict__ lo, float4 *__restrict__ hi, float4 *__restrict__ cent) {
    if (run_failed(ctr)) return;
    constexpr int W = SD == 8 ? 8 : 4, BW = W / 4;
    const int m = ctr->m;
    const int lane = threadIdx.x & 31;
    // cells per warp work item: 32 (lane-wise small cells) or 1
    const int chunk = (long long)m >= 32ll * warps_global() ? 32 : 1;
    for (long long c0 = (long long)warp_id_global() * chunk; c0 < m; c0 += (long long)warps_global() * chunk) {
        const bool own = lane < chunk && c0 + lane < m;
        const int c = own ? (int)(c0 + lane) : 0;
        int s0 = 0, s1 = 0;
        if (own) { s0 = start[c]; s1 = start[c + 1]; }
        const bool small = chunk == 32 && own && s1 - s0 <= kBoxSmall;
        if (small) {
            float l[W], h[W], sm[W];
#pragma unroll
            for (int j = 0; j < W; ++j) { l[j] = INFINITY; h[j] = -INFINITY; sm[j] = 0.f; }
            for (int t = s0; t < s1; ++t) {
                float x[W];
                box_point<SD, W>(pts, t, x);
#pragma unroll
                for (int j = 0; j < W; ++j) { l[j] = fminf(l[j], x[j]); h[j] = fmaxf(h[j], x[j]); sm[j] += x[j]; }
            }
#pragma unroll
            for (int b = 0; b < BW; ++b) box_store<W>(c, s1 - s0, l, h, sm, b, lo, hi, cent);
        }
        for (unsigned big = __ballot_sync(0xffffffffu, own && !small); big; big &= big - 1) {
            const int src = __ffs(big) - 1;
            const int cb = (int)(c0 + src);
            const int b0 = __shfl_sync(0xffffffffu, s0, src), b1 = __shfl_sync(0xffffffffu, s1, src);
            float l[W], h[W], sm[W];
#pragma unroll
            for (int j = 0; j < W; ++j) { l[j] = INFINITY; h[j] = -INFINITY; sm[j] = 0.f; }
            for (int t = b0 + lane; t < b1; t += 32) {
                float x[W];
                box_point<SD, W>(pts, t, x);
#pragma unroll
                for (int j = 0; j < W; ++j) { l[j] = fminf(l[j], x[j]); h[j] = fmaxf(h[j], x[j]); sm[j] += x[j]; }
            }
#pragma unroll
            for (int j = 0; j < W; ++j) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    l[j] = fminf(l[j], __shfl_xor_sync(0xffffffffu, l[j], o));
                    h[j] = fmaxf(h[j], __shfl_xor_sync(0xffffffffu, h[j], o));
                    if (cent) sm[j] += __shfl_xor_sync(0xffffffffu, sm[j], o);
                }
            }
            if (lane < BW) box_store<W>(cb, b1 - b0, l, h, sm, lane, lo, hi, cent);
        }
    }
}

void launch_boxes(int SD, const float *pts, const int *start, const DevCounters *ctr, float4 *lo, float4 *hi,
                  cudaStream_t s, float4 *cent) {
    auto go = [&](auto k) {
        const int g = grid_for((const void *)k, 256);
        k<<<g, 256, 0, s>>>(pts, start, ctr, lo, hi, cent);
        count_launch();
    };
    if (SD == 2) go(k_boxes<2>);
    else if (SD == 4) go(k_boxes<4>);
    else go(k_boxes<8>);
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
k_neighbors(const uint64_t *__restrict__ cell_key, const ulonglong2 *__restrict__ ht, uint64_t mask, int lg,
            const unsigned *__restrict__ bloom, int blg, const int *__restrict__ cell_start,
            int *__restrict__ nbr_pts,
            RunParams P,
            const signed char *__restrict__ offs, int noff, int n_near, const float4 *__restrict__ blo,
            const float4 *__restrict__ bhi, int *__restrict__ nbr_cnt, int *__restrict__ nbr_near,
            int *__restrict__ nbr, int only_dense, DevCounters *ctr) {
    if (run_failed(ctr)) return;
    const int m = ctr->m;
    if (only_dense && !grid_dense(P.n, m)) return;  // k_neighbors_super takes sparse grids
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    long long total = 0;
    for (int c = warp_id_global(); c < m; c += warps_global()) {
        const int ii = inst_of_cell(P, c);
        const Inst &I = P.inst[ii];
        const uint64_t ibits = P.ninst > 1 ? ((uint64_t)ii << P.inst_shift) : 0;
        const uint64_t ckey = cell_key[c] ^ ibits;  // Morton part
        int cc[D];
        {
            int tmp[kMaxDim];
            morton_decode(ckey, D, I.bits, tmp);
#pragma unroll
            for (int j = 0; j < D; ++j) cc[j] = tmp[j];
        }
        const long long base = (long long)c * noff;
        Bx<D> clo = zero_box<D>(), chi = clo;
        if (P.box) { clo = load_box<D>(blo, c); chi = load_box<D>(bhi, c); }
        // the wider of the two thresholds (rho-approximate connectivity keeps
        // the cell pairs within eps(1 + rho); MarkCore and border test at eps)
        const float hi_thr = I.cthr.hi;
        int cnt = 0, near = 0, pts = 0;
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
                        act[u] = act[u] && nc[j] >= 0 && nc[j] <= I.kmax[j];
                    }
                    if (act[u]) {
                        if constexpr (D == 2 || D == 3) key[u] = morton_offset<D>(ckey, dl) | ibits;
                        else key[u] = morton_encode(nc, D, I.bits) | ibits;
                        if (bloom) act[u] = bloom_may_have(bloom, key[u], blg);  // most offsets hold no cell
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
                        if (e[u].x == key[u]) { h = (int)(unsigned)e[u].y; break; }  // low word: the cell id
                        if (e[u].x == kEmptyKey) break;
                        s = (s + 1) & mask;
                        e[u] = ht[s];
                    }
                    // drop cells whose points are all farther than eps (eps(1 + rho)) from all of c's
                    if (h >= 0 && P.box && boxes_min_d2<D>(clo, chi, load_box<D>(blo, h), load_box<D>(bhi, h)) > hi_thr)
                        h = -1;
                }
                const unsigned bal = __ballot_sync(0xffffffffu, h >= 0);
                if (h >= 0) {
                    nbr[base + cnt + __popc(bal & lt)] = h;
                    if (nbr_pts) pts += cell_start[h + 1] - cell_start[h];
                }
                cnt += __popc(bal);
                const int o_first = o0 + u * 32;
                if (o_first < n_near)
                    near += __popc(bal & (n_near - o_first >= 32 ? 0xffffffffu : ((1u << (n_near - o_first)) - 1u)));
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) pts += __shfl_xor_sync(0xffffffffu, pts, o);
        if (lane == 0) {
            nbr_cnt[c] = cnt;
            nbr_near[c] = near;
            if (nbr_pts) nbr_pts[c] = pts;
        }
        total += cnt;
    }
    if (lane == 0 && total) atomicAdd((unsigned long long *)&ctr->E, (unsigned long long)total);
}

// ------------------------------------------------------- neighbours, d = 2, 3
// NeighborCells(g) through supercells.  A supercell is a block of 2^D cells
// whose coordinates agree after >> 1; its key is the cell key without its
// lowest D bits (sk = key >> D), so in Z order its cells are consecutive (the
// cell sort orders every bit above the lowest D).  The candidate cells of any
// cell of supercell S (|delta_j| <= 2, the offset rule) lie in the 3^D
// supercells S + {-1, 0, 1}^D, so one warp per supercell probes those 3^D
// supercells once in a hash of the non-empty supercells (sk -> first cell and
// cell count), gathers their cells (at most 3^D * 2^D) and applies the exact
// offset rule, sum_j max(|delta_j| - 1, 0)^2 <= d, and the box test to every
// pair of an own cell and a candidate.  That is 9 (2D) or 27 (3D) probes per
// supercell instead of 24 or 124 per cell.  The supercell hash takes the first
// 2^ceil(log2 2 ms) slots of the cell hash table, whose cells' slots are
// emptied first (the cells need no hash once they are grouped); a Bloom filter
// of the supercell keys (8 bits per cell) keeps the probes of empty supercells
// in L2 when that table does not fit there.
__host__ __device__ __forceinline__ int super_bloom_lg(int m, int bloom_lg) {
    const uint64_t cap = hash_capacity(m);  // bounds the supercell table (ms <= m)
    if (cap * 16 <= (64ull << 20)) return -1;
    const int lg = hash_log2(cap) + 2;
    return lg < bloom_lg ? lg : bloom_lg;
}

// flag[c] = 1 iff cell c is the first of its supercell; clears the Bloom
// filter of the supercell keys.
template <int D>
__global__ void __launch_bounds__(256)
k_super_flags(const uint64_t *__restrict__ cell_key, int *__restrict__ flag, unsigned *__restrict__ bloom,
              int bloom_lg, const RunParams P, const DevCounters *ctr) {
    if (run_failed(ctr)) return;
    const int m = ctr->m;
    if (grid_dense(P.n, m)) return;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    for (long long c = t0; c < m; c += stride)
        flag[c] = (c == 0 || (cell_key[c] >> D) != (cell_key[c - 1] >> D)) ? 1 : 0;
    const int blg = super_bloom_lg(m, bloom_lg);
    if (blg > 0)
        for (long long w = t0; w < (1ll << (blg - 5)); w += stride) bloom[w] = 0u;
}

// pos = exclusive scan of the flags (pos[m] = ms supercells).  Each supercell
// enters the hash with value (first cell | cell count << 32); its first cell
// goes to sc_first[pos] and its slot to sslots[pos] (for the reset).
template <int D>
__global__ void __launch_bounds__(256)
k_super_insert(const uint64_t *__restrict__ cell_key, const int *__restrict__ pos, ulonglong2 *__restrict__ ht,
               uint32_t *__restrict__ sslots, int *__restrict__ sc_first, unsigned *__restrict__ bloom, int bloom_lg,
               const RunParams P, DevCounters *ctr) {
    if (run_failed(ctr)) return;
    const int m = ctr->m;
    if (grid_dense(P.n, m)) return;
    const int ms = pos[m];
    if (blockIdx.x == 0 && threadIdx.x == 0) ctr->ms = ms;
    const uint64_t cap = hash_capacity(ms);
    const int lg = hash_log2(cap);
    const uint64_t mask = cap - 1;
    const int blg = super_bloom_lg(m, bloom_lg);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x) {
        const int p = pos[c];
        if (pos[c + 1] == p) continue;  // not the first cell of its supercell
        int k = 1;
        while (c + k < m && k < (1 << D) && pos[c + k + 1] == pos[c + k]) ++k;
        const uint64_t sk = cell_key[c] >> D;
        sc_first[p] = c;
        uint64_t s = hash_slot(sk, lg);
        bool ok = false;
        for (uint64_t it = 0; it <= mask; ++it) {
            if (ht[s].x == kEmptyKey &&
                atomicCAS(&ht[s].x, (unsigned long long)kEmptyKey, (unsigned long long)sk) == kEmptyKey) {
                ht[s].y = (unsigned long long)(unsigned)c | ((unsigned long long)k << 32);
                ok = true;
                break;
            }
            s = (s + 1) & mask;
        }
        if (!ok) {
            set_error(ctr, DBSCAN_ERR_CAPACITY, 12);
            s = 0;
        }
        sslots[p] = (uint32_t)s;
        if (blg > 0) bloom_add(bloom, sk, blg);
    }
}

constexpr int NBS_WARPS = 8;  // warps per block of k_neighbors_super

// One warp per supercell S of a sparse grid.  Lane t < 3^D probes supercell
// S + o(t) (o: the base-3 digits of t minus 1).  A candidate cell h of that
// supercell has its coordinates, relative to S's first corner, at
// 2 o + q(h), where q(h) are the lowest D bits of its key (one bit per
// dimension); an own cell c sits at p(c), its own lowest bits, so the offset
// is delta = 2 o + q(h) - p(c) without decoding any key.  Every candidate
// coordinate differs by at most 3 per dimension, and the offset rule
// sum_j max(|delta_j| - 1, 0)^2 <= d holds iff |delta_j| <= 2 in every
// dimension (a coordinate at 2 adds 1; only the instance's own d
// coordinates can differ).  Each candidate (a lane) tests all own cells;
// the 2-bit outcomes (adjacent, farther, none) of own cell i sit in bits
// 2i, 2i+1 of a register per 32-candidate chunk, and the lists are written
// adjacent cells first, from two ballots per chunk.
template <int D>
__global__ void __launch_bounds__(32 * NBS_WARPS, 5)  // 51 registers: 5 blocks (40 warps) per SM (measured faster than 4)
k_neighbors_super(const uint64_t *__restrict__ cell_key, const ulonglong2 *__restrict__ ht,
                  const unsigned *__restrict__ bloom, int bloom_lg, const int *__restrict__ sc_first,
                  const int *__restrict__ cell_start, int *__restrict__ nbr_pts, RunParams P, int stride,
                  const float4 *__restrict__ blo, const float4 *__restrict__ bhi, int *__restrict__ nbr_cnt,
                  int *__restrict__ nbr_near, int *__restrict__ nbr, DevCounters *ctr) {
    if (run_failed(ctr)) return;
    constexpr int K = 1 << D;              // cells per supercell
    constexpr int NS = D == 2 ? 9 : 27;    // supercells probed, the own one included
    constexpr int CH = (NS * K + 31) / 32; // 32-candidate chunks
    constexpr uint64_t QMASK = (1u << D) - 1u;
    __shared__ float4 s_lo[NBS_WARPS][K], s_hi[NBS_WARPS][K];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int m = ctr->m, ms = ctr->ms;
    if (grid_dense(P.n, m)) return;  // k_neighbors takes dense grids
    const uint64_t cap = hash_capacity(ms);
    const int lg = hash_log2(cap);
    const uint64_t mask = cap - 1;
    const int blg = super_bloom_lg(m, bloom_lg);
    // this lane's probe offset o(lane) + 1, 2 bits per dimension
    unsigned odig = 0;
    {
        int t = lane;
#pragma unroll
        for (int j = 0; j < D; ++j) {
            odig |= (unsigned)(t % 3) << (2 * j);
            t /= 3;
        }
    }
    long long total = 0;
    for (int si = warp_id_global(); si < ms; si += warps_global()) {
        const int c0 = sc_first[si];
        int k = (si + 1 < ms ? sc_first[si + 1] : m) - c0;
        if (k > K || k < 1) {  // cannot happen for a sorted cell table
            if (lane == 0) set_error(ctr, DBSCAN_ERR_CAPACITY, 13);
            k = k < 1 ? 0 : K;
        }
        const int ii = inst_of_cell(P, c0);
        const Inst &I = P.inst[ii];
        const uint64_t ibits = P.ninst > 1 ? ((uint64_t)ii << P.inst_shift) : 0;
        const uint64_t key0 = cell_key[c0] ^ ibits;
        // own cells: boxes to shared memory, the D-bit positions p(c) packed
        // D bits per cell into pown (warp-uniform)
        __syncwarp();
        unsigned pmine = 0;
        if (lane < k) {
            pmine = (unsigned)(cell_key[c0 + lane] & QMASK);
            if (P.box) {
                s_lo[w][lane] = blo[c0 + lane];
                s_hi[w][lane] = bhi[c0 + lane];
            }
        }
        const unsigned pown = __reduce_or_sync(0xffffffffu, lane < k ? pmine << (D * lane) : 0u);
        __syncwarp();
        // the supercell's coordinates, for the bounds of the probes
        int sc[kMaxDim];
        morton_decode(key0 >> D, D, I.bits > 1 ? I.bits - 1 : 1, sc);
        const uint64_t skey = key0 >> D;
        int t0 = 0, kt = 0;
        if (lane < NS && k > 0) {
            int o[D];
            bool in = true;
#pragma unroll
            for (int j = 0; j < D; ++j) {
                o[j] = (int)((odig >> (2 * j)) & 3u) - 1;
                const int v = sc[j] + o[j];
                in = in && v >= 0 && v <= (I.kmax[j] >> 1);
            }
            if (in) {
                const uint64_t key = morton_offset<D>(skey, o) | (ibits >> D);
                if (blg <= 0 || bloom_may_have(bloom, key, blg)) {
                    uint64_t s = hash_slot(key, lg);
                    for (uint64_t it = 0; it <= mask; ++it) {
                        const ulonglong2 e = ht[s];
                        if (e.x == key) {
                            t0 = (int)(unsigned)(e.y & 0xffffffffu);
                            kt = (int)(e.y >> 32);
                            break;
                        }
                        if (e.x == kEmptyKey) break;
                        s = (s + 1) & mask;
                    }
                }
            }
        }
        // the candidates, flattened over the lanes in probe order
        int incl = kt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        const int excl = incl - kt;
        const int ncand = __shfl_sync(0xffffffffu, incl, 31);
        const int nch = (ncand + 31) >> 5;
        const float hi_thr = I.cthr.hi;  // eps, or eps(1 + rho) for approximate connectivity
        int hreg[CH];
        unsigned cls[CH];  // 2 bits per own cell: 1 adjacent, 2 farther, 0 not a neighbour
#pragma unroll
        for (int ch = 0; ch < CH; ++ch) {
            hreg[ch] = -1;
            cls[ch] = 0u;
            if (ch >= nch) continue;
            const int f = ch * 32 + lane;
            int j = 0;  // owner lane: the last lane whose range starts at or before f
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int ex = __shfl_sync(0xffffffffu, excl, (j + step) & 31);
                if (j + step < 32 && ex <= f) j += step;
            }
            const int h = __shfl_sync(0xffffffffu, t0, j) + f - __shfl_sync(0xffffffffu, excl, j);
            const unsigned oj = __shfl_sync(0xffffffffu, odig, j);
            if (f >= ncand) continue;
            hreg[ch] = h;
            const unsigned q = (unsigned)(cell_key[h] & QMASK);
            int rel[D];  // 2 o + q, per dimension (o from the owner lane j)
            {
#pragma unroll
                for (int jj = 0; jj < D; ++jj) rel[jj] = 2 * ((int)((oj >> (2 * jj)) & 3u) - 1) + (int)((q >> jj) & 1u);
            }
            Bx<D> bl, bh;
            if (P.box) {
                bl.v[0] = blo[h];
                bh.v[0] = bhi[h];
            }
            unsigned c = 0u;
            for (int i = 0; i < k; ++i) {
                if (h == c0 + i) continue;
                const unsigned pi = (pown >> (D * i)) & (unsigned)QMASK;
                int amax = 0;
#pragma unroll
                for (int jj = 0; jj < D; ++jj) amax = max(amax, abs(rel[jj] - (int)((pi >> jj) & 1u)));
                if (amax > 2) continue;
                if (P.box) {
                    Bx<D> al, ah;
                    al.v[0] = s_lo[w][i];
                    ah.v[0] = s_hi[w][i];
                    if (boxes_min_d2<D>(al, ah, bl, bh) > hi_thr) continue;
                }
                c |= (amax <= 1 ? 1u : 2u) << (2 * i);
            }
            cls[ch] = c;
        }
        // the lists: adjacent cells first, then the farther ones
        for (int i = 0; i < k; ++i) {
            int nn = 0, nf = 0;
#pragma unroll
            for (int ch = 0; ch < CH; ++ch) {
                if (ch >= nch) break;
                const unsigned code = (cls[ch] >> (2 * i)) & 3u;
                nn += __popc(__ballot_sync(0xffffffffu, code == 1u));
                nf += __popc(__ballot_sync(0xffffffffu, code == 2u));
            }
            if (lane == 0) {
                nbr_cnt[c0 + i] = nn + nf;
                nbr_near[c0 + i] = nn;
                total += nn + nf;
            }
            const long long base = (long long)(c0 + i) * stride;
            int ncur = 0, fcur = nn, pts = 0;
#pragma unroll
            for (int ch = 0; ch < CH; ++ch) {
                if (ch >= nch) break;
                const unsigned code = (cls[ch] >> (2 * i)) & 3u;
                const unsigned nb = __ballot_sync(0xffffffffu, code == 1u);
                const unsigned fb = __ballot_sync(0xffffffffu, code == 2u);
                if (code == 1u) nbr[base + ncur + __popc(nb & lt)] = hreg[ch];
                else if (code == 2u) nbr[base + fcur + __popc(fb & lt)] = hreg[ch];
                if (nbr_pts && code) pts += cell_start[hreg[ch] + 1] - cell_start[hreg[ch]];
                ncur += __popc(nb);
                fcur += __popc(fb);
            }
            if (nbr_pts) {
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) pts += __shfl_xor_sync(0xffffffffu, pts, o);
                if (lane == 0) nbr_pts[c0 + i] = pts;
            }
        }
    }
    if (lane == 0 && total) atomicAdd((unsigned long long *)&ctr->E, (unsigned long long)total);
}

void launch_super_table(const Semisort &S, const RunParams &P, DevCounters *ctr, cudaStream_t s) {
    // the cells' slots are free again: the supercells take the table
    launch_table_reset(S, ctr, s, false);
    int *pos = S.count;  // [m + 1], scratch until the compaction
    int *sc_first = reinterpret_cast<int *>(S.rank_of);  // free once the points are scattered
    auto go = [&](auto kf, auto ki) {
        int g = grid_for((const void *)kf, 256);
        kf<<<g, 256, 0, s>>>(S.cell_key, pos, S.bloom_all, S.bloom_lg, P, ctr);
        count_launch();
        scan_i32_to_i32(pos, pos, 0, &ctr->m, P.n, S.part, s);
        g = grid_for((const void *)ki, 256);
        ki<<<g, 256, 0, s>>>(S.cell_key, pos, S.ht, S.slots, sc_first, S.bloom_all, S.bloom_lg, P, ctr);
        count_launch();
    };
    if (P.d == 2) go(k_super_flags<2>, k_super_insert<2>);
    else go(k_super_flags<3>, k_super_insert<3>);
}

void launch_neighbors_super(const Semisort &S, const RunParams &P, int stride, const float4 *blo,
                            const float4 *bhi, const int *cell_start, int *nbr_cnt, int *nbr_near, int *nbr_pts,
                            int *nbr, DevCounters *ctr, cudaStream_t s) {
    const int *sc_first = reinterpret_cast<const int *>(S.rank_of);
    auto go = [&](auto kn) {
        const int g = grid_for((const void *)kn, 32 * NBS_WARPS);
        kn<<<g, 32 * NBS_WARPS, 0, s>>>(S.cell_key, S.ht, S.bloom_all, S.bloom_lg, sc_first, cell_start, nbr_pts, P,
                                        stride, blo, bhi, nbr_cnt, nbr_near, nbr, ctr);
        count_launch();
    };
    if (P.d == 2) go(k_neighbors_super<2>);
    else go(k_neighbors_super<3>);
}

void launch_neighbors(const uint64_t *cell_key, const ulonglong2 *ht, uint64_t hcap, const unsigned *bloom,
                      int bloom_lg, const RunParams &P, const signed char *offs, int noff, int n_near,
                      const float4 *blo, const float4 *bhi, const int *cell_start, int *nbr_cnt, int *nbr_near,
                      int *nbr_pts, int *nbr, DevCounters *ctr, cudaStream_t s, bool only_dense) {
    const uint64_t mask = hcap - 1;
    const int lg = hash_log2(hcap);
    auto go = [&](auto k) {
        int g = grid_for((const void *)k, 256);
        k<<<g, 256, 0, s>>>(cell_key, ht, mask, lg, bloom, bloom_lg, cell_start, nbr_pts, P, offs, noff, n_near,
                            blo, bhi, nbr_cnt, nbr_near, nbr, only_dense ? 1 : 0, ctr);
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
