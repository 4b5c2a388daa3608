// Cells (Algorithm 1 line 2; Sec. 4.1 "Grid Computation"): bounding box,
// FP64 cell keys, grouping points by cell, the hash of non-empty cells and the
// cached neighbour-cell lists (Sec. 5.1 caches them per cell as well).
#include "geom.cuh"
#include "grid.cuh"

namespace gbdb {

// ---------------------------------------------------------------- bbox
constexpr int BB_THREADS = 256;

template <typename T>
__global__ void __launch_bounds__(BB_THREADS)
k_bbox(const T *__restrict__ X, int n, int d, double *__restrict__ part, int *__restrict__ bad) {
    __shared__ double smn[BB_THREADS / 32][kMaxDim], smx[BB_THREADS / 32][kMaxDim];
    double mn[kMaxDim], mx[kMaxDim];
#pragma unroll
    for (int j = 0; j < kMaxDim; ++j) { mn[j] = __longlong_as_double(0x7ff0000000000000ll); mx[j] = -mn[j]; }
    int nonfinite = 0;
    for (int i = blockIdx.x * BB_THREADS + threadIdx.x; i < n; i += gridDim.x * BB_THREADS) {
#pragma unroll
        for (int j = 0; j < kMaxDim; ++j) {
            if (j < d) {
                double x = (double)X[(int64_t)i * d + j];
                if (!isfinite(x)) nonfinite = 1;
                mn[j] = fmin(mn[j], x);
                mx[j] = fmax(mx[j], x);
            }
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < kMaxDim; ++j) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mn[j] = fmin(mn[j], __shfl_xor_sync(0xffffffffu, mn[j], o));
            mx[j] = fmax(mx[j], __shfl_xor_sync(0xffffffffu, mx[j], o));
        }
        if (lane == 0) { smn[warp][j] = mn[j]; smx[warp][j] = mx[j]; }
    }
    if (__any_sync(0xffffffffu, nonfinite) && lane == 0) atomicOr(bad, 1);
    __syncthreads();
    if (threadIdx.x < kMaxDim) {
        const int j = threadIdx.x;
        double a = smn[0][j], b = smx[0][j];
        for (int w = 1; w < BB_THREADS / 32; ++w) { a = fmin(a, smn[w][j]); b = fmax(b, smx[w][j]); }
        part[blockIdx.x * 2 * kMaxDim + j] = a;
        part[blockIdx.x * 2 * kMaxDim + kMaxDim + j] = b;
    }
}

// Reduce the per-block extremes: 256 threads stride over the blocks, then a
// warp-shuffle and shared-memory reduction per coordinate.
__global__ void __launch_bounds__(256) k_bbox_final(const double *__restrict__ part, int nb, const int *bad, double *out) {
    __shared__ double sh[8][2 * kMaxDim];
    double v[2 * kMaxDim];
#pragma unroll
    for (int j = 0; j < 2 * kMaxDim; ++j)
        v[j] = j < kMaxDim ? __longlong_as_double(0x7ff0000000000000ll) : __longlong_as_double(0xfff0000000000000ll);
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
#pragma unroll
        for (int j = 0; j < 2 * kMaxDim; ++j) {
            const double w = part[b * 2 * kMaxDim + j];
            v[j] = j < kMaxDim ? fmin(v[j], w) : fmax(v[j], w);
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < 2 * kMaxDim; ++j) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double w = __shfl_xor_sync(0xffffffffu, v[j], o);
            v[j] = j < kMaxDim ? fmin(v[j], w) : fmax(v[j], w);
        }
        if (lane == 0) sh[warp][j] = v[j];
    }
    __syncthreads();
    if (threadIdx.x < 2 * kMaxDim) {
        const int j = threadIdx.x;
        double r = sh[0][j];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = j < kMaxDim ? fmin(r, sh[w][j]) : fmax(r, sh[w][j]);
        out[j] = r;
    }
    if (threadIdx.x == 0) out[2 * kMaxDim] = (double)*bad;
}

void launch_bbox(const void *X, int dtype, int n, int d, double *part, int nb, int *bad,
                 double *out, cudaStream_t s) {
    if (dtype == DBSCAN_F32)
        k_bbox<float><<<nb, BB_THREADS, 0, s>>>((const float *)X, n, d, part, bad);
    else
        k_bbox<double><<<nb, BB_THREADS, 0, s>>>((const double *)X, n, d, part, bad);
    count_launch();
    k_bbox_final<<<1, 256, 0, s>>>(part, nb, bad, out); count_launch();
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
        keys[i] = morton_encode(c, P.d, P.bits);
        vals[i] = (uint32_t)i;
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
k_cell_flags(const uint64_t *__restrict__ K, int n, int *__restrict__ flags) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        flags[i] = (i == 0 || K[i] != K[i - 1]) ? 1 : 0;
}

// Gather the points into cell order, zero padded to the storage width, and
// record the cell table: cell_start[m+1], cell_key[m], cell_of[n], orig[n].
template <typename T, int SD>
__global__ void __launch_bounds__(256)
k_gather(const T *__restrict__ X, int n, int d, const uint64_t *__restrict__ K,
         const uint32_t *__restrict__ V, const int *__restrict__ flags, const int *__restrict__ cid,
         float *__restrict__ pf, double *__restrict__ pd, int *__restrict__ orig,
         int *__restrict__ cell_of, int *__restrict__ cell_start, uint64_t *__restrict__ cell_key,
         DevCounters *ctr) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int o = (int)V[i];
        const int c = cid[i] + flags[i] - 1;
        orig[i] = o;
        cell_of[i] = c;
        if (flags[i]) { cell_start[c] = i; cell_key[c] = K[i]; }
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
static void gather_sd(const void *X, int dtype, int n, int d, const uint64_t *K, const uint32_t *V,
                      const int *flags, const int *cid, float *pf, double *pd, int *orig, int *cell_of,
                      int *cell_start, uint64_t *cell_key, DevCounters *ctr, cudaStream_t s) {
    if (dtype == DBSCAN_F32) {
        int g = grid_for((const void *)k_gather<float, SD>, 256);
        k_gather<float, SD><<<g, 256, 0, s>>>((const float *)X, n, d, K, V, flags, cid, pf, nullptr, orig,
                                              cell_of, cell_start, cell_key, ctr); count_launch();
    } else {
        int g = grid_for((const void *)k_gather<double, SD>, 256);
        k_gather<double, SD><<<g, 256, 0, s>>>((const double *)X, n, d, K, V, flags, cid, pf, pd, orig,
                                               cell_of, cell_start, cell_key, ctr); count_launch();
    }
}

void launch_cells(const void *X, int dtype, int n, int d, int SD, const uint64_t *K, const uint32_t *V,
                  int *flags, int *cid, long long *part, float *pf, double *pd, int *orig,
                  int *cell_of, int *cell_start, uint64_t *cell_key, DevCounters *ctr, cudaStream_t s) {
    int g = grid_for((const void *)k_cell_flags, 256);
    k_cell_flags<<<g, 256, 0, s>>>(K, n, flags); count_launch();
    scan_i32_to_i32(flags, cid, n, nullptr, n, part, s);
    if (SD == 2)
        gather_sd<2>(X, dtype, n, d, K, V, flags, cid, pf, pd, orig, cell_of, cell_start, cell_key, ctr, s);
    else if (SD == 4)
        gather_sd<4>(X, dtype, n, d, K, V, flags, cid, pf, pd, orig, cell_of, cell_start, cell_key, ctr, s);
    else
        gather_sd<8>(X, dtype, n, d, K, V, flags, cid, pf, pd, orig, cell_of, cell_start, cell_key, ctr, s);
}

// ---------------------------------------------------------------- hash
__global__ void __launch_bounds__(256) k_hash_clear(uint64_t *__restrict__ hk, const DevCounters *ctr) {
    const uint64_t cap = hash_capacity(ctr->m);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < cap;
         i += (uint64_t)gridDim.x * blockDim.x)
        hk[i] = kEmptyKey;
}

__global__ void __launch_bounds__(256)
k_hash_insert(uint64_t *__restrict__ hk, int *__restrict__ hv, const uint64_t *__restrict__ cell_key,
              DevCounters *ctr) {
    const int m = ctr->m;
    const uint64_t mask = hash_capacity(m) - 1;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x) {
        const uint64_t key = cell_key[c];
        uint64_t s = hash_slot(key) & mask;
        bool done = false;
        for (uint64_t it = 0; it <= mask; ++it) {
            unsigned long long prev = atomicCAS((unsigned long long *)(hk + s), (unsigned long long)kEmptyKey,
                                                (unsigned long long)key);
            if (prev == kEmptyKey) { hv[s] = c; done = true; break; }
            s = (s + 1) & mask;
        }
        if (!done) set_error(ctr, DBSCAN_ERR_CAPACITY, 10);
    }
}

void launch_hash(uint64_t *hk, int *hv, const uint64_t *cell_key, DevCounters *ctr, cudaStream_t s) {
    int g = grid_for((const void *)k_hash_clear, 256);
    k_hash_clear<<<g, 256, 0, s>>>(hk, ctr); count_launch();
    g = grid_for((const void *)k_hash_insert, 256);
    k_hash_insert<<<g, 256, 0, s>>>(hk, hv, cell_key, ctr); count_launch();
}

// ---------------------------------------------------------------- neighbours
// NeighborCells(g) (Algorithm 2): every non-empty cell h != g whose integer
// offset delta from g satisfies sum_j max(|delta_j| - 1, 0)^2 <= d, looked up
// in the hash.  One warp per cell, one candidate offset per lane; the list
// keeps the offset-table order (nearest offsets first).
template <bool FILL>
__global__ void __launch_bounds__(256)
k_neighbors(const uint64_t *__restrict__ cell_key, const uint64_t *__restrict__ hk,
            const int *__restrict__ hv, RunParams P, const signed char *__restrict__ offs, int noff,
            long long *__restrict__ cnt_or_off,
            int *__restrict__ nbr, long long nbr_cap, DevCounters *ctr) {
    const int m = ctr->m;
    const uint64_t mask = hash_capacity(m) - 1;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    for (int c = warp_id_global(); c < m; c += warps_global()) {
        int cc[kMaxDim];
        morton_decode(cell_key[c], P.d, P.bits, cc);
        long long base = FILL ? cnt_or_off[c] : 0;
        int cnt = 0;
        for (int o0 = 0; o0 < noff; o0 += 32) {
            const int o = o0 + lane;
            int h = -1;
            if (o < noff) {
                int nc[kMaxDim];
                bool ok = true;
#pragma unroll
                for (int j = 0; j < kMaxEnumDim; ++j) {
                    if (j < P.d) {
                        nc[j] = cc[j] + (int)offs[o * kMaxEnumDim + j];
                        ok = ok && nc[j] >= 0 && nc[j] <= P.kmax[j];
                    }
                }
                if (ok) h = hash_find(hk, hv, morton_encode(nc, P.d, P.bits), mask);
            }
            const unsigned bal = __ballot_sync(0xffffffffu, h >= 0);
            if (FILL && h >= 0) {
                long long at = base + cnt + __popc(bal & lt);
                if (at < nbr_cap) nbr[at] = h;
                else set_error(ctr, DBSCAN_ERR_CAPACITY, 11);
            }
            cnt += __popc(bal);
        }
        if (!FILL && lane == 0) cnt_or_off[c] = cnt;
    }
}

__global__ void k_store_E(const long long *off, DevCounters *ctr) { ctr->E = off[ctr->m]; }

void launch_neighbors(const uint64_t *cell_key, const uint64_t *hk, const int *hv, const RunParams &P,
                      const signed char *offs, int noff, long long *cnt, long long *off, int *nbr, long long nbr_cap,
                      long long *part, int64_t n_max, DevCounters *ctr, cudaStream_t s) {
    int g = grid_for((const void *)k_neighbors<false>, 256);
    k_neighbors<false><<<g, 256, 0, s>>>(cell_key, hk, hv, P, offs, noff, cnt, nullptr, 0, ctr); count_launch();
    scan_i64_to_i64(cnt, off, 0, &ctr->m, n_max, part, s);
    k_store_E<<<1, 1, 0, s>>>(off, ctr); count_launch();
    k_neighbors<true><<<g, 256, 0, s>>>(cell_key, hk, hv, P, offs, noff, off, nbr, nbr_cap, ctr); count_launch();
}

}  // namespace gbdb
