// MarkCore (Algorithm 2), ClusterCore (Algorithm 3) and ClusterBorder
// (Algorithm 4) on the cell structure built by grid.cu.
#include <climits>

#include "geom.cuh"
#include "grid.cuh"

namespace gbdb {

// Sum per-thread counters over the warp and add them once per warp.
__device__ __forceinline__ void flush_counter(unsigned long long *dst, unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(dst, v);
}

// ----------------------------------------------------------------- MarkCore
// A cell with at least minPts points marks all of them core (all its points
// are within eps of each other).  In a sparser cell g each point p counts
// |g| plus RangeCount(p, eps, h) over the neighbouring cells h, scanning their
// points, and stops as soon as the count reaches minPts.  One thread per point,
// points in cell order, so the threads of a warp mostly share cells.
template <int D, int M>
__global__ void __launch_bounds__(256)
k_markcore(RunParams P, const float *__restrict__ pf, const double *__restrict__ pd,
           const int *__restrict__ cell_of, const int *__restrict__ cell_start,
           const long long *__restrict__ nbr_off, const int *__restrict__ nbr,
           int *__restrict__ core_s, DevCounters *ctr) {
    unsigned rech = 0;
    unsigned long long evals = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
        const int c = cell_of[i];
        int count = cell_start[c + 1] - cell_start[c];
        if (count >= P.min_pts) { core_s[i] = 1; continue; }
        Pt<D, M> p;
        load_pt(p, pf, pd, i);
        const long long e1 = nbr_off[c + 1];
        for (long long e = nbr_off[c]; e < e1 && count < P.min_pts; ++e) {
            const int h = nbr[e];
            const int t1 = cell_start[h + 1];
            for (int t = cell_start[h]; t < t1; ++t) {
                Pt<D, M> q;
                load_pt(q, pf, pd, t);
                if (P.stats) ++evals;
                if (within(p, q, P, pd, i, pd, t, rech) && ++count >= P.min_pts) break;
            }
        }
        core_s[i] = count >= P.min_pts ? 1 : 0;
    }
    flush_counter(&ctr->band_rechecks, rech);
    if (P.stats) flush_counter(&ctr->dist_evals[0], evals);
}

#define GBDB_DISPATCH(D, MODE, ...)                                          \
    do {                                                                      \
        switch ((D) * 4 + (MODE)) {                                           \
        case 8: { constexpr int DD = 2, MM = 0; __VA_ARGS__; } break;                \
        case 9: { constexpr int DD = 2, MM = 1; __VA_ARGS__; } break;                \
        case 10: { constexpr int DD = 2, MM = 2; __VA_ARGS__; } break;               \
        case 11: { constexpr int DD = 2, MM = 3; __VA_ARGS__; } break;               \
        case 12: { constexpr int DD = 3, MM = 0; __VA_ARGS__; } break;               \
        case 13: { constexpr int DD = 3, MM = 1; __VA_ARGS__; } break;               \
        case 14: { constexpr int DD = 3, MM = 2; __VA_ARGS__; } break;               \
        case 15: { constexpr int DD = 3, MM = 3; __VA_ARGS__; } break;               \
        case 16: { constexpr int DD = 4, MM = 0; __VA_ARGS__; } break;               \
        case 17: { constexpr int DD = 4, MM = 1; __VA_ARGS__; } break;               \
        case 18: { constexpr int DD = 4, MM = 2; __VA_ARGS__; } break;               \
        case 19: { constexpr int DD = 4, MM = 3; __VA_ARGS__; } break;               \
        default: break;                                                       \
        }                                                                     \
    } while (0)

void launch_markcore(int D, int mode, const RunParams &P, const Bufs &B, DevCounters *ctr, cudaStream_t s) {
    GBDB_DISPATCH(D, mode, {
        auto k = k_markcore<DD, MM>;
        int g = grid_for((const void *)k, 256);
        k<<<g, 256, 0, s>>>(P, B.pf, B.pd, B.cell_of, B.cell_start, B.nbr_off, B.nbr, B.core_s, ctr); count_launch();
    });
}

// ------------------------------------------------------- core compaction
// Copy the core points, in cell order, to dense arrays, so that the core
// points of cell c are [ccs[c], ccs[c+1]) (BCP runs on core points only,
// Algorithm 3).
template <int SD>
__global__ void __launch_bounds__(256)
k_core_compact(RunParams P, const float *__restrict__ pf, const double *__restrict__ pd,
               const int *__restrict__ orig, const int *__restrict__ cell_of,
               const int *__restrict__ cell_start, const int *__restrict__ core_s,
               const int *__restrict__ core_pos, float *__restrict__ cpf, double *__restrict__ cpd,
               int *__restrict__ core_orig, int *__restrict__ core_cell, int *__restrict__ ccs,
               DevCounters *ctr) {
    const int m = ctr->m;
    const int stride = gridDim.x * blockDim.x;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += stride) {
        if (!core_s[i]) continue;
        const int k = core_pos[i];
#pragma unroll
        for (int j = 0; j < SD; j += 2)
            reinterpret_cast<float2 *>(cpf)[(int64_t)k * (SD / 2) + j / 2] =
                reinterpret_cast<const float2 *>(pf)[(int64_t)i * (SD / 2) + j / 2];
        if (pd) {
#pragma unroll
            for (int j = 0; j < SD; j += 2)
                reinterpret_cast<double2 *>(cpd)[(int64_t)k * (SD / 2) + j / 2] =
                    reinterpret_cast<const double2 *>(pd)[(int64_t)i * (SD / 2) + j / 2];
        }
        core_orig[k] = orig[i];
        core_cell[k] = cell_of[i];
    }
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c <= m; c += stride)
        ccs[c] = c < m ? core_pos[cell_start[c]] : core_pos[P.n];
    if (blockIdx.x == 0 && threadIdx.x == 0) ctr->n_core = core_pos[P.n];
}

void launch_core_compact(int SD, const RunParams &P, const Bufs &B, DevCounters *ctr, cudaStream_t s) {
    scan_i32_to_i32(B.core_s, B.core_pos, P.n, nullptr, P.n, B.part, s);
    auto go = [&](auto k) {
        int g = grid_for((const void *)k, 256);
        k<<<g, 256, 0, s>>>(P, B.pf, B.pd, B.orig, B.cell_of, B.cell_start, B.core_s, B.core_pos,
                            B.cpf, B.cpd, B.core_orig, B.core_cell, B.ccs, ctr); count_launch();
    };
    if (SD == 2) go(k_core_compact<2>);
    else if (SD == 4) go(k_core_compact<4>);
    else go(k_core_compact<8>);
}

// ----------------------------------------------------------------- schedule
// SortBySize (Algorithm 3): core cells in order of non-increasing core count.
// Each unordered pair of neighbouring core cells is owned by the cell that
// comes first in that order ("g > h" in Algorithm 3), and the pair list is
// written owner by owner, so list order is test priority.
__global__ void __launch_bounds__(256)
k_size_keys(const int *__restrict__ ccs, int nkey, uint64_t *__restrict__ keys, uint32_t *__restrict__ vals,
            const DevCounters *ctr) {
    const int m = ctr->m;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x) {
        keys[c] = (uint64_t)(nkey - (ccs[c + 1] - ccs[c]));
        vals[c] = (uint32_t)c;
    }
}

__global__ void __launch_bounds__(256)
k_rank(const uint32_t *__restrict__ order, int *__restrict__ rank, const DevCounters *ctr) {
    const int m = ctr->m;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < m; r += gridDim.x * blockDim.x)
        rank[order ? (int)order[r] : r] = r;
}

template <bool FILL>
__global__ void __launch_bounds__(256)
k_pairs(const uint32_t *__restrict__ order, const int *__restrict__ rank, const int *__restrict__ ccs,
        const long long *__restrict__ nbr_off, const int *__restrict__ nbr, long long *__restrict__ cnt_or_off,
        int2 *__restrict__ pairs, long long cap, DevCounters *ctr) {
    const int m = ctr->m;
    int ncc = 0;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < m; r += gridDim.x * blockDim.x) {
        const int a = order ? (int)order[r] : r;
        long long cnt = 0;
        const long long base = FILL ? cnt_or_off[r] : 0;
        if (ccs[a + 1] > ccs[a]) {
            ++ncc;
            const long long e1 = nbr_off[a + 1];
            for (long long e = nbr_off[a]; e < e1; ++e) {
                const int b = nbr[e];
                if (ccs[b + 1] > ccs[b] && rank[b] > r) {
                    if (FILL) {
                        if (base + cnt < cap) pairs[base + cnt] = make_int2(a, b);
                        else set_error(ctr, DBSCAN_ERR_CAPACITY, 20);
                    }
                    ++cnt;
                }
            }
        }
        if (!FILL) cnt_or_off[r] = cnt;
    }
    if (!FILL) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) ncc += __shfl_xor_sync(0xffffffffu, ncc, o);
        if ((threadIdx.x & 31) == 0 && ncc) atomicAdd(&ctr->m_core, ncc);
    }
}

__global__ void k_store_P(const long long *off, DevCounters *ctr) { ctr->P = off[ctr->m]; }

void launch_schedule(int sched, const RunParams &P, const Bufs &B, DevCounters *ctr, cudaStream_t s) {
    const uint32_t *order = nullptr;
    const int *m_dev = &ctr->m;
    if (sched == DBSCAN_SCHED_SIZE) {
        int bits = 1;
        while ((1ll << bits) <= (long long)P.n) ++bits;
        const int nkey = (int)((1ll << bits) - 1);
        int g = grid_for((const void *)k_size_keys, 256);
        k_size_keys<<<g, 256, 0, s>>>(B.ccs, nkey, B.sk0, B.sv0, ctr); count_launch();
        int which = radix_sort_u64(B.sk0, B.sv0, B.sk1, B.sv1, 0, m_dev, B.n_max, bits, B.hist, B.part, s);
        order = which ? B.sv1 : B.sv0;
    }
    int g = grid_for((const void *)k_rank, 256);
    k_rank<<<g, 256, 0, s>>>(order, B.rank, ctr); count_launch();
    g = grid_for((const void *)k_pairs<false>, 256);
    k_pairs<false><<<g, 256, 0, s>>>(order, B.rank, B.ccs, B.nbr_off, B.nbr, B.pcnt, nullptr, 0, ctr); count_launch();
    scan_i64_to_i64(B.pcnt, B.poff, 0, m_dev, B.n_max, B.part, s);
    k_store_P<<<1, 1, 0, s>>>(B.poff, ctr); count_launch();
    k_pairs<true><<<g, 256, 0, s>>>(order, B.rank, B.ccs, B.nbr_off, B.nbr, B.poff, B.pairs, B.pair_cap, ctr); count_launch();
}

// ----------------------------------------------------------------- connect
// Connected(g, h) over core points (Sec. 4.4, BCP-based cell graph): stop at
// the first pair within eps.  The warp tests a block of 32 point pairs per
// step and leaves on a warp vote.  The smaller cell's points stay in
// registers: with nc <= 32 columns, each lane holds one column point and the
// warp covers 32/L rows per step (L = lanes per row).
template <int D, int M>
__device__ __forceinline__ bool bcp_warp(int r0, int nr, int c0, int nc, const float *__restrict__ cpf,
                                         const double *__restrict__ cpd, const RunParams &P,
                                         unsigned &rech, unsigned long long &evals) {
    const int lane = threadIdx.x & 31;
    if (nc <= 32) {
        int lg = 0;
        while ((1 << lg) < nc) ++lg;
        const int L = 1 << lg;
        const int R = 32 >> lg;
        const int j = lane & (L - 1), rr = lane >> lg;
        const bool qv = j < nc;
        Pt<D, M> q;
        if (qv) load_pt(q, cpf, cpd, c0 + j);
        for (int rb = 0; rb < nr; rb += R) {
            const int r = rb + rr;
            bool t = false;
            if (qv && r < nr) {
                Pt<D, M> p;
                load_pt(p, cpf, cpd, r0 + r);
                if (P.stats) ++evals;
                t = within(p, q, P, cpd, r0 + r, cpd, c0 + j, rech);
            }
            if (__any_sync(0xffffffffu, t)) return true;
        }
        return false;
    }
    for (int cb = 0; cb < nc; cb += 32) {
        const int j = cb + lane;
        const bool qv = j < nc;
        Pt<D, M> q;
        if (qv) load_pt(q, cpf, cpd, c0 + j);
        for (int r = 0; r < nr; ++r) {
            bool t = false;
            if (qv) {
                Pt<D, M> p;
                load_pt(p, cpf, cpd, r0 + r);
                if (P.stats) ++evals;
                t = within(p, q, P, cpd, r0 + r, cpd, c0 + j, rech);
            }
            if (__any_sync(0xffffffffu, t)) return true;
        }
    }
    return false;
}

// ClusterCore's pair loop (Algorithm 3): a warp takes the next 32 pairs of
// the priority-ordered list with one atomic, checks all 32 against the
// union-find in parallel (one pair per lane), and runs BCP on the survivors
// one at a time, re-checking each just before its test because earlier links
// may have joined it meanwhile ("Reducing Cell Connectivity Queries").  A hit
// links the two cells.
template <int D, int M>
__global__ void __launch_bounds__(256)
k_connect(RunParams P, const int2 *__restrict__ pairs, const int *__restrict__ ccs,
          const float *__restrict__ cpf, const double *__restrict__ cpd, int *parent, DevCounters *ctr) {
    const int lane = threadIdx.x & 31;
    const unsigned long long np = (unsigned long long)ctr->P;
    unsigned rech = 0;
    unsigned long long evals = 0, tested = 0, skipped = 0, linked = 0;
    for (;;) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&ctr->pair_next, 32ull);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= np) break;
        const unsigned long long idx = base + lane;
        const bool valid = idx < np;
        int2 pr = make_int2(0, 0);
        bool same = true;
        if (valid) {
            pr = pairs[idx];
            same = uf_find(parent, pr.x, P.max_iters, ctr) == uf_find(parent, pr.y, P.max_iters, ctr);
        }
        unsigned todo = __ballot_sync(0xffffffffu, !same);
        skipped += __popc(__ballot_sync(0xffffffffu, valid && same));
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const int a = __shfl_sync(0xffffffffu, pr.x, src);
            const int b = __shfl_sync(0xffffffffu, pr.y, src);
            int again = 0;
            if (lane == 0) again = uf_find(parent, a, P.max_iters, ctr) == uf_find(parent, b, P.max_iters, ctr);
            if (__shfl_sync(0xffffffffu, again, 0)) { ++skipped; continue; }
            ++tested;
            const int a0 = ccs[a], na = ccs[a + 1] - a0;
            const int b0 = ccs[b], nb = ccs[b + 1] - b0;
            const bool hit = na >= nb ? bcp_warp<D, M>(a0, na, b0, nb, cpf, cpd, P, rech, evals)
                                      : bcp_warp<D, M>(b0, nb, a0, na, cpf, cpd, P, rech, evals);
            if (hit) {
                ++linked;
                if (lane == 0) uf_link(parent, a, b, P.max_iters, ctr);
            }
        }
    }
    if (lane == 0) {
        if (tested) atomicAdd(&ctr->pairs_tested, tested);
        if (skipped) atomicAdd(&ctr->pairs_skipped, skipped);
        if (linked) atomicAdd(&ctr->pairs_linked, linked);
    }
    flush_counter(&ctr->band_rechecks, rech);
    if (P.stats) flush_counter(&ctr->dist_evals[1], evals);
}

__global__ void __launch_bounds__(256) k_uf_init(int *parent, const DevCounters *ctr) {
    const int m = ctr->m;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x) parent[c] = c;
}

void launch_connect(int D, int mode, const RunParams &P, const Bufs &B, DevCounters *ctr, cudaStream_t s) {
    int g = grid_for((const void *)k_uf_init, 256);
    k_uf_init<<<g, 256, 0, s>>>(B.parent, ctr); count_launch();
    GBDB_DISPATCH(D, mode, {
        auto k = k_connect<DD, MM>;
        int gg = grid_for((const void *)k, 256);
        k<<<gg, 256, 0, s>>>(P, B.pairs, B.ccs, B.cpf, B.cpd, B.parent, ctr); count_launch();
    });
}

// ----------------------------------------------------------------- labels
// clusters[p] := Find(g) for core p (Algorithm 3), renamed to the smallest
// input index of a core point in the component.
__global__ void __launch_bounds__(256) k_uf_flatten(int *parent, int *compmin, DevCounters *ctr, int max_iters) {
    const int m = ctr->m;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x) {
        parent[c] = uf_find(parent, c, max_iters, ctr);
        compmin[c] = INT_MAX;
    }
}

__global__ void __launch_bounds__(256)
k_comp_min(const int *__restrict__ ccs, const int *__restrict__ core_orig, const int *__restrict__ parent,
           int *compmin, const DevCounters *ctr) {
    const int m = ctr->m;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x) {
        const int k0 = ccs[c], k1 = ccs[c + 1];
        if (k1 == k0) continue;
        int mn = INT_MAX;
        for (int k = k0; k < k1; ++k) mn = min(mn, core_orig[k]);
        atomicMin(compmin + parent[c], mn);
    }
}

__global__ void __launch_bounds__(256)
k_label_core(RunParams P, const int *__restrict__ core_s, const int *__restrict__ orig,
             const int *__restrict__ cell_of, const int *__restrict__ parent, const int *__restrict__ compmin,
             uint8_t *__restrict__ core_out, int32_t *__restrict__ labels_out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
        const int o = orig[i];
        const int cf = core_s[i];
        core_out[o] = (uint8_t)cf;
        if (cf) labels_out[o] = compmin[parent[cell_of[i]]];
    }
}

void launch_labels(const RunParams &P, const Bufs &B, uint8_t *core_out, int32_t *labels_out,
                   DevCounters *ctr, cudaStream_t s) {
    int g = grid_for((const void *)k_uf_flatten, 256);
    k_uf_flatten<<<g, 256, 0, s>>>(B.parent, B.compmin, ctr, P.max_iters); count_launch();
    g = grid_for((const void *)k_comp_min, 256);
    k_comp_min<<<g, 256, 0, s>>>(B.ccs, B.core_orig, B.parent, B.compmin, ctr); count_launch();
    g = grid_for((const void *)k_label_core, 256);
    k_label_core<<<g, 256, 0, s>>>(P, B.core_s, B.orig, B.cell_of, B.parent, B.compmin, core_out, labels_out); count_launch();
}

// ----------------------------------------------------------------- border
// ClusterBorder (Algorithm 4): a non-core point p of cell g joins the cluster
// of every cell h in {g} and NeighborCells(g) that has a core point within eps
// of p.  The scan of h stops at its first hit, and h is not scanned at all when
// its cluster is already in p's set.  The set stays sorted in a local array:
// the core points of distinct clusters seen by p are pairwise farther than eps
// apart and all within eps of p, so there are at most kissing-number many of
// them (240 in R^8), under kBorderSetCap.
template <int D, int M, bool FILL>
__global__ void __launch_bounds__(128)
k_border(RunParams P, Bufs B, int32_t *__restrict__ labels_out, int32_t *__restrict__ ids,
         long long ids_cap, DevCounters *ctr) {
    unsigned rech = 0;
    unsigned long long evals = 0, nborder = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
        const int o = B.orig[i];
        if (B.core_s[i]) {
            if (!FILL) B.bcount[o] = 0;
            continue;
        }
        const int g = B.cell_of[i];
        Pt<D, M> p;
        load_pt(p, B.pf, B.pd, i);
        int set[kBorderSetCap];
        int ns = 0;
        const long long e0 = B.nbr_off[g], e1 = B.nbr_off[g + 1];
        for (long long e = e0 - 1; e < e1; ++e) {
            const int h = e < e0 ? g : B.nbr[e];
            const int k0 = B.ccs[h], k1 = B.ccs[h + 1];
            if (k0 == k1) continue;
            const int L = B.compmin[B.parent[h]];
            bool have = false;
            for (int t = 0; t < ns; ++t) have = have || set[t] == L;
            if (have) continue;
            for (int k = k0; k < k1; ++k) {
                Pt<D, M> q;
                load_pt(q, B.cpf, B.cpd, k);
                if (P.stats) ++evals;
                if (within(p, q, P, B.pd, i, B.cpd, k, rech)) {
                    if (ns < kBorderSetCap) {
                        int t = ns++;
                        while (t > 0 && set[t - 1] > L) { set[t] = set[t - 1]; --t; }
                        set[t] = L;
                    } else {
                        set_error(ctr, DBSCAN_ERR_CAPACITY, 30);
                    }
                    break;
                }
            }
        }
        if (!FILL) {
            B.bcount[o] = ns;
            labels_out[o] = ns ? set[0] : -1;
            nborder += ns ? 1 : 0;
        } else {
            const long long at = B.boff[o];
            if (at + ns <= ids_cap) {
                for (int t = 0; t < ns; ++t) ids[at + t] = set[t];
            } else {
                set_error(ctr, DBSCAN_ERR_CAPACITY, 31);
            }
        }
    }
    if (!FILL) {
        flush_counter(&ctr->band_rechecks, rech);
        if (P.stats) flush_counter(&ctr->dist_evals[2], evals);
        unsigned long long nb = nborder;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) nb += __shfl_xor_sync(0xffffffffu, nb, o);
        if ((threadIdx.x & 31) == 0 && nb) atomicAdd((unsigned *)&ctr->n_border, (unsigned)nb);
    }
}

__global__ void k_store_K(const long long *off, int n, DevCounters *ctr) { ctr->K = off[n]; }

void launch_border(int D, int mode, bool fill, const RunParams &P, const Bufs &B, int32_t *labels_out,
                   int32_t *ids, long long ids_cap, DevCounters *ctr, cudaStream_t s) {
    if (!fill) {
        GBDB_DISPATCH(D, mode, {
            auto k = k_border<DD, MM, false>;
            int g = grid_for((const void *)k, 128);
            k<<<g, 128, 0, s>>>(P, B, labels_out, nullptr, 0, ctr); count_launch();
        });
        scan_i64_to_i64(B.bcount, B.boff, P.n, nullptr, P.n, B.part, s);
        k_store_K<<<1, 1, 0, s>>>(B.boff, P.n, ctr); count_launch();
    } else {
        GBDB_DISPATCH(D, mode, {
            auto k = k_border<DD, MM, true>;
            int g = grid_for((const void *)k, 128);
            k<<<g, 128, 0, s>>>(P, B, labels_out, ids, ids_cap, ctr); count_launch();
        });
    }
}

}  // namespace gbdb
