// MarkCore (Algorithm 2), ClusterCore (Algorithm 3) and ClusterBorder
// (Algorithm 4) on the cell structure built by grid.cu.
#include <climits>

#include "bcp.cuh"
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
// are within eps of each other).  In a sparser cell g every point p counts
// |g| plus RangeCount(p, eps, h) over the neighbouring cells h, scanning their
// points, and stops once the count reaches minPts.
//
// One warp per cell.  The cell's own points (up to MC_OWN at a time) sit in
// shared memory and, one per lane, in registers.  In the FP32-band mode each
// neighbouring cell h is first classified per own point against h's bounding
// box (Sec. 5.2 counts whole quadtree cells the same way): entirely within eps
// -> add |h|; entirely beyond -> skip; otherwise the warp streams h 32 points
// at a time, one per lane, and for every such own point tests all 32 at once
// and adds the vote count.  The lanes stay converged, the loads coalesce, and
// the cell stops once all its points reached minPts.
constexpr int MC_THREADS = 256, MC_WARPS = MC_THREADS / 32, MC_OWN = 128;
// Sparse cells with fewer points than MC_SMALL and at most P.mc_small_nbr
// points in their neighbouring cells (0: none) go to k_markcore_small (one
// thread per point): a warp per cell would leave most of its lanes idle, and a
// thread's serial scan stays short.  The autotuner picks the limit.
constexpr int MC_SMALL = 8;
constexpr int MC_SMALL_ALL = 1 << 30;  // no neighbourhood limit (nbr_pts is then not computed)
__device__ __forceinline__ bool mc_small(const RunParams &P, int k, const int *nbr_pts, int c) {
    if (P.mc_small_nbr <= 0 || k >= MC_SMALL) return false;  // 0: the warp kernel takes all
    return P.mc_small_nbr >= MC_SMALL_ALL || nbr_pts[c] <= P.mc_small_nbr;
}

// RangeCount(p, eps, h) of Sec. 5.2 on the quadtree of cell h (points
// [t0, t1)): the points within eps of p, counted until `need` is reached.  A
// depth-first descent over the node boxes: a node whose points are all within
// eps counts whole, one with none is skipped, a leaf in between is scanned with
// the exact test (FP32 band, FP64 recheck).  Only for d >= 5 in the FP32-band
// mode; cells below QT_MIN points are scanned directly.
constexpr int QT_MIN = 32;

template <int D, int M>
__device__ __forceinline__ int qt_range_count(const Pt<D, M> &p, int t0, int t1, const QtView &Q, const Thr &T,
                                              const RunParams &P, const float *__restrict__ pf,
                                              const double *__restrict__ pd, int64_t ip, int need, unsigned &rech,
                                              unsigned long long &evals) {
    int cnt = 0;
    if constexpr (D == 8 && (M == kF32FromF32 || M == kF32FromF64)) {
        int cur[4], end[4];
        int lv = 1;
        cur[1] = Q.qpos[0][t0];
        end[1] = Q.qpos[0][t1];
        while (lv > 0) {
            if (cur[lv] >= end[lv]) {
                --lv;
                continue;
            }
            const int k = cur[lv]++;
            const int a = Q.qstart[lv - 1][k], b = Q.qstart[lv - 1][k + 1];
            const Bx<8> lo = load_box<8>(Q.qlo[lv - 1], k), hi = load_box<8>(Q.qhi[lv - 1], k);
            if (box_max_d2<8>(p.f, lo, hi) <= T.lo) {  // every point of the node within eps
                cnt += b - a;
                if (cnt >= need) return cnt;
                continue;
            }
            if (box_min_d2<8>(p.f, lo, hi) > T.hi) continue;  // none
            if (lv == Q.levels) {
                for (int u = a; u < b; ++u) {
                    Pt<D, M> q;
                    load_pt(q, pf, pd, u);
                    if (P.stats) ++evals;
                    if (within(p, q, T, pd, ip, pd, u, rech) && ++cnt >= need) return cnt;
                }
                continue;
            }
            ++lv;
            cur[lv] = Q.qpos[lv - 1][a];
            end[lv] = Q.qpos[lv - 1][b];
        }
    }
    return cnt;
}

// One batch of kb <= 32*NS own points of a sparse cell whose k points start at
// s0 (the batch starts at own index b0); own[] holds the batch.
template <int D, int M, int NS>
__device__ __forceinline__ void mc_batch(const RunParams &P, const Thr &T, const float *__restrict__ pf,
                                         const double *__restrict__ pd,
                                         const int *__restrict__ cell_start, const int *__restrict__ nl, int ne,
                                         const float4 *__restrict__ blo, const float4 *__restrict__ bhi,
                                         const Pt<D, M> *own, int s0, int b0, int k, int kb, int *__restrict__ core_s,
                                         Bx<D> (*sbox)[2], const QtView &Q, unsigned &rech,
                                         unsigned long long &evals) {
    constexpr bool BOX = (M == kF32FromF32 || M == kF32FromF64);
    const int lane = threadIdx.x & 31;
    const bool use_box = BOX && P.box;
    int cnt[NS];
    unsigned done[NS];
    Pt<D, M> mine[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        cnt[s] = k;
        const int left = kb - s * 32;
        done[s] = left <= 0 ? 0xffffffffu : (left >= 32 ? 0u : ~((1u << left) - 1u));
        if (use_box && s * 32 + lane < kb) mine[s] = own[s * 32 + lane];
    }
    bool all = false;
    for (int e0 = 0; e0 < ne && !all; e0 += 32) {
        // one lane per neighbour: fetch its range (and warm its box in L1) at once
        int h_t0 = 0, h_t1 = 0, h = 0;
        if (e0 + lane < ne) {
            h = nl[e0 + lane];
            h_t0 = cell_start[h];
            h_t1 = cell_start[h + 1];
            // and stage its box, so the loop below reads it from shared memory
            if (use_box) {
                sbox[lane][0] = load_box<D>(blo, h);
                sbox[lane][1] = load_box<D>(bhi, h);
            }
        }
        __syncwarp();
        const int ecount = min(32, ne - e0);
        for (int j = 0; j < ecount && !all; ++j) {
            const int t0 = __shfl_sync(0xffffffffu, h_t0, j), t1 = __shfl_sync(0xffffffffu, h_t1, j);
            unsigned part[NS];
            if (use_box) {
                const Bx<D> lo = sbox[j][0], hi = sbox[j][1];
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    bool partial = false;
                    if (!((done[s] >> lane) & 1u)) {
                        if constexpr (BOX) {
                            if (box_max_d2<D>(mine[s].f, lo, hi) <= T.lo) cnt[s] += t1 - t0;
                            else partial = box_min_d2<D>(mine[s].f, lo, hi) <= T.hi;
                        }
                    }
                    part[s] = __ballot_sync(0xffffffffu, partial);
                }
            } else {
#pragma unroll
                for (int s = 0; s < NS; ++s) part[s] = ~done[s];
            }
            unsigned any = 0;
#pragma unroll
            for (int s = 0; s < NS; ++s) any |= part[s];
            if constexpr (D == 8 && BOX) {
                // a large neighbouring cell: each lane left undecided by the
                // cell box descends its quadtree on its own
                if (any && Q.levels > 0 && t1 - t0 >= QT_MIN) {
#pragma unroll
                    for (int s = 0; s < NS; ++s)
                        if ((part[s] >> lane) & 1u)
                            cnt[s] += qt_range_count<D, M>(mine[s], t0, t1, Q, T, P, pf, pd, s0 + b0 + s * 32 + lane,
                                                           T.min_pts - cnt[s], rech, evals);
                    any = 0;
                }
            }
            for (int tb = t0; tb < t1 && any; tb += 32) {
                const int t = tb + lane;
                const bool qv = t < t1;
                Pt<D, M> q;
                if (qv) load_pt(q, pf, pd, t);
                any = 0;
#pragma unroll
                for (int s = 0; s < NS; ++s) {
                    unsigned todo = part[s];
                    while (todo) {
                        const int src = __ffs(todo) - 1;
                        todo &= todo - 1;
                        const int i = s * 32 + src;
                        bool hit = false;
                        if (qv) {
                            if (P.stats) ++evals;
                            hit = within(own[i], q, T, pd, s0 + b0 + i, pd, t, rech);
                        }
                        const int got = __popc(__ballot_sync(0xffffffffu, hit));
                        if (lane == src) cnt[s] += got;
                    }
                    part[s] &= ~__ballot_sync(0xffffffffu, cnt[s] >= T.min_pts);
                    any |= part[s];
                }
            }
            all = true;
#pragma unroll
            for (int s = 0; s < NS; ++s) {
                done[s] |= __ballot_sync(0xffffffffu, cnt[s] >= T.min_pts);
                all = all && done[s] == 0xffffffffu;
            }
        }
        __syncwarp();  // the stage is rewritten for the next 32 neighbours
    }
#pragma unroll
    for (int s = 0; s < NS; ++s) {
        const int i = s * 32 + lane;
        if (i < kb) core_s[s0 + b0 + i] = cnt[s] >= T.min_pts ? 1 : 0;
    }
}

template <int D, int M>
__global__ void __launch_bounds__(MC_THREADS, D <= 4 ? 6 : 4)  // d <= 4: 48 warps per SM (measured faster than 24-40)
k_markcore(RunParams P, const float *__restrict__ pf, const double *__restrict__ pd,
           const int *__restrict__ cell_start, const int *__restrict__ nbr_cnt, const int *__restrict__ nbr,
           int stride, const long long *__restrict__ nbr_off, const int *__restrict__ nbr_pts,
           const float4 *__restrict__ blo, const float4 *__restrict__ bhi, int *__restrict__ core_s,
           QtView Q, DevCounters *ctr) {
    if (run_failed(ctr)) return;
    constexpr int OWN = D == 8 ? 64 : MC_OWN;  // 8-wide points: at most two slots in registers
    __shared__ Pt<D, M> own[MC_WARPS][OWN];
    __shared__ Bx<D> sbox[MC_WARPS][32][2];  // boxes of the next 32 neighbouring cells
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int m = ctr->m;
    unsigned rech = 0;
    unsigned long long evals = 0, mc_bound = 0;
    for (int c = warp_id_global(); c < m; c += warps_global()) {
        const int s0 = cell_start[c], k = cell_start[c + 1] - s0;
        const Thr T = P.inst[inst_of_cell(P, c)].thr;
        if (k >= T.min_pts) {
            for (int i = lane; i < k; i += 32) core_s[s0 + i] = 1;
            continue;
        }
        if (mc_small(P, k, nbr_pts, c)) continue;  // k_markcore_small
        const int ne = nbr_cnt[c];
        const int *nl = nbr_list<D>(nbr, nbr_off, stride, c);
        if (P.stats) {
            // algorithmic work: |g| times the points of all neighbouring cells
            // (the own cell counts |g| without tests, Algorithm 2)
            unsigned long long pts = 0;
            for (int e = lane; e < ne; e += 32) pts += cell_start[nl[e] + 1] - cell_start[nl[e]];
            mc_bound += (unsigned long long)k * pts;
        }
        for (int b0 = 0; b0 < k; b0 += OWN) {
            const int kb = min(OWN, k - b0);
            __syncwarp();
            for (int i = lane; i < kb; i += 32) load_pt(own[w][i], pf, pd, s0 + b0 + i);
            __syncwarp();
            if (kb <= 32)
                mc_batch<D, M, 1>(P, T, pf, pd, cell_start, nl, ne, blo, bhi, own[w], s0, b0, k, kb, core_s, sbox[w], Q,
                                  rech, evals);
            else if (OWN <= 64 || kb <= 64)
                mc_batch<D, M, 2>(P, T, pf, pd, cell_start, nl, ne, blo, bhi, own[w], s0, b0, k, kb, core_s, sbox[w], Q,
                                  rech, evals);
            else
                mc_batch<D, M, (OWN > 64 ? 4 : 2)>(P, T, pf, pd, cell_start, nl, ne, blo, bhi, own[w], s0, b0, k, kb,
                                                   core_s, sbox[w], Q, rech, evals);
        }
    }
    flush_counter(&ctr->band_rechecks, rech);
    if (P.stats) {
        flush_counter(&ctr->dist_evals[0], evals);
        flush_counter(&ctr->mc_bound, mc_bound);
    }
}

// MarkCore for the points of sparse cells with fewer than MC_SMALL points and
// at most P.mc_small_nbr points in their neighbouring cells: each thread counts
// for one point, walking its cell's neighbour list with the same per-point box
// classification and early exit as the warp kernel.  Consecutive threads hold
// consecutive points in cell order, so the threads of one cell read the same
// neighbour entries.  Pays off on sparse inputs (a few points per cell).
template <int D, int M>
__global__ void __launch_bounds__(256)
k_markcore_small(RunParams P, const float *__restrict__ pf, const double *__restrict__ pd,
                 const int *__restrict__ cell_of, const int *__restrict__ cell_start, const int *__restrict__ nbr_cnt,
                 const int *__restrict__ nbr, int stride, const long long *__restrict__ nbr_off,
                 const int *__restrict__ nbr_pts, const float4 *__restrict__ blo, const float4 *__restrict__ bhi,
                 int *__restrict__ core_s, QtView Q, DevCounters *ctr) {
    if (run_failed(ctr)) return;
    constexpr bool BOX = (M == kF32FromF32 || M == kF32FromF64);
    const bool use_box = BOX && P.box;
    unsigned rech = 0;
    unsigned long long evals = 0, mc_bound = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
        const int c = cell_of[i];
        const int s0 = cell_start[c], k = cell_start[c + 1] - s0;
        const Thr T = P.inst[inst_of_cell(P, c)].thr;
        if (k >= T.min_pts || !mc_small(P, k, nbr_pts, c)) continue;  // dense, or the warp kernel's
        Pt<D, M> p;
        load_pt(p, pf, pd, i);
        int cnt = k;
        const int ne = nbr_cnt[c];
        const int *nl = nbr_list<D>(nbr, nbr_off, stride, c);
        if (P.stats)
            for (int e = 0; e < ne; ++e) mc_bound += cell_start[nl[e] + 1] - cell_start[nl[e]];
        for (int e = 0; e < ne && cnt < T.min_pts; ++e) {
            const int h = nl[e];
            const int t0 = cell_start[h], t1 = cell_start[h + 1];
            if constexpr (BOX) {
                if (use_box) {
                    const Bx<D> lo = load_box<D>(blo, h), hi = load_box<D>(bhi, h);
                    if (box_max_d2<D>(p.f, lo, hi) <= T.lo) {
                        cnt += t1 - t0;
                        continue;
                    }
                    if (box_min_d2<D>(p.f, lo, hi) > T.hi) continue;
                    if (D == 8 && Q.levels > 0 && t1 - t0 >= QT_MIN) {  // a large cell: its quadtree
                        cnt += qt_range_count<D, M>(p, t0, t1, Q, T, P, pf, pd, i, T.min_pts - cnt, rech, evals);
                        continue;
                    }
                }
            }
            for (int t = t0; t < t1 && cnt < T.min_pts; ++t) {
                Pt<D, M> q;
                load_pt(q, pf, pd, t);
                if (P.stats) ++evals;
                if (within(p, q, T, pd, i, pd, t, rech)) ++cnt;
            }
        }
        core_s[i] = cnt >= T.min_pts ? 1 : 0;
    }
    flush_counter(&ctr->band_rechecks, rech);
    if (P.stats) {
        flush_counter(&ctr->dist_evals[0], evals);
        flush_counter(&ctr->mc_bound, mc_bound);
    }
}

void launch_markcore(int D, int mode, const RunParams &P, const Bufs &B, DevCounters *ctr, cudaStream_t s) {
    if (P.mc_small_nbr > 0) GBDB_DISPATCH(D, mode, {
        auto ks = k_markcore_small<DD, MM>;
        const int gs = grid_for((const void *)ks, 256);
        ks<<<gs, 256, 0, s>>>(P, B.pf, B.pd, B.cell_of, B.cell_start, B.nbr_cnt, B.nbr, B.nbr_stride, B.nbr_off,
                              B.nbr_pts, B.blo, B.bhi, B.core_s, B.qt, ctr);
        count_launch();
    });
    GBDB_DISPATCH(D, mode, {
        auto k = k_markcore<DD, MM>;
        int g = grid_for((const void *)k, MC_THREADS);
        k<<<g, MC_THREADS, 0, s>>>(P, B.pf, B.pd, B.cell_start, B.nbr_cnt, B.nbr, B.nbr_stride, B.nbr_off,
                                   B.nbr_pts, B.blo, B.bhi, B.core_s, B.qt, ctr);
        count_launch();
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
    if (run_failed(ctr)) return;
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
    int ncc = 0;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c <= m; c += stride) {
        ccs[c] = c < m ? core_pos[cell_start[c]] : core_pos[P.n];
        if (c < m && core_pos[cell_start[c + 1]] > core_pos[cell_start[c]]) ++ncc;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ncc += __shfl_xor_sync(0xffffffffu, ncc, o);
    if ((threadIdx.x & 31) == 0 && ncc) atomicAdd(&ctr->m_core, ncc);
    if (blockIdx.x == 0 && threadIdx.x == 0) ctr->n_core = core_pos[P.n];
}

void launch_core_compact(int SD, const RunParams &P, const Bufs &B, DevCounters *ctr, cudaStream_t s) {
    scan_i32_to_i32(B.core_s, B.core_pos, P.n, nullptr, P.n, B.part, s);
    auto go = [&](auto k) {
        int g = grid_for((const void *)k, 256);
        k<<<g, 256, 0, s>>>(P, B.pf, B.pd, B.orig, B.cell_of, B.cell_start, B.core_s, B.core_pos,
                            B.cpf, B.cpd, B.core_orig, B.core_cell, B.ccs, ctr);
        count_launch();
    };
    if (SD == 2) go(k_core_compact<2>);
    else if (SD == 4) go(k_core_compact<4>);
    else go(k_core_compact<8>);
    // core-point boxes: pair verdicts and border tests, or the learned schedule's features
    if ((P.box && P.pair_box) || B.ccent) launch_boxes(SD, B.cpf, B.ccs, ctr, B.cblo, B.cbhi, s, B.ccent);
}

// ----------------------------------------------------------------- schedule
// SortBySize (Algorithm 3): cells in order of non-increasing core count
// (counts saturate at 65535; ties keep cell order).  rank[c] is the position
// of cell c; the pair {g, h} of neighbouring core cells is tested by whichever
// of the two comes first ("g > h" in Algorithm 3).
constexpr int kSizeKeyBits = 16;

__global__ void __launch_bounds__(256)
k_size_keys(const int *__restrict__ ccs, uint64_t *__restrict__ keys, const DevCounters *ctr) {
    if (run_failed(ctr)) return;
    const int m = ctr->m;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x) {
        const int nc = min(ccs[c + 1] - ccs[c], (1 << kSizeKeyBits) - 1);
        keys[c] = ((uint64_t)(((1 << kSizeKeyBits) - 1) - nc) << 32) | (uint64_t)c;
    }
}

// rank[c] = position of cell c in the test order; order[r] = cell at r.
__global__ void __launch_bounds__(256)
k_rank(const uint64_t *__restrict__ sorted, uint32_t *__restrict__ order, int *__restrict__ rank,
       const DevCounters *ctr) {
    if (run_failed(ctr)) return;
    const int m = ctr->m;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < m; r += gridDim.x * blockDim.x) {
        const int c = sorted ? (int)(sorted[r] & 0xffffffffu) : r;
        if (sorted) order[r] = (uint32_t)c;
        rank[c] = r;
    }
}

const uint32_t *launch_schedule(int sched, const RunParams &P, const Bufs &B, DevCounters *ctr, cudaStream_t s) {
    const uint64_t *sorted = nullptr;
    if (sched == DBSCAN_SCHED_SIZE) {
        int g = grid_for((const void *)k_size_keys, 256);
        k_size_keys<<<g, 256, 0, s>>>(B.ccs, B.sk0, ctr); count_launch();
        int which = radix_sort_u64(B.sk0, nullptr, B.sk1, nullptr, 0, &ctr->m, B.n_max, 32, kSizeKeyBits,
                                   B.sort_scratch, B.sort_scratch_size, ctr, P.max_iters, s);
        sorted = which ? B.sk1 : B.sk0;
    }
    int g = grid_for((const void *)k_rank, 256);
    k_rank<<<g, 256, 0, s>>>(sorted, B.sv0, B.rank, ctr); count_launch();
    return sorted ? B.sv0 : nullptr;
}

// ----------------------------------------------------------------- connect
// ClusterCore's pair loop (Algorithm 3).  A warp takes the next P.cn_cells
// core cells in SortBySize order with one atomic; each cell owns its pairs with
// neighbouring core cells that come later in that order.  The warp flattens
// those pairs over its lanes (one (g, h) pair per lane, whatever cell it
// belongs to), so the loads of 32 pairs are in flight together; each lane
// checks its pair against the two cells' core-point boxes and the union-find;
// the survivors get a BCP test one at a time, each re-checked just before its
// test because a link made meanwhile may already join the two ("Reducing Cell
// Connectivity Queries").  A hit links the two cells.

template <int D, int M, int WAVE>
// 64 warps per SM hide the union-find latency (measured faster than 32-48 on the 2D/3D
// batch and than 32 on the 5D/7D workloads)
__global__ void __launch_bounds__(256, 8)
k_connect(RunParams P, const uint32_t *__restrict__ order, const int *__restrict__ rank,
          const int *__restrict__ ccs, const int *__restrict__ nbr_cnt, const int *__restrict__ nbr_near,
          const int *__restrict__ nbr, int stride, const long long *__restrict__ nbr_off,
          const float *__restrict__ cpf, const double *__restrict__ cpd, const float4 *__restrict__ cblo,
          const float4 *__restrict__ cbhi, int *parent, DevCounters *ctr) {
    if (run_failed(ctr)) return;
    constexpr bool BOX = (M == kF32FromF32 || M == kF32FromF64);
    const int lane = threadIdx.x & 31;
    const int m = ctr->m;
    const bool use_box = BOX && P.box && P.pair_box;
    // WAVE 0: adjacent-cell pairs (current parents compared); 1: farther pairs
    // after compression (finds); 2: all pairs in one wave (finds)
    int *next = WAVE == 1 ? &ctr->cell_next2 : &ctr->cell_next;
    const int cells = P.cn_cells;
    unsigned rech = 0;
    unsigned long long evals = 0, tested = 0, skipped = 0, linked = 0, cand_pairs = 0, boxed = 0;
    for (;;) {
        int base = 0;
        if (lane == 0) base = atomicAdd(next, cells);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= m) break;
        // lane l < cells: the cell at rank base + l and the range of its pair list
        int ca = 0, ca0 = 0, cna = 0, cbeg = 0, ccnt = 0;
        if (lane < cells && base + lane < m) {
            ca = order ? (int)order[base + lane] : base + lane;
            ca0 = ccs[ca];
            cna = ccs[ca + 1] - ca0;
            if (cna > 0) {
                const int near = nbr_near[ca];
                cbeg = WAVE == 1 ? near : 0;
                ccnt = (WAVE == 0 ? near : nbr_cnt[ca]) - cbeg;
            }
        }
        int incl = ccnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        const int cexcl = incl - ccnt;
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        for (int f0 = 0; f0 < total; f0 += 32) {
            const int f = f0 + lane;
            // owner lane: the last lane whose range starts at or before f
            int j = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int ex = __shfl_sync(0xffffffffu, cexcl, (j + step) & 31);
                if (j + step < 32 && ex <= f) j += step;
            }
            const int a = __shfl_sync(0xffffffffu, ca, j);
            const int a0 = __shfl_sync(0xffffffffu, ca0, j);
            const int na = __shfl_sync(0xffffffffu, cna, j);
            const int e = __shfl_sync(0xffffffffu, cbeg, j) + f - __shfl_sync(0xffffffffu, cexcl, j);
            const int r = base + j;
            int b = 0, b0 = 0, nb = 0;
            bool cand = false;
            if (f < total) {
                b = nbr_list<D>(nbr, nbr_off, stride, a)[e];
                b0 = ccs[b];
                nb = ccs[b + 1] - b0;
                // in cell order (no order array) the rank of a cell is its index
                cand = nb > 0 && (order ? rank[b] > r : b > a);
            }
            // union-find check first (most candidate pairs are already joined):
            // in the near wave only the current parents are compared (trees are
            // being built); the far wave runs after every path was compressed,
            // so its finds are short.  First on the L1 view of the forest (a
            // "same" there is final), then fresh
            bool same = true;
            if (cand) {
                if (WAVE == 0) {
                    same = __ldca(parent + a) == __ldca(parent + b) || uf_load(parent + a) == uf_load(parent + b);
                } else {
                    same = uf_find_stale(parent, a, P.max_iters) == uf_find_stale(parent, b, P.max_iters) ||
                           uf_find(parent, a, P.max_iters, ctr) == uf_find(parent, b, P.max_iters, ctr);
                }
            }
            // then the bounding boxes of the two cells' core points: every pair
            // beyond eps -> not connected; every pair within eps -> connected
            int verdict = 0;
            if (use_box && cand && !same) {
                const Thr T = P.inst[inst_of_cell(P, a)].cthr;
                const Bx<D> alo = load_box<D>(cblo, a), ahi = load_box<D>(cbhi, a);
                const Bx<D> blo = load_box<D>(cblo, b), bhi = load_box<D>(cbhi, b);
                if (boxes_min_d2<D>(alo, ahi, blo, bhi) > T.hi) verdict = -1;
                else if (boxes_max_d2<D>(alo, ahi, blo, bhi) <= T.lo) verdict = 1;
            }
            // a box verdict: every pair of core points is within eps, so the
            // first core points of the two cells witness the link
            if (cand && verdict > 0 && !same && uf_link(parent, a, b, P.max_iters, ctr)) record_link(P, ctr, a0, b0);
            cand_pairs += __popc(__ballot_sync(0xffffffffu, cand));
            boxed += __popc(__ballot_sync(0xffffffffu, cand && !same && verdict != 0));
            linked += __popc(__ballot_sync(0xffffffffu, cand && verdict > 0 && !same));
            skipped += __popc(__ballot_sync(0xffffffffu, cand && same));
            unsigned todo = __ballot_sync(0xffffffffu, cand && verdict == 0 && !same);
            while (todo) {
                const int src = __ffs(todo) - 1;
                todo &= todo - 1;
                const int sa = __shfl_sync(0xffffffffu, a, src), sa0 = __shfl_sync(0xffffffffu, a0, src);
                const int sna = __shfl_sync(0xffffffffu, na, src);
                const int sb = __shfl_sync(0xffffffffu, b, src), sb0 = __shfl_sync(0xffffffffu, b0, src);
                const int snb = __shfl_sync(0xffffffffu, nb, src);
                int again = 0;
                if (lane == 0) again = uf_find(parent, sa, P.max_iters, ctr) == uf_find(parent, sb, P.max_iters, ctr);
                if (__shfl_sync(0xffffffffu, again, 0)) { ++skipped; continue; }
                ++tested;
                const Thr T = P.inst[inst_of_cell(P, sa)].cthr;
                int2 wp;
                const bool hit = sna >= snb ? bcp_warp<D, M>(sa0, sna, sb0, snb, cpf, cpd, P, T, rech, evals, wp)
                                            : bcp_warp<D, M>(sb0, snb, sa0, sna, cpf, cpd, P, T, rech, evals, wp);
                if (hit) {
                    ++linked;
                    if (lane == 0 && uf_link(parent, sa, sb, P.max_iters, ctr)) record_link(P, ctr, wp.x, wp.y);
                }
            }
        }
    }
    if (lane == 0) {
        if (tested) atomicAdd(&ctr->pairs_tested, tested);
        if (skipped) atomicAdd(&ctr->pairs_skipped, skipped);
        if (linked) atomicAdd(&ctr->pairs_linked, linked);
        if (boxed) atomicAdd(&ctr->pairs_box, boxed);
        if (cand_pairs) atomicAdd((unsigned long long *)&ctr->P, cand_pairs);
    }
    flush_counter(&ctr->band_rechecks, rech);
    if (P.stats) flush_counter(&ctr->dist_evals[1], evals);
}

// Full path compression between the two waves.
__global__ void __launch_bounds__(256) k_uf_compress(int *parent, DevCounters *ctr, int max_iters) {
    if (run_failed(ctr)) return;
    const int m = ctr->m;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x)
        parent[c] = uf_find(parent, c, max_iters, ctr);
}

void launch_uf_compress(int *parent, DevCounters *ctr, int max_iters, cudaStream_t s) {
    const int g = grid_for((const void *)k_uf_compress, 256);
    k_uf_compress<<<g, 256, 0, s>>>(parent, ctr, max_iters);
    count_launch();
}

__global__ void __launch_bounds__(256) k_uf_init(int *parent, const DevCounters *ctr) {
    if (run_failed(ctr)) return;
    const int m = ctr->m;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x) parent[c] = c;
}

// Two waves over the priority order (the batches of "bucketing", Sec. 4.4):
// first every core cell's pairs with the adjacent cells (|delta|_inf <= 1),
// which are the likeliest to connect, then, after full path compression, the
// pairs with the farther cells, most of which union-find then skips.
void launch_connect(int D, int mode, const uint32_t *order, const RunParams &P, const Bufs &B, DevCounters *ctr,
                    cudaStream_t s) {
    int g = grid_for((const void *)k_uf_init, 256);
    k_uf_init<<<g, 256, 0, s>>>(B.parent, ctr); count_launch();
    GBDB_DISPATCH(D, mode, {
        if (P.waves == 1) {
            auto k2 = k_connect<DD, MM, 2>;
            const int g2 = grid_for((const void *)k2, 256);
            k2<<<g2, 256, 0, s>>>(P, order, B.rank, B.ccs, B.nbr_cnt, B.nbr_near, B.nbr, B.nbr_stride, B.nbr_off,
                                  B.cpf, B.cpd, B.cblo, B.cbhi, B.parent, ctr);
            count_launch();
            break;
        }
        auto k0 = k_connect<DD, MM, 0>;
        int gg = grid_for((const void *)k0, 256);
        k0<<<gg, 256, 0, s>>>(P, order, B.rank, B.ccs, B.nbr_cnt, B.nbr_near, B.nbr, B.nbr_stride, B.nbr_off, B.cpf, B.cpd,
                              B.cblo, B.cbhi, B.parent, ctr);
        count_launch();
        int gc = grid_for((const void *)k_uf_compress, 256);
        k_uf_compress<<<gc, 256, 0, s>>>(B.parent, ctr, P.max_iters); count_launch();
        auto k1 = k_connect<DD, MM, 1>;
        k1<<<gg, 256, 0, s>>>(P, order, B.rank, B.ccs, B.nbr_cnt, B.nbr_near, B.nbr, B.nbr_stride, B.nbr_off, B.cpf, B.cpd,
                              B.cblo, B.cbhi, B.parent, ctr);
        count_launch();
    });
}

// ----------------------------------------------------------------- labels
// clusters[p] := Find(g) for core p (Algorithm 3), renamed to the smallest
// input index of a core point in the component.  The same pass lists the
// non-core points for ClusterBorder.
// Flattening takes three passes.  A compressing find per cell (k_uf_compress)
// leaves every cell within a step or two of its root, but not always on it: a
// path-halving store of another thread may land after a cell's own store of its
// root.  So the roots are then read without any store (the forest is static
// during that pass), into compmin, and written to parent by a third pass.
__global__ void __launch_bounds__(256) k_uf_roots(const int *__restrict__ parent, int *__restrict__ root,
                                                  DevCounters *ctr, int max_iters) {
    if (run_failed(ctr)) return;
    const int m = ctr->m;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x) {
        int x = c, it = 0;
        for (; it < max_iters; ++it) {
            const int p = parent[x];
            if (p == x) break;
            x = p;
        }
        if (it == max_iters) set_error(ctr, DBSCAN_ERR_DEVICE_TIMEOUT, 3);
        root[c] = x;
    }
}

__global__ void __launch_bounds__(256) k_uf_flatten(int *__restrict__ parent, int *__restrict__ compmin,
                                                    const DevCounters *ctr) {
    if (run_failed(ctr)) return;
    const int m = ctr->m;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x) {
        parent[c] = compmin[c];  // the root found by k_uf_roots
        compmin[c] = INT_MAX;
    }
}

__global__ void __launch_bounds__(256)
k_comp_min(const int *__restrict__ ccs, const int *__restrict__ core_orig, const int *__restrict__ parent,
           int *compmin, const DevCounters *ctr) {
    if (run_failed(ctr)) return;
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
             uint8_t *__restrict__ core_out, int32_t *__restrict__ labels_out, int *__restrict__ noncore,
             DevCounters *ctr) {
    if (run_failed(ctr)) return;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    // trip count rounded up to whole warps so the ballot below is warp-uniform
    const int stride = gridDim.x * blockDim.x;
    const int nr = (P.n + 31) & ~31;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += stride) {
        bool nc = false;
        if (i < P.n) {
            const int o = orig[i];
            const int cf = core_s[i];
            core_out[o] = (uint8_t)cf;
            if (cf) {
                const int c = cell_of[i];
                labels_out[o] = compmin[parent[c]] - P.inst[inst_of_cell(P, c)].row0;
            }
            nc = !cf;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, nc);
        if (bal) {
            int base = 0;
            if (lane == 0) base = atomicAdd(&ctr->n_noncore, __popc(bal));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (nc) noncore[base + __popc(bal & lt)] = i;
        }
    }
}

void launch_labels(const RunParams &P, const Bufs &B, uint8_t *core_out, int32_t *labels_out,
                   DevCounters *ctr, cudaStream_t s) {
    launch_uf_compress(B.parent, ctr, P.max_iters, s);
    int g = grid_for((const void *)k_uf_roots, 256);
    k_uf_roots<<<g, 256, 0, s>>>(B.parent, B.compmin, ctr, P.max_iters); count_launch();
    g = grid_for((const void *)k_uf_flatten, 256);
    k_uf_flatten<<<g, 256, 0, s>>>(B.parent, B.compmin, ctr); count_launch();
    g = grid_for((const void *)k_comp_min, 256);
    k_comp_min<<<g, 256, 0, s>>>(B.ccs, B.core_orig, B.parent, B.compmin, ctr); count_launch();
    g = grid_for((const void *)k_label_core, 256);
    // border counts start at zero (core points keep it); ClusterBorder writes the others
    cudaMemsetAsync(B.bcount, 0, sizeof(long long) * (size_t)P.n, s);
    k_label_core<<<g, 256, 0, s>>>(P, B.core_s, B.orig, B.cell_of, B.parent, B.compmin, core_out, labels_out,
                                   B.noncore, ctr);
    count_launch();
}

// ----------------------------------------------------------------- witnesses
// The link witnesses of a run in input indices.  rep[o] for every core point
// (input index o): the input index of the first core point of its cell (any
// two points of one cell are within eps, Sec. 3); links[2i], links[2i+1]: the
// pair recorded for hook i of the union-find.
__global__ void __launch_bounds__(256)
k_witness_export(const int *__restrict__ ccs, const int *__restrict__ core_orig, const int *__restrict__ core_cell,
                 int n_core, const int2 *__restrict__ wit, long long nwit, int32_t *__restrict__ rep,
                 int32_t *__restrict__ links) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n_core; k += stride)
        rep[core_orig[k]] = core_orig[ccs[core_cell[k]]];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nwit; i += stride) {
        const int2 w = wit[i];
        links[2 * i] = core_orig[w.x];
        links[2 * i + 1] = core_orig[w.y];
    }
}

void launch_witness_export(const Bufs &B, int n_core, const int2 *wit, long long nwit, int32_t *rep,
                           int32_t *links, cudaStream_t s) {
    const int g = grid_for((const void *)k_witness_export, 256);
    k_witness_export<<<g, 256, 0, s>>>(B.ccs, B.core_orig, B.core_cell, n_core, wit, nwit, rep, links);
    count_launch();
}

// ----------------------------------------------------------------- border
// ClusterBorder (Algorithm 4): a non-core point p of cell g joins the cluster
// of every cell h in {g} and NeighborCells(g) that has a core point within eps
// of p.  One warp per non-core point; the core points of h are tested 32 at a
// time and h's scan stops at its first hit; h is skipped when its cluster is
// already in p's set.  The set is kept sorted in shared memory.  The core
// points of distinct clusters seen by p are pairwise farther than eps apart
// and all within eps of p, so there are at most kissing-number many of them
// (240 in R^8), under kBorderSetCap.
//
// The count pass (inside the run) keeps every set of at most 2 names in
// bcache and lists the other points (the "heavy" ones) in bheavy; the fill
// pass (dbscan_border_ids) copies the cached sets with one thread per point
// and recomputes only the heavy points, with this kernel.
constexpr int BD_THREADS = 256, BD_WARPS = BD_THREADS / 32;

__device__ __forceinline__ void note_heavy(const Bufs &B, DevCounters *ctr, int t) {
    const int k = atomicAdd(&ctr->n_heavy, 1);
    B.bheavy[k] = t;  // k < n_noncore <= N
}

template <int D, int M, bool FILL>
__global__ void __launch_bounds__(BD_THREADS, D <= 4 ? 8 : 6)  // 64 (d <= 4) or 48 warps per SM (measured faster than 40, 48 / than unbounded)
k_border(RunParams P, Bufs B, int32_t *__restrict__ labels_out, int32_t *__restrict__ ids,
         long long ids_cap, DevCounters *ctr) {
    if (run_failed(ctr)) return;
    __shared__ int sset[BD_WARPS][kBorderSetCap];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nn = FILL ? ctr->n_heavy : ctr->n_noncore;
    unsigned rech = 0;
    unsigned long long evals = 0, nborder = 0, members = 0;
    for (int u0 = warp_id_global(); u0 < nn; u0 += warps_global()) {
        const int t = FILL ? B.bheavy[u0] : u0;
        const int i = B.noncore[t];
        const int g = B.cell_of[i];
        const int o = B.orig[i];
        // the count pass leaves the points of small cells to k_border_small,
        // unless their set overflowed there
        if (!FILL && P.mc_small_nbr > 0 &&
            mc_small(P, B.cell_start[g + 1] - B.cell_start[g], B.nbr_pts, g) && !B.bbig[o])
            continue;
        const Inst &I = P.inst[inst_of_cell(P, g)];
        const Thr T = I.thr;
        const int row0 = I.row0;
        Pt<D, M> p;
        load_pt(p, B.pf, B.pd, i);
        int ns = 0;
        const int ne = B.nbr_cnt[g];
        const int *nl = nbr_list<D>(B.nbr, B.nbr_off, B.nbr_stride, g);
        for (int e = -1; e < ne; ++e) {
            const int h = e < 0 ? g : nl[e];
            const int k0 = B.ccs[h], k1 = B.ccs[h + 1];
            if (k0 == k1) continue;
            const int L = B.compmin[B.parent[h]] - row0;
            bool have = false;
            for (int u = lane; u < ns; u += 32) have = have || sset[w][u] == L;
            if (__any_sync(0xffffffffu, have)) continue;
            bool found = false;
            if constexpr (M == kF32FromF32 || M == kF32FromF64) {
                if (P.box && P.pair_box) {
                    const Bx<D> lo = load_box<D>(B.cblo, h), hi = load_box<D>(B.cbhi, h);
                    if (box_min_d2<D>(p.f, lo, hi) > T.hi) continue;  // no core point of h within eps
                    found = box_max_d2<D>(p.f, lo, hi) <= T.lo;      // every core point of h within eps
                }
            }
            for (int kb = k0; kb < k1 && !found; kb += 32) {
                const int k = kb + lane;
                bool hit = false;
                if (k < k1) {
                    Pt<D, M> q;
                    load_pt(q, B.cpf, B.cpd, k);
                    if (P.stats) ++evals;
                    hit = within(p, q, T, B.pd, i, B.cpd, k, rech);
                }
                found = __any_sync(0xffffffffu, hit);
            }
            if (found) {
                if (ns < kBorderSetCap) {
                    if (lane == 0) {
                        int u = ns;
                        while (u > 0 && sset[w][u - 1] > L) { sset[w][u] = sset[w][u - 1]; --u; }
                        sset[w][u] = L;
                    }
                    ++ns;
                } else if (lane == 0) {
                    set_error(ctr, DBSCAN_ERR_CAPACITY, 30);
                }
                __syncwarp();
            }
        }
        if (!FILL) {
            if (lane == 0) {
                B.bcount[o] = ns;
                labels_out[o] = ns ? sset[w][0] : -1;
                if (ns <= 2) B.bcache[o] = make_int2(ns > 0 ? sset[w][0] : -1, ns > 1 ? sset[w][1] : -1);
                else note_heavy(B, ctr, t);
            }
            nborder += ns ? 1 : 0;
            members += ns;
        } else {
            const long long at = B.boff[o];
            if (at + ns <= ids_cap) {
                for (int u = lane; u < ns; u += 32) ids[at + u] = sset[w][u];
            } else if (lane == 0) {
                set_error(ctr, DBSCAN_ERR_CAPACITY, 31);
            }
        }
        __syncwarp();
    }
    if (!FILL) {
        flush_counter(&ctr->band_rechecks, rech);
        if (P.stats) flush_counter(&ctr->dist_evals[2], evals);
        if (lane == 0 && nborder) atomicAdd((unsigned *)&ctr->n_border, (unsigned)nborder);
        if (lane == 0 && members) atomicAdd((unsigned long long *)&ctr->K, members);  // total set length
    }
}

// Fill pass, cached part: the sets of at most 2 names kept by the count pass,
// one thread per non-core point.
__global__ void __launch_bounds__(256)
k_border_fill_cached(Bufs B, int32_t *__restrict__ ids, long long ids_cap, DevCounters *ctr) {
    if (run_failed(ctr)) return;
    const int nn = ctr->n_noncore;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nn; t += gridDim.x * blockDim.x) {
        const int o = B.orig[B.noncore[t]];
        const long long ns = B.bcount[o];
        if (ns == 0 || ns > 2) continue;
        const long long at = B.boff[o];
        if (at + ns > ids_cap) {
            set_error(ctr, DBSCAN_ERR_CAPACITY, 33);
            continue;
        }
        const int2 cs = B.bcache[o];
        ids[at] = cs.x;
        if (ns > 1) ids[at + 1] = cs.y;
    }
}

// CSR offsets of the border sets: exclusive scan of the per-point counts.
void launch_border_offsets(const RunParams &P, const Bufs &B, cudaStream_t s) {
    scan_i64_to_i64(B.bcount, B.boff, P.n, nullptr, P.n, B.part, s);
}

// ClusterBorder's count pass for the non-core points of small cells (the cells
// k_markcore_small takes): one thread per point, the set of cluster names in
// registers (up to kSmallSet, sorted).  A point whose set would grow beyond
// that is flagged in bbig and left to k_border.
constexpr int kSmallSet = 8;

template <int D, int M>
__global__ void __launch_bounds__(256, 5)  // 40 warps per SM (measured faster than 32)
k_border_small(RunParams P, Bufs B, int32_t *__restrict__ labels_out, DevCounters *ctr) {
    if (run_failed(ctr)) return;
    constexpr bool BOX = (M == kF32FromF32 || M == kF32FromF64);
    const int nn = ctr->n_noncore;
    unsigned rech = 0;
    unsigned long long evals = 0, nborder = 0, members = 0;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nn; t += gridDim.x * blockDim.x) {
        const int i = B.noncore[t];
        const int g = B.cell_of[i];
        const int o = B.orig[i];
        if (!mc_small(P, B.cell_start[g + 1] - B.cell_start[g], B.nbr_pts, g)) continue;
        const Inst &I = P.inst[inst_of_cell(P, g)];
        const Thr T = I.thr;
        const int row0 = I.row0;
        Pt<D, M> p;
        load_pt(p, B.pf, B.pd, i);
        int set[kSmallSet];
        int ns = 0;
        bool big = false;
        const int ne = B.nbr_cnt[g];
        const int *nl = nbr_list<D>(B.nbr, B.nbr_off, B.nbr_stride, g);
        for (int e = -1; e < ne && !big; ++e) {
            const int h = e < 0 ? g : nl[e];
            const int k0 = B.ccs[h], k1 = B.ccs[h + 1];
            if (k0 == k1) continue;
            const int L = B.compmin[B.parent[h]] - row0;
            bool have = false;
            for (int u = 0; u < ns; ++u) have = have || set[u] == L;
            if (have) continue;
            bool found = false;
            if constexpr (BOX) {
                if (P.box && P.pair_box) {
                    const Bx<D> lo = load_box<D>(B.cblo, h), hi = load_box<D>(B.cbhi, h);
                    if (box_min_d2<D>(p.f, lo, hi) > T.hi) continue;
                    found = box_max_d2<D>(p.f, lo, hi) <= T.lo;
                }
            }
            for (int k = k0; k < k1 && !found; ++k) {
                Pt<D, M> q;
                load_pt(q, B.cpf, B.cpd, k);
                if (P.stats) ++evals;
                found = within(p, q, T, B.pd, i, B.cpd, k, rech);
            }
            if (!found) continue;
            if (ns == kSmallSet) {
                big = true;
                break;
            }
            int u = ns++;
            while (u > 0 && set[u - 1] > L) { set[u] = set[u - 1]; --u; }
            set[u] = L;
        }
        B.bbig[o] = big ? 1 : 0;
        if (big) continue;  // k_border redoes this point
        B.bcount[o] = ns;
        labels_out[o] = ns ? set[0] : -1;
        if (ns <= 2) B.bcache[o] = make_int2(ns > 0 ? set[0] : -1, ns > 1 ? set[1] : -1);
        else note_heavy(B, ctr, t);
        nborder += ns ? 1 : 0;
        members += ns;
    }
    flush_counter(&ctr->band_rechecks, rech);
    if (P.stats) flush_counter(&ctr->dist_evals[2], evals);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nborder += __shfl_xor_sync(0xffffffffu, nborder, o);
    if ((threadIdx.x & 31) == 0 && nborder) atomicAdd((unsigned *)&ctr->n_border, (unsigned)nborder);
    flush_counter((unsigned long long *)&ctr->K, members);
}

void launch_border(int D, int mode, bool fill, const RunParams &P, const Bufs &B, int32_t *labels_out,
                   int32_t *ids, long long ids_cap, DevCounters *ctr, cudaStream_t s, bool offsets) {
    if (!fill) {
        if (P.mc_small_nbr > 0)
            GBDB_DISPATCH(D, mode, {
                auto k = k_border_small<DD, MM>;
                const int g = grid_for((const void *)k, 256);
                k<<<g, 256, 0, s>>>(P, B, labels_out, ctr);
                count_launch();
            });
        GBDB_DISPATCH(D, mode, {
            auto k = k_border<DD, MM, false>;
            int g = grid_for((const void *)k, BD_THREADS);
            k<<<g, BD_THREADS, 0, s>>>(P, B, labels_out, nullptr, 0, ctr);
            count_launch();
        });
        if (offsets) launch_border_offsets(P, B, s);
    } else {
        const int gc = grid_for((const void *)k_border_fill_cached, 256);
        k_border_fill_cached<<<gc, 256, 0, s>>>(B, ids, ids_cap, ctr);
        count_launch();
        GBDB_DISPATCH(D, mode, {
            auto k = k_border<DD, MM, true>;
            int g = grid_for((const void *)k, BD_THREADS);
            k<<<g, BD_THREADS, 0, s>>>(P, B, labels_out, ids, ids_cap, ctr);
            count_launch();
        });
    }
}

}  // namespace gbdb
