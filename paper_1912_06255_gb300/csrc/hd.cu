// Cells and neighbour lists for 5 <= d <= 8.
//
// Enumerating neighbour offsets does not scale with d: the rule
// sum_j max(|delta_j| - 1, 0)^2 <= d admits 6,095 offsets in 5D and 257,675
// in 7D, almost all of them empty cells.  Sec. 5.1 therefore finds the
// neighbouring cells of high-dimensional inputs with a spatial tree over the
// non-empty cells.  This file builds that tree the GPU way:
//   1. every point gets a 128-bit Morton key of its cell coordinates (at most
//      15 bits per dimension);
//   2. a stable LSD radix sort orders the points by key (low word, then high
//      word), which groups them by cell and lays the cells out in Z order;
//   3. a linear BVH over the cells in that order (each internal node splits at
//      the highest differing key bit, built for all nodes at once), with
//      integer cell-coordinate bounds set bottom-up;
//   4. one packet walk per 32 Z-ordered cells lists the cells that satisfy
//      the offset rule exactly (integer arithmetic), at CSR offsets reserved
//      per packet, cells at |delta|_inf <= 1 first.
#include <cuda_runtime.h>

#include <algorithm>
#include <initializer_list>

#include "geom.cuh"
#include "grid.cuh"

namespace gbdb {

namespace {

// Stack of the tree walks: a depth-first walk that pushes at most both
// children of a node keeps at most one pending node per level of the tree
// (at most key bits + 1 levels); the bound leaves a 4x margin.
constexpr int kStack = 4 * 132;

// Cell coordinates are packed as 8 unsigned 16-bit values in an int4
// (component k holds dimensions 2k and 2k + 1).
__device__ __forceinline__ int unpack16(const int4 &v, int j) {
    const int w = (j >> 1) == 0 ? v.x : ((j >> 1) == 1 ? v.y : ((j >> 1) == 2 ? v.z : v.w));
    return (j & 1) ? ((unsigned)w >> 16) : (w & 0xffff);
}
__device__ __forceinline__ int4 pack16(const int (&c)[8]) {
    return make_int4(c[0] | (c[1] << 16), c[2] | (c[3] << 16), c[4] | (c[5] << 16), c[6] | (c[7] << 16));
}

// Bit b of dimension j goes to key bit b*d + j of the 128-bit key (hi:lo).
__device__ __forceinline__ void morton128(const int (&c)[8], int d, int bits, uint64_t &lo, uint64_t &hi) {
    lo = 0;
    hi = 0;
    for (int b = 0; b < bits; ++b)
        for (int j = 0; j < d; ++j) {
            const uint64_t bit = (uint64_t)((c[j] >> b) & 1);
            const int p = b * d + j;
            if (p < 64) lo |= bit << p;
            else hi |= bit << (p - 64);
        }
}

__device__ __forceinline__ void unmorton128(uint64_t lo, uint64_t hi, int d, int bits, int (&c)[8]) {
#pragma unroll
    for (int j = 0; j < 8; ++j) c[j] = 0;
    for (int b = 0; b < bits; ++b)
        for (int j = 0; j < d; ++j) {
            const int p = b * d + j;
            const int bit = (int)((p < 64 ? (lo >> p) : (hi >> (p - 64))) & 1);
            c[j] |= bit << b;
        }
}

template <typename T>
__global__ void __launch_bounds__(256)
k_hd_keys(const T *__restrict__ X, RunParams P, uint64_t *__restrict__ klo, uint64_t *__restrict__ khi,
          uint64_t *__restrict__ k0, uint32_t *__restrict__ v0, unsigned *__restrict__ qsub) {
    const Inst &I = P.inst[0];
    const int L = P.qt;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += gridDim.x * blockDim.x) {
        int c[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) c[j] = j < P.d ? cell_coord<T>(X[(int64_t)i * P.d + j], I, j) : 0;
        uint64_t lo, hi;
        morton128(c, P.d, I.bits, lo, hi);
        klo[i] = lo;
        khi[i] = hi;
        if (L > 0) {
            // quadtree sub-cell of the point, L levels below its cell, Morton
            // interleaved with the coarsest level in the top bits; only the
            // grouping matters (node boxes bound the points), so FP32 suffices
            unsigned q = 0;
            for (int j = 0; j < P.d; ++j) {
                const float t = ((float)X[(int64_t)i * P.d + j] - I.origin32[j]) * I.inv_s32;
                int u = (int)floorf(t * (float)(1 << L)) - (c[j] << L);
                u = u < 0 ? 0 : (u >= (1 << L) ? (1 << L) - 1 : u);
                for (int b = 0; b < L; ++b) q |= (unsigned)((u >> b) & 1) << (b * P.d + j);
            }
            qsub[i] = q;
            k0[i] = q;
        } else {
            k0[i] = lo;
        }
        v0[i] = (uint32_t)i;
    }
}

// kh[t] = khi[idx[t]]: a key word in the order of the previous sort pass.
__global__ void __launch_bounds__(256)
k_hd_gather_hi(const uint64_t *__restrict__ khi, const uint32_t *__restrict__ idx, uint64_t *__restrict__ kh, int n,
               const DevCounters *ctr) {
    if (run_failed(ctr)) return;  // the sort gave up: idx is incomplete
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) kh[t] = khi[idx[t]];
}

// flag[t] = 1 where a new cell starts in the sorted order.
__global__ void __launch_bounds__(256)
k_hd_flags(const uint64_t *__restrict__ klo, const uint64_t *__restrict__ khi, const uint32_t *__restrict__ idx,
           int *__restrict__ flag, int n, const DevCounters *ctr) {
    if (run_failed(ctr)) return;  // the sort gave up: idx is incomplete
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        int f = 1;
        if (t > 0) {
            const uint32_t a = idx[t], b = idx[t - 1];
            f = (klo[a] != klo[b] || khi[a] != khi[b]) ? 1 : 0;
        }
        flag[t] = f;
    }
}

// Cells in sorted order: cell ids, starts, keys and coordinates; the points
// move to cell order (FP32 copy zero-padded to 8, FP64 copy when kept).
template <typename T>
__global__ void __launch_bounds__(256)
k_hd_cells(const T *__restrict__ X, RunParams P, const uint32_t *__restrict__ idx, const uint64_t *__restrict__ klo,
           const uint64_t *__restrict__ khi, const unsigned *__restrict__ qsub_in, unsigned *__restrict__ qsub,
           const int *__restrict__ flag, const int *__restrict__ cpos,
           int *__restrict__ cell_start, uint64_t *__restrict__ ckey_lo, uint64_t *__restrict__ ckey_hi,
           int4 *__restrict__ ccoord, float *__restrict__ pf, double *__restrict__ pd, int *__restrict__ orig,
           int *__restrict__ cell_of, DevCounters *ctr) {
    if (run_failed(ctr)) return;
    const int n = P.n, d = P.d;
    const Inst &I = P.inst[0];
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const int i = (int)idx[t];
        const int f = flag[t];
        const int c = cpos[t] + f - 1;
        orig[t] = i;
        cell_of[t] = c;
        if (qsub) qsub[t] = qsub_in[i];
        float x32[8];
        double x64[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            x64[j] = j < d ? (double)X[(int64_t)i * d + j] : 0.0;
            x32[j] = (float)x64[j];
        }
        reinterpret_cast<float4 *>(pf)[(int64_t)t * 2] = make_float4(x32[0], x32[1], x32[2], x32[3]);
        reinterpret_cast<float4 *>(pf)[(int64_t)t * 2 + 1] = make_float4(x32[4], x32[5], x32[6], x32[7]);
        if (pd) {
#pragma unroll
            for (int j = 0; j < 8; j += 2)
                reinterpret_cast<double2 *>(pd)[(int64_t)t * 4 + j / 2] = make_double2(x64[j], x64[j + 1]);
        }
        if (f) {
            const uint64_t lo = klo[i], hi = khi[i];
            cell_start[c] = t;
            ckey_lo[c] = lo;
            ckey_hi[c] = hi;
            int cc[8];
            unmorton128(lo, hi, d, I.bits, cc);
            ccoord[c] = pack16(cc);
        }
        if (t == 0) {
            const int m = cpos[n];
            ctr->m = m;
            cell_start[m] = n;
        }
    }
}

// ------------------------------------------------------------------ LBVH
// Nodes 0 .. m-2 are internal (node 0 is the root), node m-1+c is the leaf of
// cell c.  Internal node i covers a key range with i at one end; its other end
// and its split are found by binary search over common-prefix lengths.
__device__ __forceinline__ int prefix(const uint64_t *__restrict__ lo, const uint64_t *__restrict__ hi, int m, int i,
                                      long long j) {
    if (j < 0 || j >= m) return -1;
    const uint64_t a = hi[i] ^ hi[j];
    if (a) return __clzll((long long)a);
    return 64 + __clzll((long long)(lo[i] ^ lo[j]));  // keys are distinct
}

__global__ void __launch_bounds__(256)
k_lbvh_nodes(const uint64_t *__restrict__ klo, const uint64_t *__restrict__ khi, int2 *__restrict__ child,
             int *__restrict__ parent, int *__restrict__ flag, int *__restrict__ nmax, const DevCounters *ctr) {
    if (run_failed(ctr)) return;
    const int m = ctr->m;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m - 1; i += gridDim.x * blockDim.x) {
        flag[i] = 0;
        const int dir = prefix(klo, khi, m, i, i + 1) > prefix(klo, khi, m, i, i - 1) ? 1 : -1;
        const int dmin = prefix(klo, khi, m, i, i - dir);
        long long lmax = 2;
        while (lmax <= m && prefix(klo, khi, m, i, i + lmax * dir) > dmin) lmax <<= 1;
        long long l = 0;
        for (long long t = lmax >> 1; t >= 1; t >>= 1)
            if (prefix(klo, khi, m, i, i + (l + t) * dir) > dmin) l += t;
        const int j = (int)(i + l * dir);
        const int dnode = prefix(klo, khi, m, i, j);
        long long s = 0;
        for (long long t = (l + 1) >> 1;; t = (t + 1) >> 1) {
            if (prefix(klo, khi, m, i, i + (s + t) * dir) > dnode) s += t;
            if (t <= 1) break;
        }
        const int g = (int)(i + s * dir + (dir < 0 ? -1 : 0));
        const int lo = i < j ? i : j, hi = i < j ? j : i;
        const int left = lo == g ? (m - 1) + g : g;
        const int right = hi == g + 1 ? (m - 1) + g + 1 : g + 1;
        child[i] = make_int2(left, right);
        nmax[i] = hi;  // the node covers the cells lo .. hi
        parent[left] = i;
        parent[right] = i;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) parent[0] = -1;  // the root (or the only leaf when m == 1)
}

// Bounds bottom-up: a leaf's thread climbs while it is the second child to
// arrive at the parent (atomic counter), so each node is merged once, after
// both children are final.
__global__ void __launch_bounds__(256)
k_lbvh_bounds(const int2 *__restrict__ child, const int *__restrict__ parent, int *__restrict__ flag,
              const int4 *__restrict__ ccoord, int4 *__restrict__ nlo, int4 *__restrict__ nhi, int d,
              const float4 *__restrict__ blo, const float4 *__restrict__ bhi, float4 *__restrict__ nblo,
              float4 *__restrict__ nbhi, DevCounters *ctr) {
    if (run_failed(ctr)) return;
    const int m = ctr->m;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x) {
        int node = (m - 1) + c;
        for (int it = 0;; ++it) {
            if (it > kStack) {
                set_error(ctr, DBSCAN_ERR_CAPACITY, 71);
                break;
            }
            const int p = m > 1 ? parent[node] : -1;
            if (p < 0) break;
            __threadfence();
            if (atomicAdd(flag + p, 1) == 0) break;  // the sibling's subtree is not finished yet
            __threadfence();
            const int2 ch = child[p];
            int lo[8], hi[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) { lo[j] = 0x7fffffff; hi[j] = 0; }
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int q = k ? ch.y : ch.x;
                int4 a, b;
                if (q >= m - 1) {
                    a = b = ccoord[q - (m - 1)];
                } else {
                    a = __ldcg(nlo + q);
                    b = __ldcg(nhi + q);
                }
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    lo[j] = min(lo[j], unpack16(a, j));
                    hi[j] = max(hi[j], unpack16(b, j));
                }
            }
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if (j >= d) lo[j] = hi[j] = 0;
            __stcg(nlo + p, pack16(lo));
            __stcg(nhi + p, pack16(hi));
            if (nblo) {
                // point boxes: the union of the children's (cells' or nodes') boxes
                float4 l0 = make_float4(INFINITY, INFINITY, INFINITY, INFINITY), l1 = l0;
                float4 h0 = make_float4(-INFINITY, -INFINITY, -INFINITY, -INFINITY), h1 = h0;
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const int q = k ? ch.y : ch.x;
                    float4 a0, a1, b0, b1;
                    if (q >= m - 1) {
                        const int64_t cq = q - (m - 1);
                        a0 = blo[cq * 2]; a1 = blo[cq * 2 + 1];
                        b0 = bhi[cq * 2]; b1 = bhi[cq * 2 + 1];
                    } else {
                        a0 = __ldcg(nblo + (int64_t)q * 2); a1 = __ldcg(nblo + (int64_t)q * 2 + 1);
                        b0 = __ldcg(nbhi + (int64_t)q * 2); b1 = __ldcg(nbhi + (int64_t)q * 2 + 1);
                    }
                    l0 = make_float4(fminf(l0.x, a0.x), fminf(l0.y, a0.y), fminf(l0.z, a0.z), fminf(l0.w, a0.w));
                    l1 = make_float4(fminf(l1.x, a1.x), fminf(l1.y, a1.y), fminf(l1.z, a1.z), fminf(l1.w, a1.w));
                    h0 = make_float4(fmaxf(h0.x, b0.x), fmaxf(h0.y, b0.y), fmaxf(h0.z, b0.z), fmaxf(h0.w, b0.w));
                    h1 = make_float4(fmaxf(h1.x, b1.x), fmaxf(h1.y, b1.y), fmaxf(h1.z, b1.z), fmaxf(h1.w, b1.w));
                }
                __stcg(nblo + (int64_t)p * 2, l0);
                __stcg(nblo + (int64_t)p * 2 + 1, l1);
                __stcg(nbhi + (int64_t)p * 2, h0);
                __stcg(nbhi + (int64_t)p * 2 + 1, h1);
            }
            node = p;
        }
    }
}

// Two 16-bit lanes per 32-bit word (the packed cell coordinates): unsigned
// maximum and minimum per lane, and the sum of the squares of two lane values
// below 128 added to s (a two-way dot product of the word with its own low
// bytes).  Coordinates are below 2^15, so a difference biased by 2^15 stays
// inside its lane: with x = a - b + 0x80008000 each lane holds a - b + 2^15.
__device__ __forceinline__ unsigned vmax_u16x2(unsigned a, unsigned b) {
    unsigned r;
    asm("max.u16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}
__device__ __forceinline__ unsigned vmin_u16x2(unsigned a, unsigned b) {
    unsigned r;
    asm("min.u16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
    return r;
}
__device__ __forceinline__ int add_sq2(unsigned t, int s) { return __dp2a_lo((int)t, (int)(t | (t >> 8)), s); }
__device__ __forceinline__ unsigned word(const int4 &v, int k) {
    return (unsigned)(k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w)));
}

// Smallest sum over the node of max(|delta_j| - 1, 0)^2 against the packed
// cell coordinates c, each term capped at 81 (any term above 8 already fails).
// Unused dimensions are zero in c and in the bounds and add nothing.
template <int DD>
__device__ __forceinline__ int gap2(const int4 &c, const int4 &lo, const int4 &hi) {
    int s = 0;
#pragma unroll
    for (int k = 0; k < (DD + 1) / 2; ++k) {
        const unsigned x = word(lo, k) - word(c, k) + 0x7fff7fffu;  // lo - c - 1, biased
        const unsigned y = word(c, k) - word(hi, k) + 0x7fff7fffu;  // c - hi - 1, biased
        const unsigned g = vmin_u16x2(vmax_u16x2(vmax_u16x2(x, y), 0x80008000u), 0x80098009u) - 0x80008000u;
        s = add_sq2(g, s);
    }
    return s;
}

// NeighborCells(g) for every cell g (Algorithm 2), as a packet traversal: a
// warp walks the tree once for 32 consecutive cells in Z order (one per
// lane), which are close in space and so share most of the walk.  A node is
// entered when it may hold a neighbour of any lane's cell; at a leaf every
// lane applies the exact offset rule to its own cell.  In the FP32-band mode
// nodes and cells whose point boxes are farther than eps apart are skipped,
// as in the enumeration of low dimensions.
//
// One walk per packet: the leaves that pass for some lane go to the warp's
// scratch (kScr entries in global memory, each the leaf and the masks of the
// lanes that found it adjacent or farther), each lane counts its own, the
// packet reserves its lists' space with one atomic on ctr->E, and the lanes
// then fill their lists from the scratch, cells at |delta|_inf <= 1 first.
// A packet whose leaves overflow the scratch walks the tree a second time to
// fill.  Space beyond cap is not written: the host sees ctr->E > cap, grows
// the list buffer and runs the kernel again.
constexpr int QW = 4;         // warps per block of the query
constexpr int kScr = 8192;    // scratch entries (16 bytes each) per warp

struct Walk {
    int4 c;  // packed cell coordinates
    Bx<8> glo, ghi;
    int g;
    bool valid;
};

// Smallest squared distance between two 8-wide boxes over their first DD
// dimensions (the others are zero in both).
template <int DD>
__device__ __forceinline__ float boxes_min_d2_dd(const Bx<8> &alo, const Bx<8> &ahi, const Bx<8> &blo,
                                                 const Bx<8> &bhi) {
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < DD; ++j) {
        const float a = fmaxf(fmaxf(bget<8>(blo, j) - bget<8>(ahi, j), bget<8>(alo, j) - bget<8>(bhi, j)), 0.f);
        s = j == 0 ? a * a : __fmaf_rn(a, a, s);
    }
    return s;
}

// The leaf test of one lane: offset rule (exact, integers), then the boxes.
template <int DD>
__device__ __forceinline__ int leaf_test(const Walk &W, int h, const int4 *__restrict__ ccoord, bool box,
                                         const float4 *__restrict__ blo, const float4 *__restrict__ bhi,
                                         float hi_thr) {
    if (!W.valid || h <= W.g) return 0;  // each unordered pair once: from the lower cell
    const int4 ch4 = ccoord[h];
    unsigned a = 0;
    int s = 0;
#pragma unroll
    for (int k = 0; k < (DD + 1) / 2; ++k) {
        const unsigned dd = vmax_u16x2(word(ch4, k) - word(W.c, k) + 0x80008000u,
                                       word(W.c, k) - word(ch4, k) + 0x80008000u);  // |delta| + 2^15
        a = vmax_u16x2(a, dd);
        s = add_sq2(vmin_u16x2(vmax_u16x2(dd, 0x80018001u) - 0x80018001u, 0x00090009u), s);
    }
    const int inf = (int)max(a & 0xffffu, a >> 16) - 32768;
    if (s > DD) return 0;
    if (box && boxes_min_d2_dd<DD>(W.glo, W.ghi, load_box<8>(blo, h), load_box<8>(bhi, h)) > hi_thr) return 0;
    return inf <= 1 ? 1 : 2;  // 1: adjacent, 2: farther
}

// The walk of one packet.  EMIT: write each lane's hits at its list cursors;
// otherwise append the leaves that pass for some lane to scr (up to kScr;
// *ncand counts them all) and count each lane's hits.
template <int DD, bool EMIT>
__device__ __forceinline__ void walk(const Walk &W, int m, bool box, float hi_thr, int *stk,
                                     const int2 *__restrict__ child, const int *__restrict__ nmax,
                                     const int4 *__restrict__ nlo,
                                     const int4 *__restrict__ nhi, const float4 *__restrict__ nblo,
                                     const float4 *__restrict__ nbhi, const int4 *__restrict__ ccoord,
                                     const float4 *__restrict__ blo, const float4 *__restrict__ bhi, int *scr,
                                     int &ncand, int &n_near, int &n_far, int *nbr, long long &near_at,
                                     long long &far_at, DevCounters *ctr) {
    const int lane = threadIdx.x & 31;
    int sp = 0;
    if (m > 1) {
        if (lane == 0) stk[0] = 0;
        sp = 1;
    }
    __syncwarp();
    while (sp > 0) {
        const int node = stk[--sp];
        __syncwarp();
        const int2 ch = child[node];
#pragma unroll
        for (int k = 1; k >= 0; --k) {  // the right child pushed first, so the left one is popped first
            const int q = k ? ch.y : ch.x;
            if (q >= m - 1) {
                const int h = q - (m - 1);
                const int t = leaf_test<DD>(W, h, ccoord, box, blo, bhi, hi_thr);
                if (EMIT) {
                    if (t == 1) nbr[near_at++] = h;
                    else if (t == 2) nbr[far_at++] = h;
                } else {
                    if (t == 1) ++n_near;
                    else if (t == 2) ++n_far;
                    const unsigned near_m = __ballot_sync(0xffffffffu, t == 1);
                    const unsigned far_m = __ballot_sync(0xffffffffu, t == 2);
                    if (near_m | far_m) {
                        if (lane == 0 && ncand < kScr) reinterpret_cast<int4 *>(scr)[ncand] =
                            make_int4(h, (int)near_m, (int)far_m, 0);
                        ++ncand;
                    }
                }
            } else {
                // only subtrees holding a cell after the lane's own (forward pairs)
                bool enter = W.valid && nmax[q] > W.g && gap2<DD>(W.c, nlo[q], nhi[q]) <= DD;
                if (enter && box)
                    enter = boxes_min_d2_dd<DD>(W.glo, W.ghi, load_box<8>(nblo, q), load_box<8>(nbhi, q)) <= hi_thr;
                if (__any_sync(0xffffffffu, enter)) {
                    if (sp < kStack) {
                        if (lane == 0) stk[sp] = q;
                        ++sp;
                    } else if (lane == 0) {
                        set_error(ctr, DBSCAN_ERR_CAPACITY, 72);
                    }
                }
            }
        }
        __syncwarp();
    }
}

template <int DD>
__global__ void __launch_bounds__(32 * QW)
k_lbvh_neighbors(RunParams P, const int2 *__restrict__ child, const int *__restrict__ nmax,
                 const int4 *__restrict__ nlo, const int4 *__restrict__ nhi, const float4 *__restrict__ nblo,
                 const float4 *__restrict__ nbhi, const int4 *__restrict__ ccoord, const float4 *__restrict__ blo,
                 const float4 *__restrict__ bhi, int *__restrict__ scratch, int *__restrict__ fn,
                 int *__restrict__ ff, long long *__restrict__ off, int *__restrict__ nbr, long long cap,
                 long long max_warps, DevCounters *ctr) {
    if (run_failed(ctr)) return;
    __shared__ int stk[QW][kStack];
    if (warps_global() > max_warps) {  // the scratch has no room for this grid (cannot happen: sized for the largest)
        if (threadIdx.x == 0 && blockIdx.x == 0) set_error(ctr, DBSCAN_ERR_CAPACITY, 73);
        return;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int m = ctr->m;
    const bool box = P.box != 0;
    const float hi_thr = P.inst[0].cthr.hi;  // eps, or eps(1 + rho) for approximate connectivity
    int *scr = scratch + (long long)warp_id_global() * kScr * 4;
    const int packets = (m + 31) >> 5;
    for (int pk = warp_id_global(); pk < packets; pk += warps_global()) {
        Walk W;
        W.g = pk * 32 + lane;
        W.valid = W.g < m;
        W.c = W.valid ? ccoord[W.g] : make_int4(0, 0, 0, 0);
        W.glo = zero_box<8>();
        W.ghi = W.glo;
        if (box && W.valid) {
            W.glo = load_box<8>(blo, W.g);
            W.ghi = load_box<8>(bhi, W.g);
        }
        int ncand = 0, n_near = 0, n_far = 0;
        long long near_at = 0, far_at = 0;
        walk<DD, false>(W, m, box, hi_thr, stk[w], child, nmax, nlo, nhi, nblo, nbhi, ccoord, blo, bhi, scr, ncand,
                        n_near, n_far, nbr, near_at, far_at, ctr);
        // reserve the packet's space: lane offsets by an exclusive scan of the counts
        const int mine = n_near + n_far;
        int incl = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        unsigned long long base = 0;
        if (lane == 0 && total) base = atomicAdd((unsigned long long *)&ctr->E, (unsigned long long)total);
        base = __shfl_sync(0xffffffffu, base, 0);
        const long long at = (long long)base + (incl - mine);
        if (W.valid) {
            off[W.g] = at;
            fn[W.g] = n_near;
            ff[W.g] = n_far;
        }
        if ((long long)base + total > cap) continue;  // the host grows the buffer and runs again
        near_at = at;
        far_at = at + n_near;
        if (ncand <= kScr) {
            for (int i = 0; i < ncand; ++i) {
                const int4 e = reinterpret_cast<const int4 *>(scr)[i];  // one broadcast load for the warp
                if (((unsigned)e.y >> lane) & 1u) nbr[near_at++] = e.x;
                else if (((unsigned)e.z >> lane) & 1u) nbr[far_at++] = e.x;
            }
        } else {
            walk<DD, true>(W, m, box, hi_thr, stk[w], child, nmax, nlo, nhi, nblo, nbhi, ccoord, blo, bhi, scr,
                           ncand, n_near, n_far, nbr, near_at, far_at, ctr);
        }
        __syncwarp();
    }
}

template <typename T> void hd_launch_keys(const void *X, const RunParams &P, const HdBufs &H, const Bufs &B,
                                       cudaStream_t s) {
    const int g = grid_for((const void *)k_hd_keys<T>, 256);
    k_hd_keys<T><<<g, 256, 0, s>>>((const T *)X, P, H.klo, H.khi, B.sk0, B.sv0, H.qsub_in);
    count_launch();
}

template <typename T> void hd_launch_cells(const void *X, const RunParams &P, const HdBufs &H, const Bufs &B,
                                        const uint32_t *idx, DevCounters *ctr, cudaStream_t s) {
    const int g = grid_for((const void *)k_hd_cells<T>, 256);
    // the cell table and the sorted points are this step's outputs
    k_hd_cells<T><<<g, 256, 0, s>>>((const T *)X, P, idx, H.klo, H.khi, H.qsub_in, P.qt > 0 ? H.qsub : nullptr,
                                    B.core_s, B.core_pos,
                                    const_cast<int *>(B.cell_start), H.ckey_lo, H.ckey_hi, H.ccoord,
                                    const_cast<float *>(B.pf), const_cast<double *>(B.pd),
                                    const_cast<int *>(B.orig), const_cast<int *>(B.cell_of), ctr);
    count_launch();
}

}  // namespace

// Steps 1-2 above: keys, sort, cells.
void hd_cells(const void *X, int dtype, const RunParams &P, int key_bits, const HdBufs &H, const Bufs &B,
              DevCounters *ctr, cudaStream_t s) {
    const int n = P.n;
    const int bits = key_bits;
    if (dtype == DBSCAN_F32) hd_launch_keys<float>(X, P, H, B, s);
    else hd_launch_keys<double>(X, P, H, B, s);
    // stable LSD sort: the quadtree sub-cell key first (when used), then the
    // low word of the cell key, then its high word.  k_hd_keys left the first
    // pass's (key, index) in buffer 0; kc / vc name the buffers that hold the
    // current keys and values, the others are free.
    const int lo_bits = bits < 64 ? bits : 64;
    uint64_t *kbuf[2] = {B.sk0, B.sk1};
    uint32_t *vbuf[2] = {B.sv0, B.sv1};
    int kc = 0, vc = 0;
    auto sort_pass = [&](int nbits) {
        if (radix_sort_u64(kbuf[kc], vbuf[vc], kbuf[kc ^ 1], vbuf[vc ^ 1], n, nullptr, n, 0, nbits, B.sort_scratch,
                           B.sort_scratch_size, ctr, P.max_iters, s)) {
            kc ^= 1;
            vc ^= 1;
        }
    };
    auto regather = [&](const uint64_t *src) {  // the keys of the current order into the free key buffer
        const int g = grid_for((const void *)k_hd_gather_hi, 256);
        k_hd_gather_hi<<<g, 256, 0, s>>>(src, vbuf[vc], kbuf[kc ^ 1], n, ctr);
        count_launch();
        kc ^= 1;
    };
    if (P.qt > 0) {
        sort_pass(P.d * P.qt);
        regather(H.klo);
    }
    sort_pass(lo_bits);
    if (bits > 64) {
        regather(H.khi);
        sort_pass(bits - 64);
    }
    const uint32_t *idx = vbuf[vc];
    {
        int g = grid_for((const void *)k_hd_flags, 256);
        k_hd_flags<<<g, 256, 0, s>>>(H.klo, H.khi, idx, B.core_s, n, ctr);
        count_launch();
    }
    scan_i32_to_i32(B.core_s, B.core_pos, n, nullptr, n, B.part, s);
    if (dtype == DBSCAN_F32) hd_launch_cells<float>(X, P, H, B, idx, ctr, s);
    else hd_launch_cells<double>(X, P, H, B, idx, ctr, s);
}

// ------------------------------------------------------------ quadtree
// The range-counting quadtree of Sec. 5.2, L levels below each cell.  The
// points are sorted by (cell, sub-cell key), so a node of level l (the points
// of one cell whose sub-cell keys share their top d*l bits) is a run of
// consecutive points, and its children are runs inside it.  Per level:
// qpos[t] = the number of level-l nodes that start before point t (so node k
// starts at the point t with qpos[t] = k and qpos[t+1] = k+1), qstart[k] its
// first point (qstart[count] = n), and the FP32 box of its points.
__global__ void __launch_bounds__(256)
k_qt_flags(const int *__restrict__ cell_of, const unsigned *__restrict__ qsub, int shift, int n, int *__restrict__ flag,
           const DevCounters *ctr) {
    if (run_failed(ctr)) return;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x)
        flag[t] = (t == 0 || cell_of[t] != cell_of[t - 1] || (qsub[t] >> shift) != (qsub[t - 1] >> shift)) ? 1 : 0;
}

__global__ void __launch_bounds__(256)
k_qt_nodes(const int *__restrict__ pos, int n, const float *__restrict__ pf, int *__restrict__ qstart,
           float4 *__restrict__ qlo, float4 *__restrict__ qhi, const DevCounters *ctr) {
    if (run_failed(ctr)) return;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t <= n; t += gridDim.x * blockDim.x) {
        if (t == n) {
            qstart[pos[n]] = n;
            continue;
        }
        const int k = pos[t];
        if (pos[t + 1] == k) continue;  // not the first point of its node
        qstart[k] = t;
        int e = t + 1;
        while (e < n && pos[e + 1] == pos[e]) ++e;  // the node's points are [t, e)
        float lo[8], hi[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) { lo[j] = INFINITY; hi[j] = -INFINITY; }
        for (int u = t; u < e; ++u) {
            const float4 a = reinterpret_cast<const float4 *>(pf)[(int64_t)u * 2];
            const float4 b = reinterpret_cast<const float4 *>(pf)[(int64_t)u * 2 + 1];
            const float x[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
            for (int j = 0; j < 8; ++j) { lo[j] = fminf(lo[j], x[j]); hi[j] = fmaxf(hi[j], x[j]); }
        }
        qlo[(int64_t)k * 2] = make_float4(lo[0], lo[1], lo[2], lo[3]);
        qlo[(int64_t)k * 2 + 1] = make_float4(lo[4], lo[5], lo[6], lo[7]);
        qhi[(int64_t)k * 2] = make_float4(hi[0], hi[1], hi[2], hi[3]);
        qhi[(int64_t)k * 2 + 1] = make_float4(hi[4], hi[5], hi[6], hi[7]);
    }
}

static void hd_quadtree(const RunParams &P, const HdBufs &H, const Bufs &B, DevCounters *ctr, cudaStream_t s) {
    const int n = P.n;
    for (int l = 1; l <= P.qt; ++l) {
        int *pos = H.qpos[l - 1];
        int g = grid_for((const void *)k_qt_flags, 256);
        k_qt_flags<<<g, 256, 0, s>>>(B.cell_of, H.qsub, P.d * (P.qt - l), n, pos, ctr);
        count_launch();
        scan_i32_to_i32(pos, pos, n, nullptr, n, B.part, s);
        g = grid_for((const void *)k_qt_nodes, 256);
        k_qt_nodes<<<g, 256, 0, s>>>(pos, n, B.pf, H.qstart[l - 1], H.qlo[l - 1], H.qhi[l - 1], ctr);
        count_launch();
    }
}

// Step 3: the cells' point boxes, the tree over the cells, and the
// quadtrees of the cells when MarkCore counts with them.
void hd_tree(const RunParams &P, const HdBufs &H, const Bufs &B, DevCounters *ctr, cudaStream_t s) {
    if (P.qt > 0) hd_quadtree(P, H, B, ctr, s);
    if (P.box) launch_boxes(8, B.pf, B.cell_start, ctr, const_cast<float4 *>(B.blo), const_cast<float4 *>(B.bhi), s);
    int g = grid_for((const void *)k_lbvh_nodes, 256);
    k_lbvh_nodes<<<g, 256, 0, s>>>(H.ckey_lo, H.ckey_hi, H.child, H.parent, H.flag, H.nmax, ctr);
    count_launch();
    g = grid_for((const void *)k_lbvh_bounds, 256);
    k_lbvh_bounds<<<g, 256, 0, s>>>(H.child, H.parent, H.flag, H.ccoord, H.nlo, H.nhi, P.d, B.blo, B.bhi,
                                    P.box ? H.nblo : nullptr, P.box ? H.nbhi : nullptr, ctr);
    count_launch();
}

// Warps of the neighbour kernel's largest grid (no blocks-per-SM cap): the
// scratch holds kScr entries for each.
static long long hd_max_warps() {
    const int cap = grid_cap();
    set_grid_cap(0);
    long long w = 0;
    for (const void *k : {(const void *)k_lbvh_neighbors<5>, (const void *)k_lbvh_neighbors<6>,
                          (const void *)k_lbvh_neighbors<7>, (const void *)k_lbvh_neighbors<8>})
        w = std::max(w, (long long)grid_for(k, 32 * QW) * QW);
    set_grid_cap(cap);
    return w;
}
long long hd_scratch_ints() { return hd_max_warps() * kScr * 4; }

// Step 4: the neighbour lists into nbr (cap entries); ctr->E must be 0 before.
void hd_neighbors(const RunParams &P, const HdBufs &H, const Bufs &B, int *fwd, long long cap, DevCounters *ctr,
                  cudaStream_t s) {
    const long long maxw = hd_max_warps();
    auto go = [&](auto k) {
        const int g = grid_for((const void *)k, 32 * QW);
        k<<<g, 32 * QW, 0, s>>>(P, H.child, H.nmax, H.nlo, H.nhi, H.nblo, H.nbhi, H.ccoord, B.blo, B.bhi, H.scratch,
                                H.fn, H.ff, H.fwd_off, fwd, cap, maxw, ctr);
    };
    // one instantiation per dimension: the offset and box tests cover only the used coordinates
    switch (P.d) {
    case 5: go(k_lbvh_neighbors<5>); break;
    case 6: go(k_lbvh_neighbors<6>); break;
    case 7: go(k_lbvh_neighbors<7>); break;
    default: go(k_lbvh_neighbors<8>); break;
    }
    count_launch();
}

// ------------------------------------------------------------ transpose
// The walk lists every unordered pair once, from its lower cell (forward
// lists: adjacent cells first).  The full lists add each pair to the higher
// cell too: a warp per cell g counts, for every forward entry h, its place in
// h's backward list (an atomic per entry, also the number of points in the
// neighbouring cells when MarkCore needs it); the totals are scanned into the
// final offsets; a second pass writes every cell's list as [forward adjacent,
// backward adjacent, forward farther, backward farther].
__global__ void __launch_bounds__(256)
k_hd_back_count(const long long *__restrict__ fo, const int *__restrict__ fn, const int *__restrict__ ff,
                const int *__restrict__ fwd, int *__restrict__ rank, int *__restrict__ bn, int *__restrict__ bf,
                const int *__restrict__ cell_start, int *__restrict__ nbr_pts, DevCounters *ctr) {
    if (run_failed(ctr)) return;
    const int lane = threadIdx.x & 31;
    const int m = ctr->m;
    for (int g = warp_id_global(); g < m; g += warps_global()) {
        const long long f0 = fo[g];
        const int a = fn[g], cnt = a + ff[g];
        const int gsz = nbr_pts ? cell_start[g + 1] - cell_start[g] : 0;
        int pts = 0;
        for (int e = lane; e < cnt; e += 32) {
            const int h = fwd[f0 + e];
            rank[f0 + e] = atomicAdd(e < a ? bn + h : bf + h, 1);
            if (nbr_pts) {
                pts += cell_start[h + 1] - cell_start[h];
                atomicAdd(nbr_pts + h, gsz);
            }
        }
        if (nbr_pts) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) pts += __shfl_xor_sync(0xffffffffu, pts, o);
            if (lane == 0 && pts) atomicAdd(nbr_pts + g, pts);
        }
    }
}

__global__ void __launch_bounds__(256)
k_hd_totals(const int *__restrict__ fn, const int *__restrict__ ff, const int *__restrict__ bn,
            const int *__restrict__ bf, long long *__restrict__ tot, int *__restrict__ nbr_cnt,
            int *__restrict__ nbr_near, DevCounters *ctr) {
    if (run_failed(ctr)) return;
    const int m = ctr->m;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < m; g += gridDim.x * blockDim.x) {
        const int t = fn[g] + ff[g] + bn[g] + bf[g];
        tot[g] = t;
        nbr_cnt[g] = t;
        nbr_near[g] = fn[g] + bn[g];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) ctr->E *= 2;  // every pair now in both lists
}

__global__ void __launch_bounds__(256)
k_hd_fill(const long long *__restrict__ fo, const int *__restrict__ fn, const int *__restrict__ ff,
          const int *__restrict__ bn, const int *__restrict__ fwd, const int *__restrict__ rank,
          const long long *__restrict__ off, int *__restrict__ nbr, DevCounters *ctr) {
    if (run_failed(ctr)) return;
    const int lane = threadIdx.x & 31;
    const int m = ctr->m;
    for (int g = warp_id_global(); g < m; g += warps_global()) {
        const long long f0 = fo[g], o = off[g];
        const int a = fn[g], cnt = a + ff[g], bng = bn[g];
        for (int e = lane; e < cnt; e += 32) {
            const int h = fwd[f0 + e];
            const int r = rank[f0 + e];
            const long long oh = off[h] + fn[h];
            if (e < a) {
                nbr[o + e] = h;
                nbr[oh + r] = g;
            } else {
                nbr[o + bng + e] = h;
                nbr[oh + bn[h] + ff[h] + r] = g;
            }
        }
    }
}

void hd_transpose(const RunParams &P, const HdBufs &H, const Bufs &B, const int *fwd, int *rank, int *nbr,
                  DevCounters *ctr, cudaStream_t s) {
    const bool pts = P.mc_small_nbr > 0 && P.mc_small_nbr < (1 << 30);
    int g = grid_for((const void *)k_hd_back_count, 256);
    k_hd_back_count<<<g, 256, 0, s>>>(H.fwd_off, H.fn, H.ff, fwd, rank, H.bn, H.bf, B.cell_start,
                                      pts ? const_cast<int *>(B.nbr_pts) : nullptr, ctr);
    count_launch();
    g = grid_for((const void *)k_hd_totals, 256);
    k_hd_totals<<<g, 256, 0, s>>>(H.fn, H.ff, H.bn, H.bf, H.nbr_off, const_cast<int *>(B.nbr_cnt),
                                  const_cast<int *>(B.nbr_near), ctr);
    count_launch();
    scan_i64_to_i64(H.nbr_off, H.nbr_off, 0, &ctr->m, B.n_max, B.part, s);
    g = grid_for((const void *)k_hd_fill, 256);
    k_hd_fill<<<g, 256, 0, s>>>(H.fwd_off, H.fn, H.ff, H.bn, fwd, rank, H.nbr_off, nbr, ctr);
    count_launch();
}

}  // namespace gbdb
