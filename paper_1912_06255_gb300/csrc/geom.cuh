// Device helpers shared by the distance kernels: point loads, the exact FP64
// predicate, the FP32 band test, Morton packing of cell coordinates, the cell
// hash and the union-find.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.cuh"

namespace gbdb {

// ------------------------------------------------------------ point loads
template <int D> __device__ __forceinline__ void load_f(const float *__restrict__ pf, int64_t i, float (&x)[D]) {
    constexpr int SD = Store<D>::SD;
    const float *p = pf + i * SD;
    if constexpr (SD == 2) {
        float2 a = *reinterpret_cast<const float2 *>(p);
        x[0] = a.x;
        if constexpr (D > 1) x[1] = a.y;
    } else if constexpr (SD == 4) {
        float4 a = *reinterpret_cast<const float4 *>(p);
        x[0] = a.x;
        if constexpr (D > 1) x[1] = a.y;
        if constexpr (D > 2) x[2] = a.z;
        if constexpr (D > 3) x[3] = a.w;
    } else {
        float4 a = *reinterpret_cast<const float4 *>(p);
        float4 b = *reinterpret_cast<const float4 *>(p + 4);
        float t[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
        for (int j = 0; j < D; ++j) x[j] = t[j];
    }
}

template <int D> __device__ __forceinline__ void load_d(const double *__restrict__ pd, int64_t i, double (&x)[D]) {
    constexpr int SD = Store<D>::SD;
    const double *p = pd + i * SD;
#pragma unroll
    for (int j = 0; j < D; j += 2) {
        double2 a = *reinterpret_cast<const double2 *>(p + j);
        x[j] = a.x;
        if (j + 1 < D) x[j + 1] = a.y;
    }
}

// Sec. 2 predicate, d(p,q) <= eps, as  sum_i (p_i - q_i)^2 <= fl(eps^2)  in
// FP64: left to right, each subtraction, product and sum rounded to nearest,
// no fused multiply-add.  Zero-padded coordinates add exact zeros.
template <int D>
__device__ __forceinline__ bool pred64(const double (&a)[D], const double (&b)[D], double eps2) {
    double t = __dsub_rn(a[0], b[0]);
    double s = __dmul_rn(t, t);
#pragma unroll
    for (int j = 1; j < D; ++j) {
        double u = __dsub_rn(a[j], b[j]);
        s = __dadd_rn(s, __dmul_rn(u, u));
    }
    return s <= eps2;
}

// Squared distance in FP32 (its error bound is what the band is derived from).
template <int D> __device__ __forceinline__ float d2f(const float (&a)[D], const float (&b)[D]) {
    float t = a[0] - b[0];
    float s = t * t;
#pragma unroll
    for (int j = 1; j < D; ++j) {
        float u = a[j] - b[j];
        s = __fmaf_rn(u, u, s);
    }
    return s;
}

// A point held in registers or shared memory: FP32 coordinates, or FP64 in
// the FP64-storage FP64-predicate mode.
template <int D, int M, bool DBL = (M == kF64FromF64)> struct Pt;
template <int D, int M> struct alignas(D >= 3 ? 16 : 8) Pt<D, M, false> { float f[D]; };
template <int D, int M> struct alignas(16) Pt<D, M, true> { double x[D]; };

template <int D, int M>
__device__ __forceinline__ void load_pt(Pt<D, M> &p, const float *__restrict__ pf,
                                        const double *__restrict__ pd, int64_t i) {
    if constexpr (M == kF64FromF64) load_d<D>(pd, i, p.x);
    else load_f<D>(pf, i, p.f);
}

// within(p, q).  ip/iq index p and q in pdp/pdq, the FP64 copies consulted by
// the recheck of the FP32-band mode on FP64 storage.  *rechecks counts FP32
// decisions sent to FP64.
template <int D, int M>
__device__ __forceinline__ bool within(const Pt<D, M> &p, const Pt<D, M> &q, const Thr &P,
                                       const double *__restrict__ pdp, int64_t ip,
                                       const double *__restrict__ pdq, int64_t iq,
                                       unsigned &rechecks) {
    if constexpr (M == kF64FromF64) {
        return pred64<D>(p.x, q.x, P.eps2);
    } else if constexpr (M == kF64FromF32) {
        double a[D], b[D];
#pragma unroll
        for (int j = 0; j < D; ++j) { a[j] = (double)p.f[j]; b[j] = (double)q.f[j]; }
        return pred64<D>(a, b, P.eps2);
    } else {
        float s = d2f<D>(p.f, q.f);
        if (s <= P.lo) return true;
        if (s > P.hi) return false;
        ++rechecks;
        double a[D], b[D];
        if constexpr (M == kF32FromF32) {
#pragma unroll
            for (int j = 0; j < D; ++j) { a[j] = (double)p.f[j]; b[j] = (double)q.f[j]; }
        } else {
            load_d<D>(pdp, ip, a);
            load_d<D>(pdq, iq, b);
        }
        return pred64<D>(a, b, P.eps2);
    }
}

// ------------------------------------------------------------ box bounds
// Cell-level pruning (a one-level form of the range counting of Sec. 5.2): for
// an axis-aligned box [lo, hi] that contains every point of a cell, bounds of
// the squared distance from a point (or another box) to all of those points.
// Each coordinate term is one FP32 subtraction of exact FP32 values (the max
// and the clamp at 0 are exact), squared and summed like d2f, so the value
// carries the same forward-error bound as d2f and the FP32 band applies:
// max_d2 <= lo means every pair passes the FP64 predicate, min_d2 > hi that
// none does.
// Boxes are stored per cell as box_w<D>() float4 values (one for d <= 4, two
// above), zero-padded past the instance's own dimension.
template <int D> __host__ __device__ constexpr int box_w() { return D <= 4 ? 1 : 2; }
template <int D> struct Bx { float4 v[box_w<D>()]; };

__device__ __forceinline__ float cget(const float4 &v, int j) {
    return j == 0 ? v.x : (j == 1 ? v.y : (j == 2 ? v.z : v.w));
}
template <int D> __device__ __forceinline__ float bget(const Bx<D> &b, int j) { return cget(b.v[j >> 2], j & 3); }

template <int D> __device__ __forceinline__ Bx<D> load_box(const float4 *__restrict__ base, int64_t c) {
    Bx<D> r;
#pragma unroll
    for (int k = 0; k < box_w<D>(); ++k) r.v[k] = base[c * box_w<D>() + k];
    return r;
}
template <int D> __device__ __forceinline__ Bx<D> zero_box() {
    Bx<D> r;
#pragma unroll
    for (int k = 0; k < box_w<D>(); ++k) r.v[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    return r;
}

template <int D>
__device__ __forceinline__ float box_max_d2(const float (&p)[D], const Bx<D> &lo, const Bx<D> &hi) {
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const float a = fmaxf(p[j] - bget<D>(lo, j), bget<D>(hi, j) - p[j]);
        s = j == 0 ? a * a : __fmaf_rn(a, a, s);
    }
    return s;
}

template <int D>
__device__ __forceinline__ float box_min_d2(const float (&p)[D], const Bx<D> &lo, const Bx<D> &hi) {
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const float a = fmaxf(fmaxf(bget<D>(lo, j) - p[j], p[j] - bget<D>(hi, j)), 0.f);
        s = j == 0 ? a * a : __fmaf_rn(a, a, s);
    }
    return s;
}

template <int D>
__device__ __forceinline__ float boxes_min_d2(const Bx<D> &alo, const Bx<D> &ahi, const Bx<D> &blo,
                                              const Bx<D> &bhi) {
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const float a =
            fmaxf(fmaxf(bget<D>(blo, j) - bget<D>(ahi, j), bget<D>(alo, j) - bget<D>(bhi, j)), 0.f);
        s = j == 0 ? a * a : __fmaf_rn(a, a, s);
    }
    return s;
}

template <int D>
__device__ __forceinline__ float boxes_max_d2(const Bx<D> &alo, const Bx<D> &ahi, const Bx<D> &blo,
                                              const Bx<D> &bhi) {
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const float a = fmaxf(bget<D>(bhi, j) - bget<D>(alo, j), bget<D>(ahi, j) - bget<D>(blo, j));
        s = j == 0 ? a * a : __fmaf_rn(a, a, s);
    }
    return s;
}

// ------------------------------------------------------------ cell coordinates
// Cell coordinate of coordinate j of a point: floor(fl64(fl64(x - o) * inv_s)),
// clamped to [0, kmax].  For FP32 input the FP32 estimate
// t32 = fl32(fl32(x - o) * fl32(inv_s)) is within eps_t = t * 3.01 * 2^-24 (+ the
// FP64 value's own 3 * 2^-53 * t) of the FP64 value t64 (x and o = the minimum
// of FP32 values are exact FP32 numbers), so when t32 is farther than eps_t
// from an integer both floors agree; only the rest is recomputed in FP64.
template <typename T>
__device__ __forceinline__ int cell_coord(T x, const Inst &I, int j) {
    if constexpr (sizeof(T) == 4) {
        const float t32 = __fmul_rn(__fsub_rn(x, I.origin32[j]), I.inv_s32);
        const float fl = floorf(t32);
        const float e = t32 * 1.8e-7f + 1e-30f;
        if (t32 - fl > e && (fl + 1.0f) - t32 > e) {
            const int k = (int)fl;
            return k < 0 ? 0 : (k > I.kmax[j] ? I.kmax[j] : k);
        }
    }
    const double t = __dmul_rn(__dsub_rn((double)x, I.origin[j]), I.inv_s);
    const int k = (int)floor(t);
    return k < 0 ? 0 : (k > I.kmax[j] ? I.kmax[j] : k);
}

// ------------------------------------------------------------ Morton keys
__host__ __device__ __forceinline__ uint64_t spread2(uint64_t x) {
    x &= 0xffffffffull;
    x = (x | (x << 16)) & 0x0000ffff0000ffffull;
    x = (x | (x << 8)) & 0x00ff00ff00ff00ffull;
    x = (x | (x << 4)) & 0x0f0f0f0f0f0f0f0full;
    x = (x | (x << 2)) & 0x3333333333333333ull;
    x = (x | (x << 1)) & 0x5555555555555555ull;
    return x;
}
__host__ __device__ __forceinline__ uint64_t compact2(uint64_t x) {
    x &= 0x5555555555555555ull;
    x = (x | (x >> 1)) & 0x3333333333333333ull;
    x = (x | (x >> 2)) & 0x0f0f0f0f0f0f0f0full;
    x = (x | (x >> 4)) & 0x00ff00ff00ff00ffull;
    x = (x | (x >> 8)) & 0x0000ffff0000ffffull;
    x = (x | (x >> 16)) & 0x00000000ffffffffull;
    return x;
}
__host__ __device__ __forceinline__ uint64_t spread3(uint64_t x) {
    x &= 0x1fffffull;
    x = (x | (x << 32)) & 0x001f00000000ffffull;
    x = (x | (x << 16)) & 0x001f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}
__host__ __device__ __forceinline__ uint64_t compact3(uint64_t x) {
    x &= 0x1249249249249249ull;
    x = (x | (x >> 2)) & 0x10c30c30c30c30c3ull;
    x = (x | (x >> 4)) & 0x100f00f00f00f00full;
    x = (x | (x >> 8)) & 0x001f0000ff0000ffull;
    x = (x | (x >> 16)) & 0x001f00000000ffffull;
    x = (x | (x >> 32)) & 0x1fffffull;
    return x;
}

// Interleave d cell coordinates of `bits` bits each (bit b of dimension j goes
// to key bit b*d + j).  d*bits <= 63.
__host__ __device__ __forceinline__ uint64_t morton_encode(const int *c, int d, int bits) {
    if (d == 1) return (uint64_t)c[0];
    if (d == 2) return spread2((uint64_t)c[0]) | (spread2((uint64_t)c[1]) << 1);
    if (d == 3)
        return spread3((uint64_t)c[0]) | (spread3((uint64_t)c[1]) << 1) |
               (spread3((uint64_t)c[2]) << 2);
    uint64_t k = 0;
    for (int b = 0; b < bits; ++b)
        for (int j = 0; j < d; ++j) k |= (uint64_t)((c[j] >> b) & 1) << (b * d + j);
    return k;
}

__host__ __device__ __forceinline__ void morton_decode(uint64_t k, int d, int bits, int *c) {
    if (d == 1) { c[0] = (int)k; return; }
    if (d == 2) { c[0] = (int)compact2(k); c[1] = (int)compact2(k >> 1); return; }
    if (d == 3) {
        c[0] = (int)compact3(k);
        c[1] = (int)compact3(k >> 1);
        c[2] = (int)compact3(k >> 2);
        return;
    }
    for (int j = 0; j < d; ++j) c[j] = 0;
    for (int b = 0; b < bits; ++b)
        for (int j = 0; j < d; ++j) c[j] |= (int)((k >> (b * d + j)) & 1) << b;
}

// ------------------------------------------------------------ cell hash
// Open addressing with linear probing, keyed by the packed cell key (Sec. 4.1
// stores the non-empty cells in a hash table).  Capacity: power of two >= 2m.
__host__ __device__ __forceinline__ uint64_t hash_capacity(int m) {
    uint64_t c = 16;
    while (c < 2ull * (uint64_t)m) c <<= 1;
    return c;
}
__host__ __device__ __forceinline__ int hash_log2(uint64_t cap) {
    int l = 0;
    while ((1ull << l) < cap) ++l;
    return l;
}
// Multiplicative (Fibonacci) hashing: the top lg bits of key * 2^64/phi.
__device__ __forceinline__ uint64_t hash_slot(uint64_t k, int lg) {
    return (k * 0x9e3779b97f4a7c15ull) >> (64 - lg);
}

// Bloom filter of the non-empty cells (two bits per key in a table of 2^lg
// bits), kept in L2: probes for empty neighbouring cells stop here instead of
// reaching the hash table.
__device__ __forceinline__ void bloom_bits(uint64_t k, int lg, uint64_t &b0, uint64_t &b1) {
    const uint64_t h = k * 0xd6e8feb86659fd93ull;
    b0 = h >> (64 - lg);
    b1 = (h * 0x9e3779b97f4a7c15ull + 0x632be59bd9b4e019ull) >> (64 - lg);
}
__device__ __forceinline__ void bloom_add(unsigned *bloom, uint64_t k, int lg) {
    uint64_t b0, b1;
    bloom_bits(k, lg, b0, b1);
    atomicOr(bloom + (b0 >> 5), 1u << (b0 & 31));
    atomicOr(bloom + (b1 >> 5), 1u << (b1 & 31));
}
__device__ __forceinline__ bool bloom_may_have(const unsigned *__restrict__ bloom, uint64_t k, int lg) {
    uint64_t b0, b1;
    bloom_bits(k, lg, b0, b1);
    return ((bloom[b0 >> 5] >> (b0 & 31)) & 1u) && ((bloom[b1 >> 5] >> (b1 & 31)) & 1u);
}

// A slot is 16 bytes: .x the key (kEmptyKey when free), .y the cell id, so a
// probe is one load (k_insert, k_neighbors).

// Morton key of the cell at c + delta from the key of c (D = 2 or 3), by
// dilated-integer addition: per dimension, the key's bits of that dimension
// with the other bits set to one (for +) or zero (for -) absorb the carries
// or borrows.  |delta_j| <= 3 and c + delta stays inside the grid.
template <int D>
__device__ __forceinline__ uint64_t morton_offset(uint64_t key, const int (&delta)[D]) {
    uint64_t out = 0;
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const uint64_t M = (D == 3 ? 0x1249249249249249ull : 0x5555555555555555ull) << j;
        uint64_t part = key & M;
        const int dj = delta[j];
        const int a = dj < 0 ? -dj : dj;
        const uint64_t v = (uint64_t)((a & 1) | ((a & 2) << (D - 1))) << j;
        if (dj > 0) part = ((part | ~M) + v) & M;
        else if (dj < 0) part = (part - v) & M;
        out |= part;
    }
    return out;
}

// ------------------------------------------------------------ union-find
// Lock-free union-find over cells (Algorithm 3).  Link hooks the larger root
// under the smaller one, so parent[x] <= x always and every root is the
// smallest cell of its set.  Find halves paths with plain stores: each store
// replaces a parent by one of its ancestors, which keeps the forest valid
// under races.
__device__ __forceinline__ int uf_load(const int *p) { return *(const volatile int *)p; }

__device__ __forceinline__ int uf_find(int *parent, int x, int max_iters, DevCounters *ctr) {
    for (int it = 0; it < max_iters; ++it) {
        int p = uf_load(parent + x);
        if (p == x) return x;
        int g = uf_load(parent + p);
        if (g != p) *(volatile int *)(parent + x) = g;
        x = g;
    }
    set_error(ctr, DBSCAN_ERR_DEVICE_TIMEOUT, 1);
    return x;
}

// Find on a possibly stale view of the forest, through L1 (ld.global.ca),
// without stores.  Every parent value ever written joins two cells of one set
// and sets only merge, so two cells whose stale walks end at the same cell are
// in one set now: a "same" answer is final, a "different" one needs uf_find.
// Parents only decrease along a walk (parent[x] <= x), so the walk ends.
__device__ __forceinline__ int uf_find_stale(const int *parent, int x, int max_iters) {
    for (int it = 0; it < max_iters; ++it) {
        const int p = __ldca(parent + x);
        if (p == x) return x;
        x = p;
    }
    return x;
}

// Returns true iff this call hooked one root under another (the two sets
// were separate and are now one).
__device__ __forceinline__ bool uf_link(int *parent, int a, int b, int max_iters, DevCounters *ctr) {
    for (int it = 0; it < max_iters; ++it) {
        int ra = uf_find(parent, a, max_iters, ctr);
        int rb = uf_find(parent, b, max_iters, ctr);
        if (ra == rb) return false;
        if (ra < rb) { int t = ra; ra = rb; rb = t; }  // ra is the larger root
        if (atomicCAS(parent + ra, ra, rb) == ra) return true;
    }
    set_error(ctr, DBSCAN_ERR_DEVICE_TIMEOUT, 2);
    return false;
}

// Link witnesses (optional, P.wit non-null): every hook of the union-find is
// recorded with one pair of core points (compacted indices) that the run
// found within eps, so that a checker can verify each cluster as a connected
// graph of eps-edges.  The hooks number m_core minus the components, so
// wit_cap = m is never exceeded.
__device__ __forceinline__ void record_link(const RunParams &P, DevCounters *ctr, int ka, int kb) {
    if (!P.wit) return;
    const unsigned long long k = atomicAdd(&ctr->n_wit, 1ull);
    if (k < (unsigned long long)P.wit_cap) P.wit[k] = make_int2(ka, kb);
    else set_error(ctr, DBSCAN_ERR_CAPACITY, 60);
}

// Neighbour list of cell c: CSR offsets for d >= 5 (compiled width 8), a
// fixed stride per cell below.
template <int D>
__device__ __forceinline__ const int *nbr_list(const int *nbr, const long long *off, int stride, int c) {
    if constexpr (D == 8) return nbr + off[c];
    else return nbr + (long long)c * stride;
}

__device__ __forceinline__ int warp_id_global() {
    return (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
}
__device__ __forceinline__ int warps_global() { return (int)((gridDim.x * (int64_t)blockDim.x) >> 5); }

}  // namespace gbdb
