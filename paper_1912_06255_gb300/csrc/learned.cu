// Learned core-cell pair scheduler.
//
// Algorithm 3 tests neighbouring core cells in a priority order (SortBySize)
// so that union-find skips the tests of pairs already joined through other
// cells ("Reducing Cell Connectivity Queries").  This file replaces that
// heuristic order with a learned one: a small MLP scores every undecided pair
// by how likely its two cells are to be connected, and the pairs are tested
// likeliest first.  Every connectivity decision is still the exact BCP test,
// so the clustering does not depend on the network; only the number of tests
// does.  The network is trained on (features, outcome) records logged by the
// method itself (a logging run tests every undecided pair exactly), with
// hand-written forward/backward and Adam kernels.
#include <cuda_runtime.h>

#include <climits>

#include "bcp.cuh"
#include "geom.cuh"
#include "grid.cuh"
#include "learned.cuh"

namespace gbdb {

__device__ __forceinline__ void flush_warp_counter(unsigned long long *dst, unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(dst, v);
}

__global__ void __launch_bounds__(256) k_uf_reset(int *parent, uint64_t *best, const DevCounters *ctr) {
    if (run_failed(ctr)) return;
    const int m = ctr->m;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < m; c += gridDim.x * blockDim.x) {
        parent[c] = c;
        best[c] = ~0ull;
    }
}

// Clamp the pair count to the list capacity (the overflow is already an error).
__global__ void k_clamp_pairs(DevCounters *ctr, long long cap) {
    const unsigned long long d = ctr->P_demand;
    ctr->P_list = (int)(d < (unsigned long long)cap ? d : (unsigned long long)cap);
}

// ----------------------------------------------------------------- features
// Symmetric in the two cells: log2(1 + larger core count), log2(1 + smaller
// core count), core-centroid distance / eps, core-box minimum and maximum
// distance / eps, smaller / larger core count.
template <int D>
__device__ __forceinline__ void pair_features(int a, int b, const int *__restrict__ ccs,
                                              const float4 *__restrict__ cent, const float4 *__restrict__ cblo,
                                              const float4 *__restrict__ cbhi, float eps, float (&f)[kMlpIn]) {
    const int na = ccs[a + 1] - ccs[a], nb = ccs[b + 1] - ccs[b];
    const int big = na > nb ? na : nb, small = na > nb ? nb : na;
    const Bx<D> ca = load_box<D>(cent, a), cb = load_box<D>(cent, b);
    float c2 = 0.f;
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const float t = bget<D>(ca, j) - bget<D>(cb, j);
        c2 = __fmaf_rn(t, t, c2);
    }
    const Bx<D> alo = load_box<D>(cblo, a), ahi = load_box<D>(cbhi, a);
    const Bx<D> blo = load_box<D>(cblo, b), bhi = load_box<D>(cbhi, b);
    const float inv = 1.f / eps;
    f[0] = log2f(1.f + (float)big);
    f[1] = log2f(1.f + (float)small);
    f[2] = sqrtf(c2) * inv;
    f[3] = sqrtf(boxes_min_d2<D>(alo, ahi, blo, bhi)) * inv;
    f[4] = sqrtf(boxes_max_d2<D>(alo, ahi, blo, bhi)) * inv;
    f[5] = big > 0 ? (float)small / (float)big : 0.f;
}

// ----------------------------------------------------------------- the MLP
// kMlpIn -> kMlpHid -> kMlpHid -> 1, ReLU hidden layers, logit output.
// Parameter layout: W1[H][F], b1[H], W2[H][H], b2[H], w3[H], b3.
__device__ __forceinline__ float mlp_forward(const float *__restrict__ w, const float (&x)[kMlpIn],
                                             float (&h1)[kMlpHid], float (&h2)[kMlpHid]) {
#pragma unroll
    for (int j = 0; j < kMlpHid; ++j) {
        float s = w[kOB1 + j];
#pragma unroll
        for (int i = 0; i < kMlpIn; ++i) s = __fmaf_rn(w[kOW1 + j * kMlpIn + i], x[i], s);
        h1[j] = fmaxf(s, 0.f);
    }
#pragma unroll
    for (int j = 0; j < kMlpHid; ++j) {
        float s = w[kOB2 + j];
#pragma unroll
        for (int i = 0; i < kMlpHid; ++i) s = __fmaf_rn(w[kOW2 + j * kMlpHid + i], h1[i], s);
        h2[j] = fmaxf(s, 0.f);
    }
    float z = w[kOB3];
#pragma unroll
    for (int i = 0; i < kMlpHid; ++i) z = __fmaf_rn(w[kOW3 + i], h2[i], z);
    return z;
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Loss and gradient of the mean binary cross-entropy with logits over samples
// [0, n): one sample per lane; each parameter's gradient is summed over the
// warp and added to grad[] once per warp; loss[0] gets the summed loss.
__global__ void __launch_bounds__(256)
k_mlp_grad(const float *__restrict__ w, const float *__restrict__ feat, const unsigned char *__restrict__ lab,
           long long first, long long n, long long total, float scale, float *__restrict__ grad,
           float *__restrict__ loss) {
    __shared__ float sw[kMlpParams];
    for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) sw[i] = w[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    for (long long base = (long long)warp_id_global() * 32; base < n; base += (long long)warps_global() * 32) {
        const long long k = base + lane;
        const bool ok = k < n;
        const long long row = ok ? (first + k) % total : 0;
        float x[kMlpIn], h1[kMlpHid], h2[kMlpHid];
#pragma unroll
        for (int i = 0; i < kMlpIn; ++i) x[i] = ok ? feat[row * kMlpIn + i] : 0.f;
        const float y = ok ? (float)lab[row] : 0.f;
        const float z = mlp_forward(sw, x, h1, h2);
        // BCE with logits: max(z,0) - z*y + log(1 + exp(-|z|)); d/dz = sigmoid(z) - y
        const float l = ok ? fmaxf(z, 0.f) - z * y + log1pf(__expf(-fabsf(z))) : 0.f;
        const float dz = ok ? (1.f / (1.f + __expf(-z)) - y) * scale : 0.f;
        const float ls = warp_sum(l);
        if (lane == 0) atomicAdd(loss, ls * scale);
        float d2[kMlpHid];
#pragma unroll
        for (int i = 0; i < kMlpHid; ++i) d2[i] = h2[i] > 0.f ? dz * sw[kOW3 + i] : 0.f;
        // output layer
        {
            const float g = warp_sum(dz);
            if (lane == 0) atomicAdd(grad + kOB3, g);
        }
        for (int i = 0; i < kMlpHid; ++i) {
            const float g = warp_sum(dz * h2[i]);
            if (lane == 0) atomicAdd(grad + kOW3 + i, g);
        }
        // second layer
        float d1[kMlpHid];
#pragma unroll
        for (int i = 0; i < kMlpHid; ++i) d1[i] = 0.f;
        for (int j = 0; j < kMlpHid; ++j) {
            const float gb = warp_sum(d2[j]);
            if (lane == 0) atomicAdd(grad + kOB2 + j, gb);
#pragma unroll
            for (int i = 0; i < kMlpHid; ++i) {
                const float g = warp_sum(d2[j] * h1[i]);
                if (lane == 0) atomicAdd(grad + kOW2 + j * kMlpHid + i, g);
                d1[i] = __fmaf_rn(d2[j], sw[kOW2 + j * kMlpHid + i], d1[i]);
            }
        }
        // first layer
        for (int j = 0; j < kMlpHid; ++j) {
            const float dj = h1[j] > 0.f ? d1[j] : 0.f;
            const float gb = warp_sum(dj);
            if (lane == 0) atomicAdd(grad + kOB1 + j, gb);
#pragma unroll
            for (int i = 0; i < kMlpIn; ++i) {
                const float g = warp_sum(dj * x[i]);
                if (lane == 0) atomicAdd(grad + kOW1 + j * kMlpIn + i, g);
            }
        }
    }
}

// Adam step on all parameters (t = step number, from 1).
__global__ void k_adam(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m1,
                       float *__restrict__ m2, float lr, int t) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kMlpParams) return;
    const float b1 = 0.9f, b2 = 0.999f;
    m1[i] = b1 * m1[i] + (1.f - b1) * g[i];
    m2[i] = b2 * m2[i] + (1.f - b2) * g[i] * g[i];
    const float mh = m1[i] / (1.f - powf(b1, (float)t));
    const float vh = m2[i] / (1.f - powf(b2, (float)t));
    w[i] -= lr * mh / (sqrtf(vh) + 1e-8f);
}

void mlp_loss_grad(const float *w, const float *feat, const unsigned char *lab, long long first, long long n,
                   long long total, float *grad, float *loss, cudaStream_t s) {
    const int g = grid_for((const void *)k_mlp_grad, 256);
    k_mlp_grad<<<g, 256, 0, s>>>(w, feat, lab, first, n, total, 1.f / (float)(n > 0 ? n : 1), grad, loss);
    count_launch();
}

void mlp_adam(float *w, const float *g, float *m1, float *m2, float lr, int t, cudaStream_t s) {
    k_adam<<<(kMlpParams + 255) / 256, 256, 0, s>>>(w, g, m1, m2, lr, t);
    count_launch();
}

// ----------------------------------------------------------------- pairs
// Every pair of neighbouring core cells (a, b), a < b, once.  The core-point
// boxes settle some outright (all pairs within eps: link; none: drop).
//   PASS 0: the box decisions only (links), before any listing;
//   PASS 1: after compression, the undecided pairs whose cells union-find has
//           not joined yet are appended to the pair list (the others count as
//           skipped);
//   PASS 2: the logging run: box decisions and every undecided pair listed,
//           in one pass (nothing may be skipped there).
template <int D, int PASS>
__global__ void __launch_bounds__(256)
k_collect_pairs(RunParams P, const int *__restrict__ ccs, const int *__restrict__ nbr_cnt,
                const int *__restrict__ nbr, int stride, const long long *__restrict__ nbr_off,
                const float4 *__restrict__ cblo,
                const float4 *__restrict__ cbhi, int *parent, int2 *__restrict__ pairs, long long cap,
                int count_cands, DevCounters *ctr) {
    if (run_failed(ctr)) return;
    const int m = ctr->m;
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    unsigned long long cand_pairs = 0, boxed = 0, linked = 0, skipped = 0;
    for (int a = warp_id_global(); a < m; a += warps_global()) {
        if (ccs[a + 1] == ccs[a]) continue;
        const Thr T = P.inst[inst_of_cell(P, a)].cthr;
        const Bx<D> alo = load_box<D>(cblo, a), ahi = load_box<D>(cbhi, a);
        const int ne = nbr_cnt[a];
        const int *nl = nbr_list<D>(nbr, nbr_off, stride, a);
        int ra = PASS == 1 ? uf_find(parent, a, P.max_iters, ctr) : a;
        for (int e0 = 0; e0 < ne; e0 += 32) {
            const int e = e0 + lane;
            int b = 0;
            bool cand = false;
            int verdict = 0;
            if (e < ne) {
                b = nl[e];
                cand = b > a && ccs[b + 1] > ccs[b];
                if (cand && P.box) {
                    const Bx<D> blo = load_box<D>(cblo, b), bhi = load_box<D>(cbhi, b);
                    if (boxes_min_d2<D>(alo, ahi, blo, bhi) > T.hi) verdict = -1;
                    else if (boxes_max_d2<D>(alo, ahi, blo, bhi) <= T.lo) verdict = 1;
                }
            }
            if (PASS != 1 && cand && verdict > 0 && uf_link(parent, a, b, P.max_iters, ctr))
                record_link(P, ctr, ccs[a], ccs[b]);  // every core pair is within eps
            bool keep = PASS != 0 && cand && verdict == 0;
            if (PASS == 1 && keep && uf_find(parent, b, P.max_iters, ctr) == ra) {
                keep = false;
                ++skipped;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, keep);
            long long at = 0;
            if (lane == 0 && bal) at = (long long)atomicAdd(&ctr->P_demand, (unsigned long long)__popc(bal));
            at = __shfl_sync(0xffffffffu, at, 0);
            if (keep) {
                const long long k = at + __popc(bal & lt);
                if (k < cap) pairs[k] = make_int2(a, b);
                else set_error(ctr, DBSCAN_ERR_CAPACITY, 50);
            }
            if (count_cands) {  // the run's first pass over the pairs
                cand_pairs += __popc(__ballot_sync(0xffffffffu, cand));
                boxed += __popc(__ballot_sync(0xffffffffu, cand && verdict != 0));
                linked += __popc(__ballot_sync(0xffffffffu, cand && verdict > 0));
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) skipped += __shfl_xor_sync(0xffffffffu, skipped, o);
    if (lane == 0) {
        if (cand_pairs) atomicAdd((unsigned long long *)&ctr->P, cand_pairs);
        if (boxed) atomicAdd(&ctr->pairs_box, boxed);
        if (linked) atomicAdd(&ctr->pairs_linked, linked);
        if (skipped) atomicAdd(&ctr->pairs_skipped, skipped);
    }
}

// Score every listed pair with the MLP; the sort key puts the likeliest first:
// key = (clamp((16 - logit) * 2048) << 32) | pair index, so the pairs the
// network predicts connected (logit > 0) are exactly those with a score below
// 2^15; they are counted in P_pos.  Each cell also keeps the smallest key of
// its pairs among those (best[], 64-bit atomicMin): its likeliest link.
template <int D>
__global__ void __launch_bounds__(256)
k_score_pairs(RunParams P, const int2 *__restrict__ pairs, const float *__restrict__ w, const int *__restrict__ ccs,
              const float4 *__restrict__ cent, const float4 *__restrict__ cblo, const float4 *__restrict__ cbhi,
              uint64_t *__restrict__ keys, unsigned long long *__restrict__ best, DevCounters *ctr) {
    if (run_failed_block(ctr)) return;
    __shared__ float sw[kMlpParams];
    for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) sw[i] = w[i];
    __syncthreads();
    const long long np = ctr->P_list;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long np_pad = (np + 31) / 32 * 32;  // whole warps for the ballot
    int pos = 0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < np_pad; k += stride) {
        bool positive = false;
        if (k < np) {
            const int2 pr = pairs[k];
            const float eps = sqrtf((float)P.inst[inst_of_cell(P, pr.x)].cthr.eps2);
            float x[kMlpIn], h1[kMlpHid], h2[kMlpHid];
            pair_features<D>(pr.x, pr.y, ccs, cent, cblo, cbhi, eps, x);
            const float z = mlp_forward(sw, x, h1, h2);
            const unsigned q = (unsigned)fminf(fmaxf((16.f - z) * 2048.f, 0.f), 65535.f);
            const uint64_t key = ((uint64_t)q << 32) | (uint64_t)k;
            keys[k] = key;
            positive = q < 32768u;
            if (positive) {
                atomicMin(best + pr.x, (unsigned long long)key);
                atomicMin(best + pr.y, (unsigned long long)key);
            }
        }
        pos += __popc(__ballot_sync(0xffffffffu, positive));
    }
    if ((threadIdx.x & 31) == 0 && pos) atomicAdd(&ctr->P_pos, pos);
}

// BCP tests of the learned schedule, in waves separated by full path
// compression of the union-find:
//   WAVE 0: every core cell tests its likeliest link (best[]), each pair once
//           (a Boruvka-style hooking step: one test per cell builds the
//           large components before anything else runs);
//   WAVE 1: the other pairs predicted connected, likeliest first;
//   WAVE 2: the remaining pairs.
// In waves 1 and 2 a warp takes the next 32 positions of the sorted list with
// one atomic, checks them against the union-find one per lane, and runs BCP
// on the survivors one at a time (each re-checked just before its test).
// WAVE 3 is the logging run: every listed pair, in list order, tested with no
// skipping, its features and outcome recorded at its list index.
template <int D, int M, int WAVE>
__global__ void __launch_bounds__(256, 2)
k_test_pairs(RunParams P, const int2 *__restrict__ pairs, const uint64_t *__restrict__ sorted,
             const unsigned long long *__restrict__ best, const int *__restrict__ ccs, const float *__restrict__ cpf,
             const double *__restrict__ cpd, const float4 *__restrict__ cent, const float4 *__restrict__ cblo,
             const float4 *__restrict__ cbhi, int *parent, float *__restrict__ log_feat,
             unsigned char *__restrict__ log_lab, long long log_cap, DevCounters *ctr) {
    if (run_failed(ctr)) return;
    constexpr bool LOG = WAVE == 3;
    const int lane = threadIdx.x & 31;
    long long lo = 0, hi = 0;
    if (WAVE == 0) hi = ctr->m;
    else if (WAVE == 1) hi = ctr->P_pos;
    else if (WAVE == 2) { lo = ctr->P_pos; hi = ctr->P_list; }
    else hi = ctr->P_list;
    unsigned rech = 0;
    unsigned long long evals = 0, tested = 0, skipped = 0, linked = 0;
    for (;;) {
        unsigned long long base = 0;
        if (lane == 0) {
            if (WAVE == 0) base = (unsigned long long)atomicAdd(&ctr->cell_next, 32);
            else base = atomicAdd(WAVE == 2 ? &ctr->pair_next2 : &ctr->pair_next, 32ull);
        }
        base = __shfl_sync(0xffffffffu, base, 0);
        if ((long long)base + lo >= hi) break;
        const long long k = lo + (long long)base + lane;
        int a = 0, b = 0;
        bool valid = k < hi;
        if (valid) {
            if (WAVE == 0) {
                // cell k's likeliest link, unless the other cell takes the same pair
                const unsigned long long mine = best[k];
                valid = mine != ~0ull;
                if (valid) {
                    const int2 pr = pairs[(long long)(mine & 0xffffffffu)];
                    const int other = pr.x == (int)k ? pr.y : pr.x;
                    valid = !(best[other] == mine && other < (int)k);
                    a = pr.x;
                    b = pr.y;
                }
            } else {
                const long long idx = LOG ? k : (long long)(sorted[k] & 0xffffffffu);
                const int2 pr = pairs[idx];
                a = pr.x;
                b = pr.y;
                if (!LOG) {
                    // pairs that were some cell's likeliest link ran in wave 0
                    const unsigned long long ba = best[a], bb = best[b];
                    valid = (long long)(ba & 0xffffffffu) != idx && (long long)(bb & 0xffffffffu) != idx;
                }
            }
        }
        bool same = !valid;
        if (valid && !LOG) same = uf_find(parent, a, P.max_iters, ctr) == uf_find(parent, b, P.max_iters, ctr);
        skipped += __popc(__ballot_sync(0xffffffffu, valid && same));
        unsigned todo = __ballot_sync(0xffffffffu, valid && !same);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const int sa = __shfl_sync(0xffffffffu, a, src), sb = __shfl_sync(0xffffffffu, b, src);
            if (!LOG) {
                int again = 0;
                if (lane == 0) again = uf_find(parent, sa, P.max_iters, ctr) == uf_find(parent, sb, P.max_iters, ctr);
                if (__shfl_sync(0xffffffffu, again, 0)) { ++skipped; continue; }
            }
            ++tested;
            const Thr T = P.inst[inst_of_cell(P, sa)].cthr;
            const int a0 = ccs[sa], na = ccs[sa + 1] - a0, b0 = ccs[sb], nb = ccs[sb + 1] - b0;
            int2 wp;
            const bool hit = na >= nb ? bcp_warp<D, M>(a0, na, b0, nb, cpf, cpd, P, T, rech, evals, wp)
                                      : bcp_warp<D, M>(b0, nb, a0, na, cpf, cpd, P, T, rech, evals, wp);
            if (hit) {
                ++linked;
                if (lane == 0 && uf_link(parent, sa, sb, P.max_iters, ctr)) record_link(P, ctr, wp.x, wp.y);
            }
            if (LOG && lane == 0) {
                const long long slot = (long long)base + src;
                if (slot < log_cap) {
                    float x[kMlpIn];
                    pair_features<D>(sa, sb, ccs, cent, cblo, cbhi, sqrtf((float)T.eps2), x);
#pragma unroll
                    for (int i = 0; i < kMlpIn; ++i) log_feat[slot * kMlpIn + i] = x[i];
                    log_lab[slot] = hit ? 1 : 0;
                }
            }
        }
    }
    if (lane == 0) {
        if (tested) atomicAdd(&ctr->pairs_tested, tested);
        if (skipped) atomicAdd(&ctr->pairs_skipped, skipped);
        if (linked) atomicAdd(&ctr->pairs_linked, linked);
    }
    flush_warp_counter(&ctr->band_rechecks, rech);
    if (P.stats) flush_warp_counter(&ctr->dist_evals[1], evals);
}

void launch_connect_learned(int D, int mode, bool log, const RunParams &P, const Bufs &B, const Learned &L,
                            DevCounters *ctr, cudaStream_t s) {
    unsigned long long *best = reinterpret_cast<unsigned long long *>(B.sk0);  // per cell, free in this schedule
    int g = grid_for((const void *)k_uf_reset, 256);
    k_uf_reset<<<g, 256, 0, s>>>(B.parent, B.sk0, ctr); count_launch();
    int count_cands = 1;
    auto collect = [&](auto k) {
        const int gc = grid_for((const void *)k, 256);
        k<<<gc, 256, 0, s>>>(P, B.ccs, B.nbr_cnt, B.nbr, B.nbr_stride, B.nbr_off, B.cblo, B.cbhi, B.parent, L.pairs,
                             L.cap, count_cands, ctr);
        count_launch();
        count_cands = 0;
    };
    auto score = [&](auto k) {
        const int gs = grid_for((const void *)k, 256);
        k<<<gs, 256, 0, s>>>(P, L.pairs, L.w, B.ccs, B.ccent, B.cblo, B.cbhi, L.k0, best, ctr);
        count_launch();
    };
    if (log) {
        // the logging run lists every undecided pair in one pass
        if (D == 8) collect(k_collect_pairs<8, 2>);
        else if (D == 4) collect(k_collect_pairs<4, 2>);
        else if (D == 3) collect(k_collect_pairs<3, 2>);
        else collect(k_collect_pairs<2, 2>);
    } else {
        // box decisions first, then only the pairs union-find has not joined
        if (P.box) {
            if (D == 8) collect(k_collect_pairs<8, 0>);
            else if (D == 4) collect(k_collect_pairs<4, 0>);
            else if (D == 3) collect(k_collect_pairs<3, 0>);
            else collect(k_collect_pairs<2, 0>);
            launch_uf_compress(B.parent, ctr, P.max_iters, s);
        }
        if (D == 8) collect(k_collect_pairs<8, 1>);
        else if (D == 4) collect(k_collect_pairs<4, 1>);
        else if (D == 3) collect(k_collect_pairs<3, 1>);
        else collect(k_collect_pairs<2, 1>);
    }
    k_clamp_pairs<<<1, 1, 0, s>>>(ctr, L.cap); count_launch();
    if (log) {
        GBDB_DISPATCH(D, mode, {
            auto k = k_test_pairs<DD, MM, 3>;
            const int gg = grid_for((const void *)k, 256);
            k<<<gg, 256, 0, s>>>(P, L.pairs, nullptr, best, B.ccs, B.cpf, B.cpd, B.ccent, B.cblo, B.cbhi, B.parent,
                                 L.log_feat, L.log_lab, L.log_cap, ctr);
            count_launch();
        });
        return;
    }
    if (D == 8) score(k_score_pairs<8>);
    else if (D == 4) score(k_score_pairs<4>);
    else if (D == 3) score(k_score_pairs<3>);
    else score(k_score_pairs<2>);
    const int which = radix_sort_u64(L.k0, nullptr, L.k1, nullptr, 0, &ctr->P_list, L.cap, 32, 16, L.scratch,
                                     L.scratch_size, ctr, P.max_iters, s);
    const uint64_t *sorted = which ? L.k1 : L.k0;
    GBDB_DISPATCH(D, mode, {
        auto k0 = k_test_pairs<DD, MM, 0>;
        auto k1 = k_test_pairs<DD, MM, 1>;
        auto k2 = k_test_pairs<DD, MM, 2>;
        const int gg = grid_for((const void *)k1, 256);
        k0<<<gg, 256, 0, s>>>(P, L.pairs, sorted, best, B.ccs, B.cpf, B.cpd, B.ccent, B.cblo, B.cbhi, B.parent,
                              nullptr, nullptr, 0, ctr);
        count_launch();
        launch_uf_compress(B.parent, ctr, P.max_iters, s);
        k1<<<gg, 256, 0, s>>>(P, L.pairs, sorted, best, B.ccs, B.cpf, B.cpd, B.ccent, B.cblo, B.cbhi, B.parent,
                              nullptr, nullptr, 0, ctr);
        count_launch();
        launch_uf_compress(B.parent, ctr, P.max_iters, s);
        k2<<<gg, 256, 0, s>>>(P, L.pairs, sorted, best, B.ccs, B.cpf, B.cpd, B.ccent, B.cblo, B.cbhi, B.parent,
                              nullptr, nullptr, 0, ctr);
        count_launch();
    });
}

}  // namespace gbdb
