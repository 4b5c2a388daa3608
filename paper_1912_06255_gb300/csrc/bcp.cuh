// BCP connectivity test of two cells' core points and the (D, mode) kernel
// dispatch, shared by the size-ordered and the learned pair schedules.
// D is the compiled width: 2, 3 or 4 for d <= 4, and 8 for 5 <= d <= 8
// (zero-padded coordinates add exact zeros to every sum).
#pragma once

#include "geom.cuh"

namespace gbdb {

#define GBDB_DISPATCH(D, MODE, ...)                                     \
    do {                                                                \
        switch ((D) * 4 + (MODE)) {                                     \
        case 8: { constexpr int DD = 2, MM = 0; __VA_ARGS__; } break;   \
        case 9: { constexpr int DD = 2, MM = 1; __VA_ARGS__; } break;   \
        case 10: { constexpr int DD = 2, MM = 2; __VA_ARGS__; } break;  \
        case 11: { constexpr int DD = 2, MM = 3; __VA_ARGS__; } break;  \
        case 12: { constexpr int DD = 3, MM = 0; __VA_ARGS__; } break;  \
        case 13: { constexpr int DD = 3, MM = 1; __VA_ARGS__; } break;  \
        case 14: { constexpr int DD = 3, MM = 2; __VA_ARGS__; } break;  \
        case 15: { constexpr int DD = 3, MM = 3; __VA_ARGS__; } break;  \
        case 16: { constexpr int DD = 4, MM = 0; __VA_ARGS__; } break;  \
        case 17: { constexpr int DD = 4, MM = 1; __VA_ARGS__; } break;  \
        case 18: { constexpr int DD = 4, MM = 2; __VA_ARGS__; } break;  \
        case 19: { constexpr int DD = 4, MM = 3; __VA_ARGS__; } break;  \
        case 32: { constexpr int DD = 8, MM = 0; __VA_ARGS__; } break;  \
        case 33: { constexpr int DD = 8, MM = 1; __VA_ARGS__; } break;  \
        case 34: { constexpr int DD = 8, MM = 2; __VA_ARGS__; } break;  \
        case 35: { constexpr int DD = 8, MM = 3; __VA_ARGS__; } break;  \
        default: break;                                                 \
        }                                                               \
    } while (0)

// Connected(g, h) over core points (Sec. 4.4, BCP-based cell graph): stop at
// the first pair within eps.  The warp tests a block of 32 point pairs per
// step and leaves on a warp vote.  The smaller cell's points stay in
// registers: with nc <= 32 columns, each lane holds one column point and the
// warp covers 32/L rows per step (L = lanes per row).  On a hit, wit (the
// same on every lane) receives the pair found, as compacted core indices.
template <int D, int M>
__device__ __forceinline__ bool bcp_warp(int r0, int nr, int c0, int nc, const float *__restrict__ cpf,
                                         const double *__restrict__ cpd, const RunParams &P, const Thr &T,
                                         unsigned &rech, unsigned long long &evals, int2 &wit) {
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
                t = within(p, q, T, cpd, r0 + r, cpd, c0 + j, rech);
            }
            const unsigned hb = __ballot_sync(0xffffffffu, t);
            if (hb) {
                const int src = __ffs(hb) - 1;
                wit = make_int2(r0 + rb + (src >> lg), c0 + (src & (L - 1)));
                return true;
            }
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
                t = within(p, q, T, cpd, r0 + r, cpd, c0 + j, rech);
            }
            const unsigned hb = __ballot_sync(0xffffffffu, t);
            if (hb) {
                wit = make_int2(r0 + r, c0 + cb + __ffs(hb) - 1);
                return true;
            }
        }
    }
    return false;
}


}  // namespace gbdb
