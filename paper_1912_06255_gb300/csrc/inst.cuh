// Grid and threshold parameters of one problem instance, built from its
// bounding box.  Host and device share this code: single runs build their
// instance on the host after reading the box back, batches build every
// instance on the device.
#pragma once

#include <math.h>

#include "internal.cuh"

namespace gbdb {

// FP32 band around T = fl(eps^2).  f is the FP32 value of sum (p'_i - q'_i)^2
// for coordinates p', q' rounded to FP32 (each within E_coord of the input);
// E is the resulting bound on |‖p'-q'‖ - ‖p-q‖|.  With the forward-error bounds
// |f - ‖p'-q'‖^2| <= g32 ‖p'-q'‖^2 and |fl64(d^2) - d^2| <= g64 d^2 (sums of
// non-negative rounded terms), f <= lo implies the FP64 predicate holds and
// f > hi implies it fails:
//   lo = (1 - g32) (sqrt(T / (1 + g64)) - E)^2,  hi = (1 + g32) (sqrt(T / (1 - g64)) + E)^2.
// Rounding of this host arithmetic is absorbed by 2^-40 margins.
__host__ __device__ inline bool fp32_band(double T, int d, double E, float *lo, float *hi) {
    if (!(T >= 0x1p-60 && T <= 0x1p60)) return false;
    const double g32 = 2.0 * (d + 2) * 0x1p-24, g64 = 2.0 * (d + 2) * 0x1p-53;
    const double rT = sqrt(T);
    if (!(E <= 0.25 * rT)) return false;
    const double a = sqrt(T / (1.0 + g64)) * (1.0 - 0x1p-40) - E;
    const double b = sqrt(T / (1.0 - g64)) * (1.0 + 0x1p-40) + E;
    const double lo_d = (1.0 - g32) * a * a * (1.0 - 0x1p-40);
    const double hi_d = (1.0 + g32) * b * b * (1.0 + 0x1p-40);
    float l = (float)lo_d, h = (float)hi_d;
    if ((double)l > lo_d) l = nextafterf(l, -INFINITY);
    if ((double)h < hi_d) h = nextafterf(h, INFINITY);
    if (!(l > 0.0f) || !isfinite(h)) return false;
    *lo = l;
    *hi = h;
    return true;
}

// Cell side s = fl(eps / sqrt(d)) * (1 - 2^-20) (Sec. 3, shrunk so that points
// of one cell pass the FP64 predicate despite rounding); cell coordinates
// k_j = floor(fl(fl(x_j - lo_j) * fl(1/s))), kmax_j from the box; Morton bits
// per dimension enough for the largest kmax.  key_limit bounds d * bits.
// want_fp32: use the FP32 band if it is valid for this instance (fp32 = 1).
// rho > 0: rho-approximate connectivity (Sec. 2, after Gan and Tao): core
// cells are joined by pairs within fl(eps * fl(1 + rho)) (cthr), while core
// points, neighbouring cells and border sets keep eps (thr).
// Returns DBSCAN_OK or DBSCAN_ERR_KEY_OVERFLOW.
__host__ __device__ inline int build_inst(Inst &I, double eps, long long min_pts, int n, int d, const double *lo,
                                          const double *hi, bool f64, bool want_fp32, int key_limit, int *fp32,
                                          double rho = 0.0) {
    for (int j = 0; j < kMaxDim; ++j) {
        I.origin[j] = 0.0;
        I.origin32[j] = 0.f;
        I.kmax[j] = 0;
    }
    I.d = d;
    I.n = n;
    I.thr.min_pts = (int)(min_pts < (long long)n + 1 ? min_pts : (long long)n + 1);
    I.thr.eps2 = eps * eps;
    I.thr.lo = 0.f;
    I.thr.hi = 0.f;
    const double side = (eps / sqrt((double)d)) * (1.0 - 0x1p-20);
    I.inv_s = 1.0 / side;
    I.inv_s32 = (float)I.inv_s;
    int kmax_all = 0;
    double M = 0.0;
    for (int j = 0; j < d; ++j) {
        I.origin[j] = lo[j];
        I.origin32[j] = (float)lo[j];
        const double t = (hi[j] - lo[j]) * I.inv_s;
        if (!(t < 0x1p30)) return DBSCAN_ERR_KEY_OVERFLOW;
        I.kmax[j] = (int)floor(t);
        kmax_all = kmax_all > I.kmax[j] ? kmax_all : I.kmax[j];
        const double a = fabs(lo[j]) > fabs(hi[j]) ? fabs(lo[j]) : fabs(hi[j]);
        M = M > a ? M : a;
    }
    int bits = 1;
    while (bits < 31 && (1 << bits) <= kmax_all) ++bits;
    I.bits = bits;
    if (d * bits > key_limit) return DBSCAN_ERR_KEY_OVERFLOW;
    *fp32 = 0;
    double E = 0.0;
    if (want_fp32) {
        E = f64 ? sqrt((double)d) * (2.0 * M * 0x1p-24 + 0x1p-148) : 0.0;
        *fp32 = fp32_band(I.thr.eps2, d, E, &I.thr.lo, &I.thr.hi) ? 1 : 0;
    }
    I.cthr = I.thr;
    if (rho > 0.0) {
        const double r = eps * (1.0 + rho);
        I.cthr.eps2 = r * r;
        // no valid band for the wider threshold: every FP32 value goes to the
        // FP64 recheck (lo = 0 only admits coincident points)
        if (*fp32 && !fp32_band(I.cthr.eps2, d, E, &I.cthr.lo, &I.cthr.hi)) {
            I.cthr.lo = 0.f;
            I.cthr.hi = INFINITY;
        }
    }
    return DBSCAN_OK;
}

}  // namespace gbdb
