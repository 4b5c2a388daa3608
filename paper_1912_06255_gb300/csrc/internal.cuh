// Internal declarations shared by the translation units of the CUDA library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dbscan_gb300.h"

namespace gbdb {

constexpr int kMaxDim = 8;        // widest point storage
constexpr int kMaxEnumDim = 4;    // neighbour cells by offset enumeration (Sec. 4.1)
constexpr int kMaxOffsets = 840;  // candidate offsets for d = 4
constexpr uint64_t kEmptyKey = ~0ull;
constexpr int kBorderSetCap = 256;  // >= kissing number of R^8 (240), see border.cu

// Device-resident status and counters of one run (zeroed at the start).
struct DevCounters {
    int err;         // first error code (dbscan_status), 0 if none
    int err_info;    // kernel-specific detail of the first error
    int m;           // non-empty cells
    int ms;          // non-empty supercells (d = 2, 3: blocks of 2^d cells)
    int m_core;      // core cells
    int n_core;      // core points
    int n_border;    // border points
    int n_noncore;   // non-core points (border candidates)
    int n_heavy;     // of which with more than 2 cluster names (recomputed by the fill pass)
    int cell_next;   // BCP work counters (ranked cells taken), near and far wave
    int cell_next2;
    int P_list;      // undecided pairs listed by the learned schedule
    int P_pos;       // ... of which the network predicts connected
    unsigned long long P_demand;  // pairs the learned schedule tried to list (sizes a retry)
    long long E;     // neighbour list entries
    long long P;     // candidate core-cell pairs
    long long K;     // border memberships
    unsigned long long pair_next, pair_next2;  // BCP work counters of the pair waves
    unsigned long long pairs_tested, pairs_skipped, pairs_linked, pairs_box;
    unsigned long long band_rechecks;
    unsigned long long dist_evals[3];  // MarkCore, BCP, border
    unsigned long long mc_bound;       // MarkCore pair tests without early exit
    unsigned long long n_wit;          // union-find hooks recorded as link witnesses
};

// Decision thresholds of one problem instance.
struct Thr {
    double eps2;  // fl(eps * eps), the FP64 threshold
    float lo, hi; // FP32 band: <= lo is in, > hi is out, otherwise FP64 recheck
    int min_pts;  // clamped to n + 1
};

// Grid and thresholds of one problem instance (one entry per instance of a
// batch; a single run has one).
struct Inst {
    double origin[kMaxDim];   // per-dimension minimum of the instance's points
    float origin32[kMaxDim];  // fl32(origin): exact for FP32 input (a minimum of FP32 values)
    double inv_s;             // 1 / cell side
    float inv_s32;            // fl32(inv_s), for the FP32 estimate of the cell coordinates
    int kmax[kMaxDim];        // largest cell coordinate per dimension
    int bits;                 // Morton bits per dimension
    int d;                    // the instance's dimension (<= the storage dimension)
    int row0, n;              // rows [row0, row0 + n) of the input
    Thr thr;                  // eps: MarkCore, ClusterBorder, neighbouring cells
    Thr cthr;                 // connectivity of core cells (ClusterCore): eps, or
                              // eps(1 + rho) for rho-approximate DBSCAN (Sec. 2)
};

// Per-run scalars passed by value to the kernels.
struct RunParams {
    int n;        // points (all instances)
    int d;        // storage dimension (padded coordinates are zero)
    int max_iters;
    int stats;    // count distance evaluations
    int box;      // cell bounding boxes prune pairs (FP32-band mode only)
    int ninst;    // instances; 1 for a single run
    int inst_shift;  // instance id sits in key bits >= inst_shift (ninst > 1)
    const Inst *inst;     // [ninst] device
    const int *cell_inst; // [m] device: instance of each cell (ninst > 1)
    int cn_cells;   // core cells per work item of the connectivity kernel
    int waves;      // 2: adjacent pairs, compression, farther pairs; 1: one wave
    int mc_small_nbr;  // neighbourhood limit of MarkCore's thread-per-point cells (0: off)
    int pair_box;      // core-point boxes decide pairs in ClusterCore and ClusterBorder (with box)
    int qt;            // quadtree levels below the cell for MarkCore's range counts (d >= 5, box mode), 0: off
    int2 *wit;         // null, or [wit_cap]: per union-find hook, a pair of compacted core points within eps
    long long wit_cap;
    // copies of instance 0 for single runs (host side convenience)
    int min_pts;
    double eps2;
    float lo, hi;
};

__device__ __forceinline__ int inst_of_cell(const RunParams &P, int c) {
    return P.ninst > 1 ? P.cell_inst[c] : 0;
}

// Storage width of a point: 2, 4 or 8 coordinates (zero padded).
template <int D> struct Store { static constexpr int SD = D <= 2 ? 2 : (D <= 4 ? 4 : 8); };

// Precision/storage modes of the distance kernels.
enum Mode : int {
    kF64FromF32 = 0,  // FP64 predicate on widened FP32 storage
    kF64FromF64 = 1,  // FP64 predicate on FP64 storage
    kF32FromF32 = 2,  // FP32 band test, FP64 recheck on widened FP32 storage
    kF32FromF64 = 3   // FP32 band test, FP64 recheck on FP64 storage
};

__device__ __forceinline__ void set_error(DevCounters *c, int code, int info) {
    if (atomicCAS(&c->err, 0, code) == 0) c->err_info = info;
}

// Once a step has failed (a bounded wait gave up, a buffer was too small),
// the kernels after it leave at entry: their inputs may be incomplete, and
// values taken from them must not be used as indices.  One lane reads the
// status word and the warp follows it, so a warp never splits before its
// full-warp collectives; run_failed_block makes the same decision for a whole
// block (kernels with __syncthreads).
__device__ __forceinline__ bool run_failed(const DevCounters *ctr) {
    return __shfl_sync(0xffffffffu, *(const volatile int *)&ctr->err, 0) != 0;
}
__device__ __forceinline__ bool run_failed_block(const DevCounters *ctr) {
    __shared__ int s_failed;
    __syncthreads();
    if (threadIdx.x == 0) s_failed = *(const volatile int *)&ctr->err;
    __syncthreads();
    return s_failed != 0;
}

// ---------------------------------------------------------------- primitives
// Exclusive scan of in[0..n) into out[0..n], out[n] = total.  n = *n_dev when
// n_dev is non-null, else n_host; n_max bounds n and sizes the grid.  out may
// alias in.  part must hold scan_partials(n_max) entries.
int64_t scan_partials(int64_t n_max);
void scan_i32_to_i32(const int *in, int *out, int64_t n_host, const int *n_dev, int64_t n_max,
                     long long *part, cudaStream_t s);
void scan_i64_to_i64(const long long *in, long long *out, int64_t n_host, const int *n_dev,
                     int64_t n_max, long long *part, cudaStream_t s);

// Stable LSD radix sort of 64-bit keys on key bits [lo, lo + bits), 8 bits a
// pass, optionally carrying 32-bit values (v0/v1 null: keys only).
// Ping-pongs between (k0, v0) and (k1, v1); returns 0 if the result is in
// (k0, v0), 1 if in (k1, v1).  scratch holds scratch_bytes bytes, at least
// sort_scratch_bytes(n_max); a smaller scratch sorts nothing and raises
// CAPACITY in ctr->err.  Look-back waits are bounded by max_iters
// (DEVICE_TIMEOUT in ctr->err).
size_t sort_scratch_bytes(int64_t n_max);
int radix_sort_u64(uint64_t *k0, uint32_t *v0, uint64_t *k1, uint32_t *v1, int n_host, const int *n_dev,
                   int64_t n_max, int lo, int bits, void *scratch, size_t scratch_bytes, DevCounters *ctr, int max_iters,
                   cudaStream_t s);

// Kernel launches issued by this thread (read before and after a run).
extern thread_local long long g_launches;
inline void count_launch() { ++g_launches; }

// Persistent-grid size for a kernel: resident blocks per SM x SM count,
// capped by the blocks-per-SM limit this thread set (0 = no cap).
int grid_for(const void *kernel, int threads, size_t smem = 0);
void set_grid_cap(int blocks_per_sm);
int grid_cap();

}  // namespace gbdb
