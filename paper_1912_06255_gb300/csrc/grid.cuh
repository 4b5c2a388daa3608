// Host-side launchers of the phase kernels (one stream, no host sync inside).
#pragma once

#include "internal.cuh"

namespace gbdb {

// ---- cells (grid.cu)
void launch_bbox(const void *X, int dtype, int n, int d, double *part, int nb, int *bad,
                 double *out, cudaStream_t s);
void launch_keys(const void *X, int dtype, const RunParams &P, uint64_t *keys, uint32_t *vals,
                 cudaStream_t s);
void launch_cells(const void *X, int dtype, int n, int d, int SD, const uint64_t *K, const uint32_t *V,
                  int *flags, int *cid, long long *part, float *pf, double *pd, int *orig,
                  int *cell_of, int *cell_start, uint64_t *cell_key, DevCounters *ctr, cudaStream_t s);
void launch_hash(uint64_t *hk, int *hv, const uint64_t *cell_key, DevCounters *ctr, cudaStream_t s);
void launch_neighbors(const uint64_t *cell_key, const uint64_t *hk, const int *hv, const RunParams &P,
                      const signed char *offs, int noff, long long *cnt, long long *off, int *nbr, long long nbr_cap,
                      long long *part, int64_t n_max, DevCounters *ctr, cudaStream_t s);

// Device arrays of one run, shared by the cluster phases.
struct Bufs {
    // sorted points and cell table
    const float *pf;
    const double *pd;  // null unless FP64 input
    const int *orig, *cell_of, *cell_start;
    const long long *nbr_off;
    const int *nbr;
    // MarkCore / compaction
    int *core_s;        // [n] 0/1 in cell order
    int *core_pos;      // [n+1] exclusive scan of core_s
    int *ccs;           // [m+1] core points of cell c: [ccs[c], ccs[c+1]) of the compacted arrays
    float *cpf;         // compacted core points
    double *cpd;
    int *core_orig;     // input index of compacted core point
    int *core_cell;     // cell of compacted core point
    // schedule
    uint64_t *sk0, *sk1;
    uint32_t *sv0, *sv1;
    unsigned *hist;
    int *rank;          // [m] position of the cell in test order
    long long *pcnt, *poff;
    int2 *pairs;
    long long pair_cap;
    // union-find and labels
    int *parent, *compmin, *cell_label;
    // border
    long long *bcount, *boff;
    long long *part;
    int64_t n_max;
};

// ---- clusters (cluster.cu)
void launch_markcore(int D, int mode, const RunParams &P, const Bufs &B, DevCounters *ctr, cudaStream_t s);
void launch_core_compact(int SD, const RunParams &P, const Bufs &B, DevCounters *ctr, cudaStream_t s);
void launch_schedule(int sched, const RunParams &P, const Bufs &B, DevCounters *ctr, cudaStream_t s);
void launch_connect(int D, int mode, const RunParams &P, const Bufs &B, DevCounters *ctr, cudaStream_t s);
void launch_labels(const RunParams &P, const Bufs &B, uint8_t *core_out, int32_t *labels_out,
                   DevCounters *ctr, cudaStream_t s);
// count pass (fill = false) or fill pass (fill = true, ids != null)
void launch_border(int D, int mode, bool fill, const RunParams &P, const Bufs &B, int32_t *labels_out,
                   int32_t *ids, long long ids_cap, DevCounters *ctr, cudaStream_t s);

}  // namespace gbdb
