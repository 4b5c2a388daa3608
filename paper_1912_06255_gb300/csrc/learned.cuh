// Learned pair scheduler: network shape, parameter layout and launchers.
#pragma once

#include "grid.cuh"

namespace gbdb {

constexpr int kMlpIn = 6, kMlpHid = 32;
constexpr int kOW1 = 0, kOB1 = kOW1 + kMlpHid * kMlpIn, kOW2 = kOB1 + kMlpHid, kOB2 = kOW2 + kMlpHid * kMlpHid;
constexpr int kOW3 = kOB2 + kMlpHid, kOB3 = kOW3 + kMlpHid;
constexpr int kMlpParams = kOB3 + 1;  // 1313

// Device state of the learned schedule.
struct Learned {
    float *w;           // [kMlpParams] network parameters
    int2 *pairs;        // [cap] undecided core-cell pairs of the run
    uint64_t *k0, *k1;  // [cap] sort keys (score, pair index)
    long long cap;
    void *scratch;      // radix-sort scratch for cap keys
    size_t scratch_size;
    float *log_feat;    // [log_cap][kMlpIn] logging run: features
    unsigned char *log_lab;  // [log_cap] logging run: 1 = connected
    long long log_cap;
};

void launch_connect_learned(int D, int mode, bool log, const RunParams &P, const Bufs &B, const Learned &L,
                            DevCounters *ctr, cudaStream_t s);

// Mean BCE-with-logits loss and its gradient over samples first .. first+n-1
// (indices taken modulo total), added into grad[] and loss[0].
void mlp_loss_grad(const float *w, const float *feat, const unsigned char *lab, long long first, long long n,
                   long long total, float *grad, float *loss, cudaStream_t s);
void mlp_adam(float *w, const float *g, float *m1, float *m2, float lr, int t, cudaStream_t s);

}  // namespace gbdb
