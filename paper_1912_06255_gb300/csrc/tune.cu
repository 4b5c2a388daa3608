// Autotuner of the run configuration: which pair schedule, whether cell boxes
// decide pairs, one or two connectivity waves, core cells per work item of
// the connectivity kernel, resident blocks per SM of the persistent kernels
// and which sparse cells MarkCore counts with one thread per point.  It times candidate configurations on the caller's own input (the
// result does not depend on any of them, only the time does) by coordinate
// descent from the context's current setting, keeps the fastest and leaves
// it set in the context.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <vector>

#include "ctx.cuh"

namespace {

struct Knob {
    int option;
    std::vector<int64_t> values;
};

template <typename RunFn>
dbscan_status tune(dbscan_ctx *c, int reps, dbscan_tuning *out, bool high_dim, RunFn run_once) {
    if (reps < 1 || reps > 100) return DBSCAN_ERR_INVALID_ARG;
    std::vector<Knob> knobs = {
        {DBSCAN_OPT_SCHEDULE, {DBSCAN_SCHED_SIZE, DBSCAN_SCHED_NONE, DBSCAN_SCHED_LEARNED}},
        {DBSCAN_OPT_CELL_BOUNDS, {1, 0}},
        {DBSCAN_OPT_CONNECT_WAVES, {2, 1}},
        {DBSCAN_OPT_CONNECT_CELLS, {1, 2, 4, 8}},
        {DBSCAN_OPT_BLOCKS_PER_SM, {0, 1, 2, 4}},
        {DBSCAN_OPT_SMALL_CELLS, {0, 128, 1 << 30}},
        {DBSCAN_OPT_PAIR_BOXES, {1, 0}},
    };
    if (high_dim && c->precision == DBSCAN_PREC_FP32_RECHECK) knobs.push_back({DBSCAN_OPT_QUADTREE, {0, 2}});
    if (c->precision != DBSCAN_PREC_FP32_RECHECK) knobs.erase(knobs.begin() + 1);  // boxes need the FP32 band
    std::vector<int64_t> cur(knobs.size());
    for (size_t k = 0; k < knobs.size(); ++k) dbscan_get_option(c, knobs[k].option, &cur[k]);
    int trials = 0;
    auto measure = [&](float *ms) -> dbscan_status {
        dbscan_status st = run_once();  // warm-up (and graph capture for batches)
        if (st != DBSCAN_OK) return st;
        float best = 0.f;
        for (int r = 0; r < reps; ++r) {
            const auto t0 = std::chrono::steady_clock::now();
            st = run_once();
            const auto t1 = std::chrono::steady_clock::now();
            if (st != DBSCAN_OK) return st;
            const float t = std::chrono::duration<float, std::milli>(t1 - t0).count();
            best = r == 0 ? t : std::min(best, t);
        }
        *ms = best;
        ++trials;
        return DBSCAN_OK;
    };
    auto apply = [&](const std::vector<int64_t> &v) {
        for (size_t k = 0; k < knobs.size(); ++k) dbscan_set_option(c, knobs[k].option, v[k]);
    };
    apply(cur);
    float best_ms = 0.f;
    dbscan_status st = measure(&best_ms);
    if (st != DBSCAN_OK) return st;
    const float default_ms = best_ms;
    for (size_t k = 0; k < knobs.size(); ++k) {
        for (int64_t v : knobs[k].values) {
            if (v == cur[k]) continue;
            std::vector<int64_t> cand = cur;
            cand[k] = v;
            apply(cand);
            float ms = 0.f;
            st = measure(&ms);
            if (st != DBSCAN_OK) {
                apply(cur);
                return st;
            }
            if (ms < best_ms) {
                best_ms = ms;
                cur = cand;
            }
        }
    }
    apply(cur);
    if (out) {
        int64_t v = 0;
        dbscan_get_option(c, DBSCAN_OPT_SCHEDULE, &v); out->schedule = (int32_t)v;
        dbscan_get_option(c, DBSCAN_OPT_CELL_BOUNDS, &v); out->cell_bounds = (int32_t)v;
        dbscan_get_option(c, DBSCAN_OPT_CONNECT_WAVES, &v); out->connect_waves = (int32_t)v;
        dbscan_get_option(c, DBSCAN_OPT_CONNECT_CELLS, &v); out->connect_cells = (int32_t)v;
        dbscan_get_option(c, DBSCAN_OPT_BLOCKS_PER_SM, &v); out->blocks_per_sm = (int32_t)v;
        dbscan_get_option(c, DBSCAN_OPT_SMALL_CELLS, &v); out->small_cells = (int32_t)v;
        dbscan_get_option(c, DBSCAN_OPT_PAIR_BOXES, &v); out->pair_boxes = (int32_t)v;
        dbscan_get_option(c, DBSCAN_OPT_QUADTREE, &v); out->quadtree = (int32_t)v;
        out->trials = trials;
        out->best_ms = best_ms;
        out->default_ms = default_ms;
    }
    return DBSCAN_OK;
}

}  // namespace

dbscan_status dbscan_autotune(dbscan_ctx *c, const void *d_points, int64_t n, int d, int dtype, double eps,
                              int64_t min_pts, int reps, dbscan_tuning *out, void *stream) {
    if (!c || n < 1 || n > c->max_points) return DBSCAN_ERR_INVALID_ARG;
    uint8_t *core = nullptr;
    int32_t *labels = nullptr;
    if (cudaMalloc((void **)&core, (size_t)n) != cudaSuccess ||
        cudaMalloc((void **)&labels, sizeof(int32_t) * (size_t)n) != cudaSuccess) {
        (void)cudaGetLastError();
        cudaFree(core);
        return DBSCAN_ERR_OOM;
    }
    const dbscan_status st = tune(c, reps, out, d >= 5, [&]() {
        return dbscan_run(c, d_points, n, d, dtype, eps, min_pts, core, labels, nullptr, nullptr, stream);
    });
    cudaFree(core);
    cudaFree(labels);
    return st;
}

dbscan_status dbscan_autotune_batch(dbscan_ctx *c, const dbscan_instance *host_desc, int count,
                                    const void *d_points, int ld, int dtype, int reps, dbscan_tuning *out,
                                    void *stream) {
    if (!c || !host_desc || count < 1) return DBSCAN_ERR_INVALID_ARG;
    int64_t total = 0;
    for (int i = 0; i < count; ++i) total += host_desc[i].n;
    if (total < 1 || total > c->max_points) return DBSCAN_ERR_INVALID_ARG;
    uint8_t *core = nullptr;
    int32_t *labels = nullptr;
    if (cudaMalloc((void **)&core, (size_t)total) != cudaSuccess ||
        cudaMalloc((void **)&labels, sizeof(int32_t) * (size_t)total) != cudaSuccess) {
        (void)cudaGetLastError();
        cudaFree(core);
        return DBSCAN_ERR_OOM;
    }
    const dbscan_status st = tune(c, reps, out, false, [&]() {
        return dbscan_run_batch(c, host_desc, count, d_points, ld, dtype, core, labels, nullptr, nullptr, stream);
    });
    cudaFree(core);
    cudaFree(labels);
    return st;
}
