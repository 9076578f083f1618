// tdse_autotune: picks the launch shape of the persistent propagation kernels by timing them.
//
// Host code layered on the public calls only (tdse_plan, tdse_set_launch, tdse_copy_state,
// tdse_propagate): the tuner is a client of the library, not a back door into it.  The knobs are
// the ones tdse_set_launch exposes:
//   warps per CTA   the number of segments each instance is cut into (capped per class by
//                   N / max(4K, 16), K the halo), i.e. the depth of the parallel split of every
//                   tridiagonal solve, and the warps sharing one SM's FP64/FP32 pipes;
//   CTAs per SM     how many of those CTAs share an SM (occupancy-limited);
//   slice steps     the time steps a CTA advances a group before it returns the group to the
//                   work queue (load balance vs. scheduling overhead).
// The search is coordinate-wise: (warps, CTAs per SM) over a small grid first, then the slice at
// the best pair.  Every trial starts from the same saved state; the state is put back at the end.
#include "tdse.h"
#include "tdse_internal.h"

#include <algorithm>
#include <string>
#include <vector>

namespace {

struct Trial {
    int warps, per_sm, slice, ctas;
    float ms;
};

}  // namespace

extern "C" tdse_status tdse_autotune(tdse_batch* b, const double* E_dev, double* d_dev, double* a_dev,
                                     int64_t sample_base, int64_t step_begin, int64_t step_end, int32_t repeats,
                                     tdse_tune_trial* trials_host, int32_t max_trials, int32_t* n_trials_host,
                                     void* stream)
{
    using tdse::set_error_message;
    if (!b || !E_dev || !d_dev || !a_dev) return set_error_message("tdse_autotune: NULL argument"), TDSE_ERR_ARG;
    if (step_end <= step_begin || step_begin < 0) return set_error_message("tdse_autotune: empty step range"), TDSE_ERR_ARG;
    if (repeats < 1 || repeats > 100) return set_error_message("tdse_autotune: repeats out of [1, 100]"), TDSE_ERR_ARG;
    if (max_trials < 0 || (max_trials > 0 && !trials_host))
        return set_error_message("tdse_autotune: trials_host is NULL"), TDSE_ERR_ARG;
    tdse_plan_info p0;
    tdse_status st = tdse_plan(b, &p0);
    if (st != TDSE_OK) return st;

    int prev_dev = -1;
    cudaGetDevice(&prev_dev);
    if (cudaSetDevice(tdse::batch_device(b)) != cudaSuccess)
        return set_error_message("tdse_autotune: cudaSetDevice failed"), TDSE_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    void* saved = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    std::vector<Trial> trials;
    auto finish = [&](tdse_status rc) {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaFree(saved);
        if (prev_dev >= 0) cudaSetDevice(prev_dev);
        return rc;
    };
    if (cudaMalloc(&saved, (size_t)std::max<int64_t>(p0.psi_bytes, 16)) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        set_error_message("tdse_autotune: allocation failed");
        return finish(TDSE_ERR_NOMEM);
    }
    if ((st = tdse_copy_state(b, saved, 0, stream)) != TDSE_OK) return finish(st);

    // one trial: set the shape, then `repeats` timed propagations, each from the saved state
    auto run = [&](int warps, int per_sm, int slice, bool warm) -> tdse_status {
        tdse_status r = tdse_set_launch(b, warps, per_sm, slice, 0);
        if (r != TDSE_OK) return r;
        tdse_plan_info p;
        if ((r = tdse_plan(b, &p)) != TDSE_OK) return r;
        for (const Trial& t : trials)   // same effective shape as an earlier trial: nothing new to learn
            if (t.warps == p.warps_per_cta && t.ctas == p.ctas && t.slice == p.slice_steps) return TDSE_OK;
        float best = 1e30f;
        for (int k = 0; k < repeats + (warm ? 1 : 0); ++k) {
            if ((r = tdse_copy_state(b, saved, 1, stream)) != TDSE_OK) return r;
            if (cudaEventRecord(e0, s) != cudaSuccess) return set_error_message("tdse_autotune: event record"), TDSE_ERR_CUDA;
            if ((r = tdse_propagate(b, E_dev, d_dev, a_dev, sample_base, step_begin, step_end, stream)) != TDSE_OK) return r;
            if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess)
                return set_error_message("tdse_autotune: probe launch failed"), TDSE_ERR_CUDA;
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (!(warm && k == 0)) best = std::min(best, ms);
        }
        trials.push_back({p.warps_per_cta, per_sm, p.slice_steps, p.ctas, best});
        return TDSE_OK;
    };

    const int warps_grid[] = {4, 6, 8, 12, 16};
    // k CTAs per SM make each group's step ~k times longer (the SM is shared): when the longest
    // group's time exceeds half the work per SM (an uneven batch), two CTAs per SM lengthen the job
    // although the first steps, which the trials time, run faster
    const int per_sm_grid[] = {1, p0.longest_share > 0.5 ? 1 : 2};
    bool first = true;
    for (int w : warps_grid)
        for (int c : per_sm_grid) {
            if ((st = run(w, c, 16, first)) != TDSE_OK) return finish(st);
            first = false;
        }
    auto best_of = [&]() {
        return *std::min_element(trials.begin(), trials.end(), [](const Trial& x, const Trial& y) { return x.ms < y.ms; });
    };
    Trial bw = best_of();
    for (int sl : {8, 32, 64})
        if ((st = run(bw.warps, bw.per_sm, sl, false)) != TDSE_OK) return finish(st);
    const Trial best = best_of();
    if ((st = tdse_set_launch(b, best.warps, best.per_sm, best.slice, 0)) != TDSE_OK) return finish(st);
    if ((st = tdse_copy_state(b, saved, 1, stream)) != TDSE_OK) return finish(st);
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        set_error_message("tdse_autotune: synchronize failed");
        return finish(TDSE_ERR_CUDA);
    }
    const int n = std::min((int)trials.size(), (int)max_trials);
    for (int i = 0; i < n; ++i) {
        trials_host[i].warps_per_cta = trials[i].warps;
        trials_host[i].ctas_per_sm = trials[i].per_sm;
        trials_host[i].slice_steps = trials[i].slice;
        trials_host[i].ctas = trials[i].ctas;
        trials_host[i].ms = trials[i].ms;
    }
    if (n_trials_host) *n_trials_host = (int32_t)trials.size();
    return finish(TDSE_OK);
}
