// k_split.h -- launcher of the two-stage fused evaluator (k_split.cu).
#pragma once

#include <cuda.h>

#include "gbk_internal.cuh"

namespace gbk {

constexpr int kSplitMaxR = 8;  // largest PSF radius the PSF stage is compiled for

// Geometries the two-stage evaluator serves (cube model, u = 1, R <= 8).
bool split_supported(const Geom &g);
// Workspace of a call over n_models (0 when the geometry is not served).
size_t split_workspace_bytes(const Geom &g, int n_models);
// chi2 (and optionally maps and residuals) of n models; asynchronous on st.
// CUDA events recorded on the launch stream around every launch of a call
// (start, after the set-up, after each stage-A and stage-B launch), for the
// per-stage timings of gbk_split_stage_times.
struct SplitTimer {
    cudaEvent_t ev[64] = {};
    int n = 0;
    cudaError_t mark(cudaStream_t st)
    {
        if (n >= 64) return cudaErrorInvalidValue;
        cudaError_t e = cudaEventCreate(&ev[n]);
        if (e != cudaSuccess) return e;
        return cudaEventRecord(ev[n++], st);
    }
    void release()
    {
        for (int i = 0; i < n; ++i) cudaEventDestroy(ev[i]);
        n = 0;
    }
};

// The driver's cuTensorMapEncodeTiled (null when the driver lacks it).
typedef CUresult (*SplitEncodeFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
SplitEncodeFn split_encode_fn();

// Per host thread and device: a stream for the PSF stages of the two-stage
// kernels, which run there while the next chunk's line stage runs on the
// caller's stream, and the events that order them (two per stage, one per
// plane buffer).  Created on first use and kept for the process.
struct SplitAux {
    cudaStream_t s = nullptr;
    cudaEvent_t line[2] = {nullptr, nullptr}, psf[2] = {nullptr, nullptr};
    cudaEvent_t start = nullptr, obs = nullptr;  // a host-buffer call's start and its maps' arrival
};
gbk_status split_aux(SplitAux **out);

// Reads and clears the PSF stage's TMA wait status (1 = a load timed out).
gbk_status split_status_read(int *v);

// A batched call's galaxies: models i*mpg .. i*mpg + mpg - 1 belong to galaxy
// i, which is compared with obs_list[i] (device, or null: *obs for all) and
// left alone when skip[i] != 0 (device, or null).
struct SplitBatch {
    const gbk_obs *obs_list;
    const int32_t *skip;
    int mpg;
};
// obs_ready (or null): an event the first PSF stage waits for (the observed
// maps' copy); the line stages do not read the maps.
gbk_status launch_split(const Geom &g, int n, const double *params, const gbk_obs *obs, float *maps, double *chi2,
                        float *resid, void *ws, size_t ws_bytes, cudaStream_t st, SplitTimer *timer = nullptr,
                        const SplitBatch *batch = nullptr, cudaEvent_t obs_ready = nullptr);

}  // namespace gbk
