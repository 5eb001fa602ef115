// k_tsplit.h -- launcher of the split-shape analytic Jacobian (k_tsplit.cu).
#pragma once

#include "gbk_internal.cuh"

namespace gbk {

constexpr int kTsplitMaxR = 8;  // largest PSF radius the stages are compiled for

// One call: n_models parameter sets, each model's galaxy from obs_list[m]
// (or obs for all), skip[m] != 0 leaves model m's outputs untouched.
struct TsplitCall {
    Geom g;
    int n_models;
    const double *params;     // device [n_models][GBK_NPAR]
    gbk_obs obs;
    const gbk_obs *obs_list;  // device [n_models] or null
    const int32_t *skip;      // device [n_models] or null
    const float *cot;         // device [n_models][2][ny][nx] or null (the residuals)
    int np;                   // free parameters (among x0 .. sigma0)
    int free_idx[GBK_NPAR];
    double *jtj;              // device [n_models][np][np] or null
    double *jtv;              // device [n_models][np] or null
    double *chi2;             // device [n_models] or null: sum of squared residuals
};

// The cube model at u = 1, PSF radius <= kTsplitMaxR, free parameters among
// x0 .. sigma0.
bool tsplit_supported(const Geom &g, int np, const int *free_idx);
// Workspace of a call over n_models (0 when the geometry is not served).
size_t tsplit_workspace_bytes(const Geom &g, int n_models);
// Asynchronous on st.
gbk_status launch_tsplit(const TsplitCall &call, void *ws, size_t ws_bytes, cudaStream_t st);
// Reads and clears the PSF stage's TMA wait status (1 = a load timed out).
gbk_status tsplit_status_read(int *v);

}  // namespace gbk
