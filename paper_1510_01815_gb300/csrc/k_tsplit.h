// k_tsplit.h -- launcher of the split-shape analytic Jacobian (k_tsplit.cu).
#pragma once

#include <vector>

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

// Ragged batches: one model per galaxy, each galaxy with its own geometry
// (the survey).  The plan holds the per-galaxy rows per stage-A CTA, table
// and plane offsets, first part slots, the chunks whose planes fit the L2
// budget (galaxies ordered by PSF radius; a chunk has one radius) and their
// work items, and the workspace layout; it depends on the geometries only.
struct TsRaggedPlan {
    bool ok = false;  // every galaxy served (cube model, u = 1, PSF radius <= kTsplitMaxR)
    int n = 0;
    std::vector<int> tab_off, ra, tile_base;
    std::vector<long long> pl_off;      // floats, in its chunk's plane buffer (chunk c: buffer c % nbuf)
    std::vector<int2> work_a, work_b;   // (galaxy, row block) and (galaxy, tile), chunk by chunk
    std::vector<int> chunk_a, chunk_b;  // work ranges of the chunks (n_chunks + 1 entries)
    std::vector<int> chunk_r;           // PSF radius of each chunk's galaxies
    std::vector<float> chunk_sig;       // and their PSF width (sigma, pixels)
    int nbuf = 1;                       // plane buffers (2: a chunk's PSF stage beside the next line stage)
    size_t smem_a = 0;
    size_t o_mcs = 0, o_tab = 0, o_pl = 0, o_part = 0, o_arr = 0, o_taboff = 0, o_ra = 0, o_tbase = 0, o_ploff = 0,
           o_wa = 0, o_wb = 0, total = 0;
};
// Plans a batch of geometries (plan->ok false when one is not served); with
// `active`, only the galaxies with active[m] != 0 get work (the offsets and
// index arrays keep the batch's galaxy numbering, and the plan needs no more
// workspace than the full one).
void tsplit_ragged_plan(const std::vector<Geom> &geo, TsRaggedPlan *plan, const std::vector<char> *active = nullptr);
// Copies the plan's index arrays into the workspace (asynchronous on st;
// the host vectors may be released afterwards).
gbk_status tsplit_ragged_upload(const TsRaggedPlan &plan, char *ws, cudaStream_t st);
// J^T J, J^T v, sum r^2 of galaxy m's model params[m] against obs_list[m]
// (geometry d_geo[m]); galaxies with skip[m] != 0 are left alone.
struct TsplitRaggedCall {
    const Geom *d_geo;        // device [n]
    const double *params;     // device [n][GBK_NPAR]
    const gbk_obs *obs_list;  // device [n]
    const int32_t *skip;      // device [n] or null
    int np;
    int free_idx[GBK_NPAR];
    double *jtj, *jtv, *chi2; // device outputs (each may be null)
};
gbk_status launch_tsplit_ragged(const TsRaggedPlan &plan, const TsplitRaggedCall &call, char *ws, cudaStream_t st);

}  // namespace gbk
