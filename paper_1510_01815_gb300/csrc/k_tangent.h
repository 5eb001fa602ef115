// k_tangent.h -- launcher of the analytic Jacobian kernel.
#pragma once

#include "gbk_internal.cuh"

namespace gbk {

constexpr int kTangentThreads = 256;

struct TangentArgs {
    Geom g;                  // u must be 1
    int n_models;
    const double *params;    // [n_models][GBK_NPAR]
    gbk_obs obs;             // single galaxy (used when obs_list is null)
    const gbk_obs *obs_list; // optional, one per galaxy
    int models_per_gal;      // model m belongs to galaxy m / models_per_gal (0: galaxy 0)
    const int32_t *skip;     // optional per-galaxy skip flags
    int np;                  // free parameters
    int free_idx[GBK_NPAR];  // their indices
    const float *cot;        // optional cotangent maps [n_models][2][ny][nx] (default: the residuals)
    double *jtj;             // [n_models][np][np] or null
    double *jtv;             // [n_models][np] or null: J^T (cot or residuals)
    double *chi2;            // [n_models] or null: sum of squared residuals
    float *jac;              // [n_models][GBK_NPAR][2][ny][nx] or null
    int cs, band;            // cluster size, most extended rows per CTA
    int direct;              // 1: the y pass reads halo rows in the neighbours' shared memory
    // Ragged batches (geoms != null): cluster w serves galaxy order[w] (or w)
    // with geometry geoms[gal], one model per galaxy; jac must be null.
    const Geom *geoms;
    const int32_t *order;
    size_t smem;             // dynamic shared memory (ragged: the largest need)
};

size_t tangent_smem_bytes_host(const Geom &g, int band, int threads, int direct, bool narrow);
// Launch shape for the eight-derivative (narrow) or the ten-derivative build.
bool tangent_config(const Geom &g, int *cs, int *band, int *direct, bool narrow);
// Whether a launch carries only x0 .. sigma0 (I0 and h fixed, J not written).
bool tangent_narrow(const TangentArgs &a);
// Launch shape of a galaxy for the narrow build as one key: cluster size +
// 32 * direct (0: no shape fits).
int tangent_cluster_for(const Geom &g);
inline int tangent_key_cs(int key) { return key & 31; }
inline int tangent_key_direct(int key) { return key >> 5; }
gbk_status launch_tangent(const TangentArgs &args, cudaStream_t stream);
// Velocity-field models (k_vfield.cu); launch_tangent dispatches to it.
gbk_status launch_vfield_tangent(const TangentArgs &args, cudaStream_t stream);

}  // namespace gbk
