// k_fused.h -- launcher of the fused forward-model kernel (host side).
#pragma once

#include "gbk_internal.cuh"

namespace gbk {

constexpr int kFusedThreads = 512;  // default block size (variants: 512, 384, 256)
// Opt-in shared memory per block is 227 KB; 2 KB are left for the static
// shared memory of the kernel.
constexpr int kFusedMaxSmem = 225 * 1024;
constexpr int kFusedMaxCluster = 16;

struct FusedArgs {
    Geom g;                 // u must be 1
    int n_models;
    const double *params;   // [n_models][GBK_NPAR]
    gbk_obs obs;            // device pointers; used when chi2 or resid is set
    const gbk_obs *obs_list;  // optional device array, one entry per galaxy (overrides obs)
    int models_per_gal;       // with obs_list / skip: model m belongs to galaxy m / models_per_gal
    const int32_t *skip;      // optional device flags per galaxy: non-zero = leave its models alone
    float *maps;            // [n_models][3][ny][nx] or null
    double *chi2;           // [n_models] or null
    float *resid;           // [n_models][2][ny][nx] or null
    int cs;                 // CTAs (cluster size) per model, 1..16
    int band;               // most extended rows of any CTA = ceil(ey / cs)
    int threads;            // block size: 512, 384 or 256
    int persistent;         // 1: one resident wave of clusters loops over the models;
                            // 0: one cluster per model
    // Ragged batches (geoms != null): galaxy gal has geometry geoms[gal] and
    // models gal * models_per_gal + s, s < models_per_gal; its maps and
    // residuals start at pixel offset pix_off[gal] * models_per_gal (times 3
    // and 2) and model s of it follows at s * nx * ny.  n_models counts the
    // models of the galaxies order[0 .. n_models / models_per_gal).
    const Geom *geoms;      // device [n_gal]
    const int64_t *pix_off; // device [n_gal]
    const int32_t *order;   // device list of the galaxies this launch serves (null: 0, 1, ...)
    size_t smem;            // dynamic shared memory (ragged: the largest geometry's need)
    // Persistent launches: optional device counters, zero at launch, that
    // hand the models to the clusters in the order they become free
    // (null: cluster c takes models c, c + clusters, ...).  work[0] serves
    // the first n_models - n_solo models to whole clusters; work[1] then
    // serves the last n_solo models (ragged launches; their galaxies must
    // fit one CTA) to single CTAs.
    int *work;
    int n_solo;
};

// Launch configuration of the fused kernel (see tune.cu).
struct FusedConfig {
    int cs;          // CTAs (cluster size) per model
    int band;        // ceil(ey / cs)
    int threads;     // block size
    int persistent;  // grid shape (see FusedArgs)
};

size_t fused_smem_bytes_host(const Geom &g, int band);
bool fused_config_ragged(const Geom *geoms, int n, int cs, int threads, size_t *smem);
bool fused_config(const Geom &g, FusedConfig *cfg);
bool fused_config_valid(const Geom &g, int cs, int threads, int persistent, FusedConfig *cfg);
gbk_status launch_fused(const FusedArgs &args, cudaStream_t stream);
// Velocity-field models (k_vfield.cu); launch_fused dispatches to it.
gbk_status launch_vfield(const FusedArgs &args, cudaStream_t stream);

}  // namespace gbk
