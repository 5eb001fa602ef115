// k_lm.h -- device state and launchers of batched Levenberg-Marquardt.
#pragma once

#include "gbk_internal.cuh"

namespace gbk {

// All pointers are device memory (workspace or caller arrays).
struct LmArgs {
    int n_gal;
    int np;                  // free parameters
    int free_idx[GBK_NPAR];  // their indices in the parameter vector
    double fd_step[GBK_NPAR];
    int m;                   // models per galaxy in the Jacobian batch (1 + np or 1 + 2 np)
    int central;             // central differences
    int np_pix;              // nx * ny
    int max_iter;
    double ftol, xtol;
    const double *lo, *hi;   // [n_gal][NPAR]
    double *params;          // [n_gal][NPAR] current point (caller array)
    double *pbatch;          // [n_gal * m][NPAR]
    float *resid;            // [n_gal * m][2][np_pix]
    double *chi2_batch;      // [n_gal * m]
    double *hstep;           // [n_gal][np] signed step (2h for central)
    double *jtj, *jtr;       // [n_gal][np][np], [n_gal][np]
    double *ptrial;          // [n_gal][NPAR]
    double *chi2_trial;      // [n_gal]
    double *chi2_cur;        // [n_gal] chi2 at params
    double *chi2_best;       // [n_gal] chi2 at the returned parameters
    double *lambda, *dnorm, *pnorm;  // [n_gal]
    double *pred;            // [n_gal] chi2 decrease the linearised model predicts for the trial step
    double *nu;              // [n_gal] factor of lambda's next rise on a rejection
    int32_t *iters, *status, *done;  // [n_gal]
    int32_t *jskip;          // [n_gal] non-zero: the Jacobian stage leaves the galaxy
                             // alone (finished, or its last step was rejected, so
                             // J^T J and J^T r at params are still in place)
    int32_t *n_active;       // [1] galaxies still running after the last accept
    const int64_t *pix_off;  // ragged batches: [n_gal + 1] pixel offsets (galaxy gal's
                             // residuals start at 2 m pix_off[gal]); null: np_pix each
};

// Tail compaction of a batch of one geometry: the running galaxies (current
// slots live[0 .. n_live), increasing) move to slots 0 .. n_live of the next
// buffers with the state that outlives an iteration; everything else is
// recomputed (their Jacobian too: the kernels are deterministic, so it is
// the one they hold).
struct LmCompactArgs {
    int n_live;
    const int32_t *live;                  // [n_live]
    const int32_t *map;                   // [n_cur] slot -> caller index, or null (identity)
    const double *params, *lo, *hi;       // current [n_cur][NPAR]
    const gbk_obs *obs;                   // current [n_cur]
    const double *lambda, *nu, *chi2_cur; // current [n_cur]
    const int32_t *iters;                 // current [n_cur]
    double *params_n, *lo_n, *hi_n;       // next [n_live][NPAR]
    gbk_obs *obs_n;                       // next [n_live]
    int32_t *map_n;                       // next [n_live]
    double *lambda_n, *nu_n, *chi2_cur_n; // next [n_live] (copied back by the caller)
    int32_t *iters_n;                     // next [n_live]
};

// Writes the results of slots 0 .. n (finished or not) to the caller's
// arrays at map[slot]; params too when params_out is not null.
struct LmScatterArgs {
    int n;
    const int32_t *map;
    const double *params, *chi2_best;
    const int32_t *iters, *status;
    double *params_out, *chi2_out;
    int32_t *iters_out, *status_out;
};

void lm_launch_compact(const LmCompactArgs &c, cudaStream_t st);
void lm_launch_scatter(const LmScatterArgs &s, cudaStream_t st);
void lm_launch_init(const LmArgs &a, double lambda0, cudaStream_t st);
void lm_launch_build_fd(const LmArgs &a, cudaStream_t st);
void lm_launch_normal_fd(const LmArgs &a, cudaStream_t st);
void lm_launch_solve(const LmArgs &a, cudaStream_t st);
void lm_launch_accept(const LmArgs &a, cudaStream_t st);

}  // namespace gbk
