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

void lm_launch_init(const LmArgs &a, double lambda0, cudaStream_t st);
void lm_launch_build_fd(const LmArgs &a, cudaStream_t st);
void lm_launch_normal_fd(const LmArgs &a, cudaStream_t st);
void lm_launch_solve(const LmArgs &a, cudaStream_t st);
void lm_launch_accept(const LmArgs &a, cudaStream_t st);

}  // namespace gbk
