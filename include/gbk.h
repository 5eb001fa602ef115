/*
 * gbk.h -- C ABI of the GB300 disc-galaxy kinematic-model library (libgbk.so).
 *
 * The library evaluates the intensity-cube forward model of Bekiaris et al.
 * 2015 (arXiv:1510.01815), Sec. 2: for each parameter set it builds the
 * (x, y, v) cube of a thin exponential disc with an arctan rotation curve and
 * a constant intrinsic dispersion (Sec. 2.1, Eqs. 1-8), convolves it with a
 * Gaussian PSF x LSF kernel (Eq. 9, Sec. 2.2.3), down-samples it (Sec. 2.2.4),
 * takes the moment-0/1/2 maps (Sec. 2.2.5) and reduces the masked chi-squared
 * of Eq. 11 against observed velocity and dispersion maps (Sec. 2.2.6).
 *
 * Conventions shared by every entry point
 *  - All arithmetic runs in the library's CUDA kernels on the device of the
 *    calling thread.  Cubes, maps and residuals are FP32; parameters and
 *    chi-squared values are FP64.
 *  - Every buffer is owned by the caller.  Pointers documented as "device"
 *    must be device (or managed) memory of the current device; "host" means
 *    ordinary host memory.  The library never allocates device memory: entry
 *    points that need scratch take a caller-provided workspace whose size is
 *    given by the matching *_workspace_bytes() query.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Entry
 *    points marked "asynchronous" only enqueue work on it.
 *  - Every function returns a gbk_status.  Arguments are validated on the
 *    host before anything is launched; on error nothing is launched and
 *    gbk_last_error() returns a message for the calling thread.  No function
 *    aborts, traps or prints.
 *  - Layouts are row-major with x fastest: a cube is [model][z][y][x], a map
 *    set is [model][3][y][x] = (m0, m1, m2), residuals are
 *    [model][2][y][x] = (velocity, dispersion).
 *  - Parameter vectors are GBK_NPAR doubles in the order of the enum below:
 *    centre (pixels), position angle and inclination (degrees), systemic and
 *    asymptotic velocities (km/s), turn-over radius (pixels), intrinsic
 *    dispersion (km/s), central surface brightness and exponential scale
 *    length (pixels).  Pixel centres sit at integer coordinates 0..N-1;
 *    channel k has velocity vc + (k - (nz-1)/2) dv.
 */
#ifndef GBK_API_H_INCLUDED
#define GBK_API_H_INCLUDED

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define GBK_API __attribute__((visibility("default")))
#else
#define GBK_API
#endif

typedef int32_t gbk_status;

#define GBK_OK          0
#define GBK_EINVAL      1  /* an argument failed validation                    */
#define GBK_ECUDA       2  /* a CUDA runtime call failed (message has details) */
#define GBK_EWORKSPACE  3  /* the workspace is missing or too small            */
#define GBK_EUNSUPPORTED 4 /* a valid request the library does not serve       */

/* Parameter order (Sec. 2.1; Vmax is the paper's V_t, h its r_0). */
enum {
    GBK_X0 = 0, GBK_Y0, GBK_PA, GBK_INCL, GBK_VSYS, GBK_VMAX, GBK_RT, GBK_SIG0,
    GBK_I0, GBK_H, GBK_NPAR
};

/* Observation geometry (host struct, passed by pointer).
 *  nx, ny, nz    data cube size: spaxels along x, y and velocity channels (>= 1)
 *  upsample      model upsampling factor u >= 1 (Sec. 2.2.2, Sec. 2.2.4)
 *  dv            channel width in km/s (> 0)
 *  vc            velocity of the band centre in km/s
 *  psf_fwhm      PSF FWHM in pixels (>= 0; 0 = no spatial convolution)
 *  lsf_fwhm      LSF FWHM in km/s (>= 0)
 *  lsf_mode      0: the LSF is a convolution along velocity (Eq. 9 as
 *                written); 1: the LSF is folded into the line width in
 *                quadrature and only the PSF is convolved
 *  halo_sigmas   kernel truncation radius in standard deviations (> 0,
 *                usually 4): R = ceil(halo_sigmas * sigma) on each axis.
 * The Gaussian kernels are sampled at integer offsets |j| <= R and
 * normalised to unit sum per axis; the model is evaluated on the data grid
 * extended by R on every side and the "valid" linear convolution is kept. */
typedef struct gbk_geom {
    int32_t nx, ny, nz;
    int32_t upsample;
    double dv;
    double vc;
    double psf_fwhm;
    double lsf_fwhm;
    int32_t lsf_mode;
    int32_t model;      /* GBK_MODEL_*: 0 (the default) is the intensity cube */
    double halo_sigmas;
} gbk_geom;

/* Modelling strategies (Sec. 2.2.1).  The intensity cube (Sec. 2.2.2-2.2.5,
 * arctan rotation curve, Eq. 6) is the default.  The velocity-field models
 * evaluate Eq. 8 at every data pixel directly -- no cube, no PSF or LSF --
 * with the arctan curve or the Epinat curve (Eq. 7),
 *   Vrot(r) = V_t (r/r_t)^g / (1 + (r/r_t)^a),
 * whose slopes a and g occupy parameter slots GBK_EPI_A = GBK_I0 and
 * GBK_EPI_G = GBK_H (a velocity field has no intensity model).  Their maps
 * are m0 = 1 (every pixel valid), m1 = the field, m2 = sigma0 (the constant
 * dispersion model, Sec. 2.1.4); nz, dv, vc, the PSF and the LSF are not
 * used, upsample must be 1; at r = 0 the field is Vsys.  Parameter domain:
 * 0 <= i < 90, r_t > 0, sigma0 >= 0, the used parameters finite.  Served by
 * the fused entry points (gbk_eval_cubes maps, gbk_chi2, gbk_fit_lm with
 * finite differences or the analytic Jacobian, gbk_jacobian, gbk_grid,
 * gbk_nested_sample); the staged path, cubes and survey batches answer
 * GBK_EUNSUPPORTED.  The analytic Jacobian of a field is zero at r = 0 for
 * the radius-dependent terms (the cusp of r), as for the cube. */
#define GBK_MODEL_CUBE           0
#define GBK_MODEL_VFIELD_ARCTAN  1
#define GBK_MODEL_VFIELD_EPINAT  2
#define GBK_EPI_A GBK_I0
#define GBK_EPI_G GBK_H

/* Observed maps of one galaxy, each ny*nx, device memory.
 *  v_obs, s_obs  observed velocity and dispersion maps (km/s)
 *  w_v, w_s      weights 1/E_v and sqrt(W)/E_s (Eq. 11 with W folded in)
 *  mask          1 = use the spaxel, 0 = leave it out */
typedef struct gbk_obs {
    const float *v_obs;
    const float *s_obs;
    const float *w_v;
    const float *w_s;
    const uint8_t *mask;
} gbk_obs;

/* Evaluation paths (the `flags` argument of gbk_chi2).  All compute the
 * same maps and chi-squared (Sec. 2.2.2-2.2.6); they differ in where the
 * intermediate values live.
 *  GBK_PATH_FUSED   one kernel, a thread-block cluster per model; the cube
 *                   never leaves the SM; needs no workspace.
 *  GBK_PATH_STAGED  model cube -> separable convolution -> moments, each
 *                   stage through HBM (the paper's pipeline).
 *  GBK_PATH_SPLIT   two kernels: each extended spaxel's line folded into a
 *                   moment triplet (16 bytes, in the workspace, sized to stay
 *                   in L2), then the PSF passes, moments and chi-squared in
 *                   tiles; the cube is never formed.  Cube model, u = 1, PSF
 *                   radius <= 8 px.
 *  GBK_PATH_AUTO    the split path when it serves the geometry and the
 *                   workspace holds what it needs, else the fused path when
 *                   it serves the geometry, else the staged path. */
#define GBK_PATH_AUTO    0u
#define GBK_PATH_FUSED   1u
#define GBK_PATH_STAGED  2u
#define GBK_PATH_SPLIT   3u

/* Bytes of workspace gbk_eval_cubes / gbk_chi2 need for n_models models on
 * the given path (0 when the path needs none; GBK_PATH_AUTO: the bytes of the
 * path it prefers for this geometry).  Host function; returns 0 and sets the
 * last error on invalid arguments. */
GBK_API size_t gbk_workspace_bytes(const gbk_geom *g, int32_t n_models, uint32_t flags);

/* Forward model, Sec. 2.2.2-2.2.5.  Asynchronous.
 *  g         geometry (host)
 *  n_models  number of parameter sets (>= 0; 0 is a no-op)
 *  params    device, [n_models][GBK_NPAR] FP64
 *  cubes     device, [n_models][nz][ny][nx] FP32, or NULL.  When non-NULL the
 *            staged path runs and the convolved, down-sampled cube is written.
 *  maps      device, [n_models][3][ny][nx] FP32 (m0, m1, m2), or NULL.
 *            m0 = sum over channels, m1 = intensity-weighted mean velocity,
 *            m2 = intensity-weighted standard deviation.  A spectrum with
 *            m0 <= 1e-20 * I0 is invalid and gets (0, Vsys, 0).
 *  workspace device scratch (may be NULL): with cubes, at least
 *            gbk_workspace_bytes(g, n_models, GBK_PATH_STAGED) bytes; without,
 *            the maps come from the split path when the workspace holds
 *            gbk_workspace_bytes(g, n_models, GBK_PATH_SPLIT) bytes, else
 *            from the fused path, else (geometries neither serves) from the
 *            staged path.
 * Validation: sizes >= 1, dv > 0, psf/lsf >= 0, halo_sigmas > 0, and for
 * every model 0 <= i < 90 deg, r_t > 0, sigma0 > 0, I0 > 0, h > 0 -- the
 * parameter checks run on the device and invalid models get NaN maps and
 * chi-squared (the host cannot read device parameters without a sync). */
GBK_API gbk_status gbk_eval_cubes(const gbk_geom *g, int32_t n_models, const double *params,
                          float *cubes, float *maps, void *workspace, size_t ws_bytes,
                          void *stream);

/* Masked chi-squared of Eq. 11 for n_models parameter sets against one
 * galaxy's observed maps.  Asynchronous.
 *  obs     host struct of device pointers (see gbk_obs)
 *  chi2    device, [n_models] FP64 (required)
 *  resid   device, [n_models][2][ny][nx] FP32 weighted residuals
 *          w_v (m1 - v_obs) and w_s (m2 - s_obs), 0 where masked or
 *          invalid; or NULL
 *  flags   GBK_PATH_AUTO, GBK_PATH_FUSED, GBK_PATH_STAGED or GBK_PATH_SPLIT
 *  workspace, ws_bytes  device scratch for the path (see
 *          gbk_workspace_bytes); NULL / 0 when the path needs none.
 * The reduction order is fixed for each path, so results are bitwise
 * reproducible. */
GBK_API gbk_status gbk_chi2(const gbk_geom *g, int32_t n_models, const double *params,
                    const gbk_obs *obs, double *chi2, float *resid, uint32_t flags,
                    void *workspace, size_t ws_bytes, void *stream);

/* gbk_chi2 on the split path with every array in HOST memory (Eq. 11; the
 * call a user with data on the host makes): the parameters are copied on
 * `stream`, the observed maps on the split evaluator's second stream so that
 * their copy overlaps the first line stage (which does not read them), and
 * chi2 comes back on `stream`.  Asynchronous: host buffers must stay valid
 * until the stream has passed the call; pinned buffers make the copies
 * asynchronous, pageable ones are copied synchronously by the runtime.
 *  params     host [n_models][GBK_NPAR] FP64
 *  obs        host struct of HOST pointers to the five maps [ny][nx]
 *  chi2       host [n_models] FP64, written when the stream reaches it
 *  workspace  device scratch of gbk_chi2_host_workspace_bytes(g, n_models)
 *             bytes (the device copies and the split evaluator's buffer)
 * GBK_EUNSUPPORTED for geometries the split path does not serve (cube model,
 * u = 1, PSF radius <= 8). */
GBK_API size_t gbk_chi2_host_workspace_bytes(const gbk_geom *g, int32_t n_models);
GBK_API gbk_status gbk_chi2_host(const gbk_geom *g, int32_t n_models, const double *params, const gbk_obs *obs,
                                 double *chi2, void *workspace, size_t ws_bytes, void *stream);

/* gbk_chi2 on the staged path for callers that cannot allocate device
 * memory (no counterpart in the paper).  A host application whose device
 * memory is owned and pre-planned by another framework, or a real-time
 * caller that forbids allocation after start-up, cannot hand the staged
 * path a workspace.  This entry point needs none: its scratch is a 32 MiB
 * array built into the library (every GPU that loads the library holds it
 * until the process exits).  Arguments, outputs and results are those of
 * gbk_chi2 with flags = GBK_PATH_STAGED.  Asynchronous.
 *  - Batches needing more than 32 MiB of scratch (see gbk_workspace_bytes
 *    with GBK_PATH_STAGED) are rejected with GBK_EWORKSPACE before anything
 *    is launched.
 *  - The first call on a device looks up the array's device address; make
 *    it before any stream capture (a first call on a capturing stream is
 *    refused with GBK_EUNSUPPORTED).  A device reset (cudaDeviceReset, or a
 *    primary context destroyed and created again) invalidates the address
 *    the library keeps, so this entry point must not be used after one.
 *  - All calls share the array: calls that overlap on the GPU (other
 *    streams, other host threads) race and must be serialised by the
 *    caller.  Nothing in the array has to start at zero.
 *  - Allocates nothing (no cudaMalloc, cudaFree or allocating library
 *    call). */
GBK_API gbk_status gbk_chi2_noalloc(const gbk_geom *g, int32_t n_models, const double *params,
                                    const gbk_obs *obs, double *chi2, float *resid, void *stream);

/* gbk_chi2 on the split path (GBK_PATH_SPLIT), timed per stage with CUDA
 * events recorded on `stream` around every launch: stage_ms (host [3])
 * receives the milliseconds of the set-up kernel, of the line stage (the
 * Gaussian lines folded into moment triplets and the PSF along x,
 * Sec. 2.2.2-2.2.3) and of the PSF-along-y stage with the moments and chi2
 * (Sec. 2.2.3-2.2.6), each summed over the model chunks; launches (host, or
 * NULL) the number of kernel launches.  Workspace as for gbk_chi2 on the split
 * path; at most 31 chunks; synchronises `stream`. */
GBK_API gbk_status gbk_split_stage_times(const gbk_geom *g, int32_t n_models, const double *params,
                                         const gbk_obs *obs, double *chi2, void *workspace, size_t ws_bytes,
                                         float *stage_ms, int32_t *launches, void *stream);

/* gbk_chi2 on the staged path (GBK_PATH_STAGED), timed per stage with CUDA
 * events on `stream` -- the per-step timings of the paper's GPU pipeline
 * (Sec. 5): stage_ms (host [4]) receives the milliseconds of the model cube
 * (a1-a2), the PSF x LSF convolution (a3), the down-sampling (a4; 0 at
 * u = 1) and the moments with the masked chi2 (a5-a6).  Workspace as for
 * gbk_chi2 on the staged path; synchronises `stream`. */
GBK_API gbk_status gbk_chi2_stage_times(const gbk_geom *g, int32_t n_models, const double *params, const gbk_obs *obs,
                                        double *chi2, void *workspace, size_t ws_bytes, float *stage_ms,
                                        void *stream);

/* Eq. 11 alone, from caller-supplied FP32 maps [n_models][3][ny][nx]
 * (device).  Spaxels with m0 <= 0 count as invalid.  Asynchronous; needs
 * no workspace. */
GBK_API gbk_status gbk_chi2_from_maps(int32_t nx, int32_t ny, int32_t n_models, const float *maps,
                              const gbk_obs *obs, double *chi2, float *resid, void *stream);

/* Analytic Jacobian of the weighted residual maps of gbk_chi2 (forward-mode
 * derivatives through Eqs. 1-11; no counterpart code in the paper, which
 * used finite differences).  Asynchronous.  For each model:
 *   J[k] = d(resid)/d(param k) for all GBK_NPAR parameters, written to jac
 *          (device, [n_models][GBK_NPAR][2][ny][nx] FP32) when jac != NULL;
 *   jtj  = J_f^T J_f, device [n_models][nf][nf] FP64, and
 *   jtv  = J_f^T v, device [n_models][nf] FP64, where J_f keeps the nf
 *          parameters selected by free_mask (in parameter order) and v is
 *          `cot` (device [n_models][2][ny][nx]) or, when cot == NULL, the
 *          residuals themselves (then jtv is the gradient of chi2 / 2);
 *   chi2 = sum of squared residuals, device [n_models] (may be NULL).
 * Masked and invalid spaxels have zero rows.  At the disc centre (r = 0)
 * the brightness derivative with respect to the centre and the angles uses
 * the one-sided value 0.  A model is split over a thread-block cluster of
 * up to 16 CTAs by rows; the y pass reads its halo rows from copies in each
 * CTA's shared memory or, where those do not fit (wide maps, e.g. above
 * about 64 x 64 spaxels at a 4-pixel PSF), in the neighbouring CTAs' shared
 * memory.  EUNSUPPORTED where even that does not fit (about 100 x 100
 * spaxels at a 4-pixel PSF). */
GBK_API gbk_status gbk_jacobian(const gbk_geom *g, int32_t n_models, const double *params,
                                const gbk_obs *obs, uint32_t free_mask, const float *cot, double *jtj,
                                double *jtv, double *chi2, float *jac, void *stream);

/* The same analytic Jacobian reductions as gbk_jacobian (J^T J, J^T v and
 * the sum of squared residuals; no J maps), computed in the split
 * evaluator's shape: a line stage forms every extended spaxel's value and
 * derivative moment triplets and filters them along x, a PSF stage filters
 * them along y and applies the quotient rule of the moments and the
 * reductions, the two meeting in a caller workspace sized to stay in L2.
 * Served: the cube model at u = 1, PSF radius <= 8 px, free parameters
 * among x0 .. sigma0 (I0 and h fixed); otherwise GBK_EUNSUPPORTED.
 * Arguments as gbk_jacobian (without jac); workspace device memory of
 * gbk_jacobian_workspace_bytes(g, n_models, free_mask) bytes (GBK_EWORKSPACE
 * if smaller).  Asynchronous; the reductions are in a fixed order. */
GBK_API size_t gbk_jacobian_workspace_bytes(const gbk_geom *g, int32_t n_models, uint32_t free_mask);
GBK_API gbk_status gbk_jacobian_ws(const gbk_geom *g, int32_t n_models, const double *params,
                                   const gbk_obs *obs, uint32_t free_mask, const float *cot, double *jtj,
                                   double *jtv, double *chi2, void *workspace, size_t ws_bytes, void *stream);

/* ------------------------------------------------------------------------
 * Levenberg-Marquardt fitting (Sec. 2.3.1).  The paper drives the C mpfit
 * library on the CPU with a forward-difference Jacobian of step ~0.1 in every
 * parameter, box constraints, one galaxy at a time; the model evaluations run
 * on the GPU.  Here the damped normal equations
 *     (J^T J + lambda diag(J^T J)) delta = -J^T r
 * are formed and solved in FP64; parameters are clipped to [lo, hi]; a step
 * is accepted when it does not raise chi2.  lambda follows the gain ratio
 * rho of the actual to the predicted chi2 decrease (-2 s.J^T r - s.J^T J s
 * for the clipped step s; mpfit steers its step by the same ratio): on
 * acceptance lambda *= max(1/10, 1 - (2 rho - 1)^3) (floor 1e-12) and
 * nu = 2, on rejection lambda *= nu and nu *= 2 (Nielsen's rule).  After a
 * rejected step the Jacobian at the unchanged point is reused.  A galaxy
 * stops when an accepted step lowers chi2 by less than ftol (relative),
 * when |delta| <= xtol (|p| + xtol), when lambda exceeds 1e12, or after
 * max_iter iterations (an iteration: one damped solve and one trial
 * evaluation, plus the Jacobian when the last step was accepted).
 * ------------------------------------------------------------------------ */
#define GBK_JAC_FD_FORWARD  0  /* (r(p + h e_j) - r(p)) / h, h = fd_step[j]        */
#define GBK_JAC_FD_CENTRAL  1  /* (r(p + h e_j) - r(p - h e_j)) / 2h               */
#define GBK_JAC_TANGENT     2  /* analytic tangent of the whole forward model      */
                               /* (gbk_jacobian's kernel; 1 evaluation-like pass) */

#define GBK_LM_BATCHED  0  /* all galaxies advance together; everything on the device */
#define GBK_LM_PLAIN    1  /* one galaxy at a time; normal equations and the solve on  */
                           /* the host in FP64 (the paper's CPU-optimiser arrangement) */

/* Per-galaxy fit status (status_out). */
#define GBK_FIT_RUNNING    0
#define GBK_FIT_FTOL       1  /* relative chi2 decrease below ftol              */
#define GBK_FIT_XTOL       2  /* step below xtol                                */
#define GBK_FIT_MAXITER    3  /* max_iter reached                               */
#define GBK_FIT_LAMBDA     4  /* lambda above 1e12: no downhill step found      */
#define GBK_FIT_NONFINITE  5  /* chi2 at the current parameters is not finite   */

typedef struct gbk_lm_opts {
    int32_t max_iter;          /* iterations (each: solve, trial; + Jacobian)     */
    int32_t jacobian;          /* GBK_JAC_*                                      */
    int32_t mode;              /* GBK_LM_*                                       */
    uint32_t free_mask;        /* bit k set: parameter k is fitted (1..10 bits)  */
    double ftol, xtol;         /* stopping tolerances (e.g. 1e-10)               */
    double lambda0;            /* initial damping (e.g. 1e-3)                    */
    double fd_step[GBK_NPAR];  /* absolute finite-difference steps (e.g. 0.1)    */
    int32_t path;              /* batched mode, one geometry: GBK_PATH_AUTO (0)  */
                               /* = the split evaluator and Jacobian where they  */
                               /* serve the geometry, GBK_PATH_SPLIT = required, */
                               /* GBK_PATH_FUSED = the cluster kernels           */
    int32_t reserved;          /* 0                                              */
} gbk_lm_opts;

/* Workspace bytes gbk_fit_lm needs (0 and last error set on bad input). */
GBK_API size_t gbk_fit_lm_workspace_bytes(const gbk_geom *g, int32_t n_gal, const gbk_lm_opts *opts);

/* Fits n_gal galaxies that share one geometry.  Synchronises `stream`.
 *  obs        device array [n_gal] of gbk_obs (each a galaxy's maps)
 *  lo, hi     device [n_gal][GBK_NPAR] box constraints
 *  params     device [n_gal][GBK_NPAR]: start on entry, fit on return
 *             (fixed parameters are left as given)
 *  chi2_out   device [n_gal] chi2 at the returned parameters
 *  iters_out  device [n_gal] iterations used
 *  status_out device [n_gal] GBK_FIT_* codes
 * The batched mode captures one iteration in a CUDA graph and replays it,
 * reading the number of running galaxies back every 8 iterations; finished
 * galaxies are skipped by the kernels. */
GBK_API gbk_status gbk_fit_lm(const gbk_geom *g, int32_t n_gal, const gbk_obs *obs, const double *lo,
                              const double *hi, double *params, const gbk_lm_opts *opts, double *chi2_out,
                              int32_t *iters_out, int32_t *status_out, void *workspace, size_t ws_bytes,
                              void *stream);

/* LM from a learned start with the plain fit as its fallback (how the CNN
 * seed below is used): every galaxy is fitted from `params` (the seed); a
 * galaxy whose seeded fit did not converge (status other than GBK_FIT_FTOL
 * or GBK_FIT_XTOL) or ended with chi2 above chi2_accept[g] is fitted again,
 * with the same options, from fallback_start[g] (the method's own start,
 * e.g. gbk_initial_guess), and of its two fits the one with the lower chi2
 * is returned.  Arguments as gbk_fit_lm, plus
 *  fallback_start device [n_gal][GBK_NPAR]
 *  chi2_accept    device [n_gal], or NULL (then only unconverged fits fall
 *                 back); e.g. 1.5 x the number of unmasked residuals
 *  used_fallback  device [n_gal] int32: 0 the seeded fit was not redone,
 *                 1 the fallback fit is returned, 2 it ran but the seeded
 *                 fit had the lower chi2 (iters_out and status_out belong to
 *                 the fit returned)
 *  workspace      gbk_fit_lm_fallback_workspace_bytes(g, n_gal, opts)
 * Synchronises `stream`; both passes run batched on the device, the
 * selection of the galaxies to refit on the host. */
GBK_API size_t gbk_fit_lm_fallback_workspace_bytes(const gbk_geom *g, int32_t n_gal, const gbk_lm_opts *opts);
GBK_API gbk_status gbk_fit_lm_fallback(const gbk_geom *g, int32_t n_gal, const gbk_obs *obs, const double *lo,
                                       const double *hi, double *params, const double *fallback_start,
                                       const double *chi2_accept, const gbk_lm_opts *opts, double *chi2_out,
                                       int32_t *iters_out, int32_t *status_out, int32_t *used_fallback,
                                       void *workspace, size_t ws_bytes, void *stream);

/* ------------------------------------------------------------------------
 * Initial model parameter values (Sec. 2.1.9), measured on each galaxy's
 * maps -- the optimisers' starting point when no better one (e.g. the CNN
 * seed below) is at hand:
 *   x0, y0  intensity-weighted mean position of the continuum map (negative
 *           values count as 0; no light: the image centre);
 *   V_sys   mean velocity of the unmasked pixels within 2.5 pixels of that
 *           centre (none that close: of all unmasked pixels; none: 0);
 *   PA      the whole degree whose split of the velocity field into the
 *           halves x_e > 0 and x_e < 0 (Eqs. 1-2) maximises the difference
 *           of their mean velocities, pixels binned by whole degrees of
 *           polar angle about the centre (ties to the smaller PA);
 *   i       from the continuum's intensity-weighted second central moments:
 *           their eigenvalues less the PSF variance have the ratio cos^2 i
 *           (the paper uses a catalogue inclination); clipped to [5, 85];
 *   r_t     h for the cube model (the photometric scale length), the
 *           caller's value for velocity fields;
 *   V_t = 150 km/s, sigma0 = 30 km/s; a = g = 1 for the Epinat curve; every
 *   other slot (I0, h) is copied from `fixed`.
 *  continuum  device [n_gal][ny][nx] FP32 continuum (intensity) maps, or
 *             NULL: the unmasked pixels then weigh 1 each
 *  obs        device [n_gal] gbk_obs (v_obs and mask are read)
 *  fixed      device [n_gal][GBK_NPAR] (I0 and h, or r_t, as above)
 *  params_out device [n_gal][GBK_NPAR]
 * Asynchronous; FP64 arithmetic, deterministic; GBK_EINVAL on bad arguments
 * and for maps above 2^26 pixels. */
GBK_API gbk_status gbk_initial_guess(const gbk_geom *g, int32_t n_gal, const float *continuum, const gbk_obs *obs,
                                     const double *fixed, double *params_out, void *stream);

/* ------------------------------------------------------------------------
 * Survey batches: galaxies of different geometry (cube size, channel width,
 * LSF, PSF) evaluated or fitted together -- the survey-scale setting of
 * Sec. 1 and Sec. 5, with the model of Sec. 2.1-2.2 and the optimiser of
 * Sec. 2.3.1 unchanged per galaxy.
 *  geoms      host [n_gal]: geometry of each galaxy (upsample must be 1)
 *  params     device [n_gal][GBK_NPAR]
 *  obs        device [n_gal] gbk_obs, galaxy i's maps of geoms[i]'s size
 *  maps       device, packed: galaxy i's [3][ny_i][nx_i] (m0, m1, m2) at
 *             float offset 3 * P_i, P_i = sum_{j<i} nx_j * ny_j; or NULL
 *  chi2       device [n_gal] or NULL
 *  resid      device, packed: galaxy i's [2][ny_i][nx_i] at 2 * P_i; or NULL
 * Every galaxy gets exactly the values gbk_chi2 / gbk_eval_cubes give it
 * on its own (maps and residuals bit for bit; chi2 up to the order of its
 * FP64 reduction).  The workspace holds the geometry tables, uploaded from
 * the host on every call, and, for the fit, the batched LM state
 * (gbk_survey_workspace_bytes with opts NULL for evaluation, with the LM
 * options for fitting).  By default the evaluator serves the whole survey
 * in one persistent launch: a resident wave of thread-block clusters of one
 * size takes the models, costliest galaxies first, from a work counter in
 * the workspace as each cluster becomes free.  The alternative shape, one
 * launch per group of galaxies needing the same cluster size, and the
 * cluster and block sizes of the single launch are a survey tuning
 * (gbk_survey_autotune below).
 * gbk_survey_fit_lm is gbk_fit_lm per galaxy; the batched mode advances all
 * galaxies together in one CUDA graph (finite-difference or analytic tangent
 * Jacobian).  With the analytic Jacobian and opts->path GBK_PATH_AUTO (or
 * GBK_PATH_SPLIT, which requires it) every galaxy takes the ragged split
 * Jacobian below when every galaxy is a cube model at u = 1 with a PSF
 * radius <= 8; with
 * GBK_PATH_FUSED (or where the split one does not serve) the cluster
 * Jacobian kernel takes the galaxies whose halo rows fit a CTA's shared
 * memory and the others are fitted in the same call with finite
 * differences.  The survey Jacobians carry the eight derivatives x0 ..
 * sigma0, so a fit that frees I0 or h uses finite differences for every
 * galaxy.  The plain mode fits one galaxy after the other with the host
 * solve and finite differences.
 * ------------------------------------------------------------------------ */
GBK_API size_t gbk_survey_workspace_bytes(const gbk_geom *geoms, int32_t n_gal, const gbk_lm_opts *opts);
GBK_API gbk_status gbk_survey_eval(const gbk_geom *geoms, int32_t n_gal, const double *params, const gbk_obs *obs,
                                   float *maps, double *chi2, float *resid, void *workspace, size_t ws_bytes,
                                   void *stream);
GBK_API gbk_status gbk_survey_fit_lm(const gbk_geom *geoms, int32_t n_gal, const gbk_obs *obs, const double *lo,
                                     const double *hi, double *params, const gbk_lm_opts *opts, double *chi2_out,
                                     int32_t *iters_out, int32_t *status_out, void *workspace, size_t ws_bytes,
                                     void *stream);

/* The analytic Jacobian of a ragged batch in the split evaluator's shape
 * (the forward-mode derivatives of gbk_jacobian, Sec. 2.3.1): for galaxy i
 * with geometry geoms[i], parameters params[i] and maps obs[i], J^T J
 * [n_gal][nf][nf], J^T r [n_gal][nf] and sum r^2 [n_gal] (each may be
 * NULL) over the nf parameters of free_mask, which must lie among x0 ..
 * sigma0.  Per galaxy the arithmetic is that of gbk_jacobian_ws on that
 * galaxy alone; the stages run over work lists of (galaxy, row block) and
 * (galaxy, tile) in chunks whose planes stay in L2, galaxies grouped by PSF
 * radius.  GBK_EUNSUPPORTED unless every galaxy is a cube model at u = 1
 * with a PSF radius <= 8.  Workspace: gbk_survey_jacobian_workspace_bytes;
 * asynchronous. */
GBK_API size_t gbk_survey_jacobian_workspace_bytes(const gbk_geom *geoms, int32_t n_gal, uint32_t free_mask);
GBK_API gbk_status gbk_survey_jacobian(const gbk_geom *geoms, int32_t n_gal, const double *params,
                                       const gbk_obs *obs, uint32_t free_mask, double *jtj, double *jtv,
                                       double *chi2, void *workspace, size_t ws_bytes, void *stream);

/* ------------------------------------------------------------------------
 * Nested grids (Sec. 2.3.3): chi2 at every node of a regular grid, then a
 * new grid with the same number of nodes around the best node over a
 * smaller volume, for `levels` levels.  Level 0 spans [lo, hi] with nodes[k]
 * points per parameter (both ends included; nodes[k] == 1 keeps parameter k
 * at fixed[k]); level l+1 spans best +- one level-l step, clipped to
 * [lo, hi].  The linear node index is row-major in parameter order (the
 * first gridded parameter varies slowest); equal chi2 values go to the
 * lowest index, NaN counts as worse than any number.  Node values are
 * lo + i * ((hi - lo) / (n - 1)) in FP64.  Nodes are evaluated `chunk` at a
 * time with the fused path.  Synchronises `stream` once per level.
 *  obs, lo, hi, nodes, fixed   host (obs holds device pointers)
 *  best_params  host [GBK_NPAR]: the best node of the last level
 *  best_index   host [levels]:   best linear index per level
 *  best_chi2    host [levels]:   its chi2
 * ------------------------------------------------------------------------ */
GBK_API size_t gbk_grid_workspace_bytes(const gbk_geom *g, const int32_t *nodes, int32_t chunk);
GBK_API gbk_status gbk_grid(const gbk_geom *g, const gbk_obs *obs, const double *lo, const double *hi,
                            const int32_t *nodes, const double *fixed, int32_t levels, int32_t chunk,
                            double *best_params, int64_t *best_index, double *best_chi2, void *workspace,
                            size_t ws_bytes, void *stream);

/* ------------------------------------------------------------------------
 * Nested sampling (Sec. 2.3.2; the paper used MultiNest).  Vanilla nested
 * sampling with an ellipsoidal bound: n_live points from the uniform prior
 * over [lo, hi] (lo == hi fixes a parameter); each iteration draws `batch`
 * proposals uniformly inside the live points' bounding ellipsoid (volume
 * enlarged by 1.1 / efr) and inside the box, evaluates all their
 * likelihoods L = exp(-chi2/2) in one fused launch, and lets each proposal
 * in draw order replace the worst live point if it beats it (ln X -= 1 /
 * n_live per replacement).  Stops when ln(Z + L_max X) - ln Z < tol or after
 * max_iter iterations.  Random numbers: SplitMix64 seeded with `seed`,
 * Box-Muller normals.  Synchronises `stream` every iteration.
 *  obs, lo, hi (host; obs holds device pointers)
 *  post_mean, post_std  host [GBK_NPAR] posterior moments
 *  log_z, n_eval, n_iter host scalars
 * ------------------------------------------------------------------------ */
typedef struct gbk_ns_opts {
    int32_t n_live;    /* live points (e.g. 50 in the paper, 400 for the FP workload) */
    int32_t batch;     /* proposals per iteration                                     */
    double tol;        /* evidence tolerance (0.5)                                   */
    double efr;        /* target efficiency: bound volume x 1.1 / efr (1.0)          */
    uint64_t seed;
    int32_t max_iter;
    int32_t reserved;  /* must be 0 */
} gbk_ns_opts;

GBK_API size_t gbk_nested_sample_workspace_bytes(const gbk_geom *g, const gbk_ns_opts *opts);
GBK_API gbk_status gbk_nested_sample(const gbk_geom *g, const gbk_obs *obs, const double *lo, const double *hi,
                                     const gbk_ns_opts *opts, double *post_mean, double *post_std, double *log_z,
                                     int64_t *n_eval, int32_t *n_iter, void *workspace, size_t ws_bytes,
                                     void *stream);

/* The sampler's trajectory (Sec. 2.3.2), for checking it step by step
 * against another implementation of the same algorithm: the initial live
 * points, and for each of the first max_iter iterations every proposal in
 * draw order, its chi2 and the live point it replaced.  All arrays are host
 * memory owned by the caller; every pointer may be NULL to skip that record.
 *  max_iter    iterations to record (>= 0)
 *  n_iter      out: iterations recorded (<= max_iter)
 *  live0       [n_live][GBK_NPAR] initial live points
 *  live0_chi2  [n_live] their chi2 (NaN outside the parameter domain)
 *  n_props     [max_iter] proposals drawn in the iteration
 *  props       [max_iter][batch][GBK_NPAR] the proposals (rows past n_props unset)
 *  chi2        [max_iter][batch] their chi2
 *  replaced    [max_iter][batch] index of the live point a proposal replaced,
 *              -1 if it did not beat the worst live point */
typedef struct gbk_ns_trace {
    int32_t max_iter;
    int32_t n_iter;
    double *live0;
    double *live0_chi2;
    int32_t *n_props;
    double *props;
    double *chi2;
    int32_t *replaced;
} gbk_ns_trace;

/* gbk_nested_sample with its trajectory recorded in *trace (NULL: no
 * record).  The sampling is the same code path, so the results equal
 * gbk_nested_sample's for the same inputs.  Errors: as gbk_nested_sample;
 * GBK_EINVAL if trace->max_iter < 0. */
GBK_API gbk_status gbk_nested_sample_traced(const gbk_geom *g, const gbk_obs *obs, const double *lo,
                                            const double *hi, const gbk_ns_opts *opts, double *post_mean,
                                            double *post_std, double *log_z, int64_t *n_eval, int32_t *n_iter,
                                            void *workspace, size_t ws_bytes, void *stream, gbk_ns_trace *trace);

/* Launch tuning of the fused path (no counterpart in the paper).  A tuning
 * is the number of CTAs that cooperate on one model (a thread-block cluster
 * of 1..16 CTAs sharing the model's extended rows through distributed shared
 * memory), the block size (512, 384 or 256 threads) and the grid shape.  The library keeps
 * one tuning per geometry (size, kernel radii, LSF mode) for the life of the
 * process; without one it uses a heuristic. */
typedef struct gbk_tuning {
    int32_t cluster_ctas;  /* CTAs per model                                  */
    int32_t threads;       /* threads per CTA                                 */
    int32_t persistent;    /* 1: one resident wave of clusters loops over the */
                           /* models; 0: one cluster per model                */
    float ms;              /* autotune: median time of the best candidate     */
    int32_t candidates;    /* autotune: configurations timed                  */
} gbk_tuning;

/* Times every valid tuning of the fused path on this batch (params, obs and
 * chi2_scratch as for gbk_chi2; chi2_scratch is overwritten) and keeps the
 * fastest for this geometry.  Synchronises `stream`; several launches per
 * candidate.  best (host) receives the choice.  Call it outside any stream
 * capture. */
GBK_API gbk_status gbk_autotune(const gbk_geom *g, int32_t n_models, const double *params,
                                const gbk_obs *obs, double *chi2_scratch, gbk_tuning *best,
                                void *stream);

/* The tuning the next fused call with this geometry will use (host out). */
GBK_API gbk_status gbk_get_tuning(const gbk_geom *g, gbk_tuning *out);

/* Sets the tuning for this geometry (e.g. one saved from an earlier
 * gbk_autotune); t == NULL forgets it.  EINVAL if it cannot run here. */
GBK_API gbk_status gbk_set_tuning(const gbk_geom *g, const gbk_tuning *t);

/* Survey tunings: how the fused evaluator serves one survey (keyed by the
 * sizes, kernel radii and LSF modes of its geometry list).  persistent = 1:
 * one persistent launch of cluster_ctas-CTA clusters of `threads` threads
 * over every galaxy; persistent = 0: one launch per cluster-size group
 * (cluster_ctas and threads 0).  gbk_survey_autotune times the per-group
 * launches and one launch with 512 and 256 threads at the four smallest
 * cluster sizes that fit every galaxy, on gbk_survey_eval of `params`
 * against `obs` (chi2_scratch [n_gal] is overwritten; the workspace is that
 * of gbk_survey_workspace_bytes(geoms, n_gal, NULL)), keeps the fastest for
 * this survey and returns it in best (host).  Synchronises `stream`; call
 * it outside any stream capture.  gbk_survey_get_tuning reports the shape
 * the next survey call will use; gbk_survey_set_tuning sets one (EINVAL if
 * it does not fit every galaxy) or, with t == NULL, forgets it. */
GBK_API gbk_status gbk_survey_autotune(const gbk_geom *geoms, int32_t n_gal, const double *params,
                                       const gbk_obs *obs, double *chi2_scratch, void *workspace, size_t ws_bytes,
                                       gbk_tuning *best, void *stream);
GBK_API gbk_status gbk_survey_get_tuning(const gbk_geom *geoms, int32_t n_gal, gbk_tuning *out);
GBK_API gbk_status gbk_survey_set_tuning(const gbk_geom *geoms, int32_t n_gal, const gbk_tuning *t);

/* Diagnostics (no counterpart in the paper): measured lane-operation rates
 * of the ALU pipes the fused evaluator is bound by -- FP32 FMA issued as
 * scalar and as packed f32x2 instructions, and the MUFU base-2 exponential
 * -- on the current device (each a 2-pass timed run of independent
 * dependency chains on every SM).  Synchronises `stream`.
 *  ffma_lane_ops_per_s    host output: scalar FFMA lane operations / s
 *  ffma2_lane_ops_per_s   host output: FMA lane operations / s via f32x2
 *  ex2_lane_ops_per_s     host output: ex2.approx lane operations / s */
GBK_API gbk_status gbk_measure_alu_peak(double *ffma_lane_ops_per_s, double *ffma2_lane_ops_per_s,
                                        double *ex2_lane_ops_per_s, void *stream);

/* Reads and clears the library's device status word (host output): 0 when
 * every bounded device-side wait since the last call completed; bit 0 set
 * when a TMA load of the staged convolution did not complete in time, bit 1
 * when a pipeline wait of the tensor-core GEMM did not (the affected blocks
 * stopped early and their output is incomplete), bit 2 when the wait of
 * gbk_wait_selfcheck ran out, bit 3 when a tile load of the PSF stage of the
 * split path or of the split Jacobian did not complete in time (that model's
 * outputs are not written).
 * Synchronising. */
GBK_API gbk_status gbk_device_status(int32_t *status);

/* Self-check of the bounded device waits: one thread runs the library's
 * mbarrier wait (at most `limit` try_wait attempts, each of which the
 * hardware may suspend for a bounded time, then give up) -- the wait the
 * TMA-fed convolution and the tensor-core GEMM use -- on a barrier that
 * nothing completes (complete = 0) or that one arrival completes first
 * (complete = 1).  A wait that runs out sets bit 2 of the device status
 * word and the kernel returns, so the timeout path is exercised without a
 * fault, a trap or a hang and the context stays usable.
 *  limit       1 .. 2^24 tries (the production waits allow 2^18: a try
 *              that finds its phase incomplete suspends about 3.75 us on
 *              GB300, so about one second)
 *  elapsed_ns  host output (or NULL): the wait's duration on the device
 *              clock (%globaltimer)
 * Synchronises `stream`; GBK_EINVAL on bad arguments. */
GBK_API gbk_status gbk_wait_selfcheck(int64_t limit, int32_t complete, int64_t *elapsed_ns, void *stream);

/* ------------------------------------------------------------------------
 * BF16 tensor-core GEMM (tcgen05, TMA-fed, FP32 accumulation in tensor
 * memory), the dense layer of the CNN that seeds the fits.  The paper has
 * no counterpart: it is the building block of the learned initial guess
 * that replaces the heuristic starting point of Sec. 2.1.9.
 *   D[m][n] = alpha * sum_k A[m][k] B[n][k] (+ bias[n]) (ReLU if relu != 0)
 *             (set to 0 where mask[m][n] <= 0, if mask != NULL)
 *  A        device BF16 [M][lda], lda >= K, lda % 8 == 0, 16-byte aligned
 *  B        device BF16 [N][ldb], ldb >= K, ldb % 8 == 0, 16-byte aligned
 *  bias     device FP32 [N] or NULL
 *  mask     device BF16 [M][ldm] or NULL
 *  out_bf16 device BF16 [M][ldo] or NULL; out_f32 device FP32 [M][ldo] or
 *           NULL (at least one)
 * Asynchronous on `stream`; GBK_EINVAL on bad sizes or pointers. */
GBK_API gbk_status gbk_gemm_bf16(int32_t M, int32_t N, int32_t K, const void *A, int32_t lda, const void *B,
                                 int32_t ldb, const float *bias, int32_t relu, const void *mask, int32_t ldm,
                                 float alpha, void *out_bf16, float *out_f32, int32_t ldo, void *stream);

/* ------------------------------------------------------------------------
 * CNN seed: a convolutional network that maps a galaxy's observed velocity
 * and dispersion maps to model parameters, the learned replacement for the
 * heuristic initial guess of the optimisers (Sec. 2.1.9).  Fixed
 * architecture for 64 x 64 maps (all convolutions 2 x 2, stride 2), four
 * convolutions and a two-layer MLP head, 1,225,968 parameters:
 *   input 64x64x4 (v / 200 km/s, sigma / 100 km/s, mask, 0; masked -> 0)
 *   conv -> 32x32x32, ReLU; conv -> 16x16x64, ReLU; conv -> 8x8x128, ReLU;
 *   conv -> 4x4x256, ReLU; dense 4096 -> 256, ReLU; dense 256 -> 16.
 * Parameters are one FP32 vector of gbk_cnn_param_count() floats: layer l
 * is [C_l][K_l + 1] (weights W_l[o][k], bias in column K_l), layers in
 * order; patch index k = (dy * p + dx) * C_in + c, and the dense layer's
 * flatten index is morton(y, x) * 256 + c with morton interleaving the bits
 * of x (even) and y (odd).  Outputs 0..9 are the normalised targets
 *   (x0 - 31.5) / 8, (y0 - 31.5) / 8, cos PA, sin PA, (i - 50) / 20,
 *   Vsys / 30, (Vmax - 175) / 75, (r_t - 4.5) / 2.5, (sigma0 - 45) / 25,
 *   (h - 7) / 3;
 * the loss is their mean squared error.  Dense products run on the tensor
 * cores (BF16 operands, FP32 accumulation); master weights, gradients and
 * Adam moments are FP32.  Maps are device FP32 [n][64][64] (v, sigma;
 * 16-byte aligned) and uint8 (mask, 1 = use; 4-byte aligned); n and the
 * batch B must be multiples of 8.  All
 * calls are asynchronous on `stream`; the workspace of
 * gbk_cnn_workspace_bytes(B) serves calls with exactly B samples.
 * ------------------------------------------------------------------------ */
GBK_API size_t gbk_cnn_param_count(void);
GBK_API size_t gbk_cnn_workspace_bytes(int32_t batch);
/* He-normal weights from a counter-based SplitMix64 stream, zero biases. */
GBK_API gbk_status gbk_cnn_init(float *params, uint64_t seed, void *stream);
/* targets [n][10] FP32 from parameter vectors [n][GBK_NPAR] FP64, and
 * parameters back from network outputs [n][16] (I0 := 1, PA in [0, 360)). */
GBK_API gbk_status gbk_cnn_targets(int32_t n, const double *params, float *targets, void *stream);
GBK_API gbk_status gbk_cnn_decode(int32_t n, const float *out, double *params, void *stream);
/* Training observations from model maps [n][3][64][64] (gbk_eval_cubes):
 * v = m1 + N(0, noise_v), sigma = m2 + N(0, sqrt(2) noise_v), mask 0 with
 * probability dead_frac or where m0 == 0.  Normal number j of the stream is
 * Box-Muller (cosine branch) of outputs 2j+1 and 2j+2 of SplitMix64 seeded
 * with `seed`; pixel i uses j = 2i (v) and 2i+1 (sigma); the dead-fibre
 * uniforms are output i+1 of SplitMix64 seeded with seed ^ 0xD1B54A32D192ED03. */
GBK_API gbk_status gbk_cnn_synth_obs(int32_t n, const float *maps, uint64_t seed, float noise_v, float dead_frac,
                                     float *v, float *sigma, uint8_t *mask, void *stream);
/* Network outputs out [n][16] FP32 for n samples (workspace for batch n). */
GBK_API gbk_status gbk_cnn_forward(const float *params, int32_t n, const float *v, const float *sigma,
                                   const uint8_t *mask, float *out, void *workspace, size_t ws_bytes, void *stream);
/* Loss and its gradient (parameter layout) for a batch of B samples with
 * targets [B][10]; grad and loss (device, 1 float) may be NULL. */
GBK_API gbk_status gbk_cnn_grad(const float *params, int32_t B, const float *v, const float *sigma,
                                const uint8_t *mask, const float *targets, float *grad, float *loss, void *workspace,
                                size_t ws_bytes, void *stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected; `step`
 * counts from 1) on params with moments adam_m, adam_v (same layout,
 * caller-zeroed before step 1). */
GBK_API gbk_status gbk_cnn_train_step(float *params, float *adam_m, float *adam_v, int32_t step, float lr,
                                      int32_t B, const float *v, const float *sigma, const uint8_t *mask,
                                      const float *targets, float *loss, void *workspace, size_t ws_bytes,
                                      void *stream);

/* Message of the last failed call on this thread ("" if none). */
GBK_API const char *gbk_last_error(void);

/* Library version string. */
GBK_API const char *gbk_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GBK_API_H_INCLUDED */
