/*
 * gbk_oracle.c -- FP64 CPU oracle of the disc-galaxy forward model.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct
 * definition of what the GPU library computes.  Only the test-suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header, table or constant generator with the CUDA path.
 *
 * Every step follows Bekiaris et al. 2015 (arXiv:1510.01815):
 *   geometry        Sec. 2.1.1, Eqs. 1-4
 *   brightness      Sec. 2.1.2, Eq. 5
 *   rotation curve  Sec. 2.1.3, Eq. 6
 *   LOS velocity    Sec. 2.1.5, Eq. 8
 *   cube            Sec. 2.2.2 (Gaussian line per spaxel, upsampling u)
 *   PSF x LSF       Sec. 2.1.7, Eq. 9 (a separable 3-D Gaussian)
 *   convolution     Sec. 2.2.3 (done here as a direct, unfactored 3-D sum)
 *   down-sampling   Sec. 2.2.4 (mean of u^3 blocks)
 *   moments         Sec. 2.2.5 (first/second moments of each spectrum)
 *   chi-squared     Sec. 2.2.6, Eq. 11 (W folded into the dispersion error)
 *
 * Readings where the paper is silent:
 *   - pixel centres sit at integer coordinates 0..N-1; channel k has velocity
 *     v_k = vc + (k - (nz-1)/2) dv;
 *   - the line is point-sampled and area-normalised:
 *       c = I(r) * dv * exp(-(v-v_los)^2 / (2 s^2)) / (s sqrt(2 pi));
 *   - Vrot(r) cos(theta) is evaluated as [Vrot(r)/r] x_e, whose r -> 0 limit
 *     is 2 Vmax / (pi r_t);
 *   - the Gaussian kernels are sampled at integer offsets |j| <= R with
 *     R = ceil(halo * sigma) and normalised to unit sum per axis;
 *   - the model is evaluated on the data grid extended by R on every side and
 *     the "valid" linear convolution is taken (no FFT, no power-of-two pad);
 *   - LSF mode 0: line width sigma0, then a 3-axis convolution; LSF mode 1:
 *     line width sqrt(sigma0^2 + sigma_LSF^2), spatial convolution only;
 *   - with u > 1, fine pixel j sits at coarse coordinate (j+0.5)/u - 0.5 and
 *     the kernel widths are scaled by u on the fine grid;
 *   - m0 = sum_k c_k; m1 = intensity-weighted mean velocity; m2 = intensity-
 *     weighted standard deviation; a spectrum with m0 <= 1e-20 I0 is invalid
 *     (m0 = 0, m1 = Vsys, m2 = 0) and is left out of chi-squared;
 *   - chi2 = sum over unmasked valid spaxels of (w_v (m1 - v_obs))^2 +
 *     (w_s (m2 - s_obs))^2 with w_v = 1/E_v and w_s = sqrt(W)/E_s.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OG_PI 3.14159265358979323846
/* FWHM = 2 sqrt(2 ln 2) sigma for a Gaussian. */
#define OG_FWHM_PER_SIGMA 2.3548200450309493
#define OG_INVALID_FRACTION 1e-20

enum { OG_X0, OG_Y0, OG_PA, OG_INCL, OG_VSYS, OG_VMAX, OG_RT, OG_SIG0, OG_I0, OG_H, OG_NPAR };

typedef struct {
    int32_t nx, ny, nz, upsample;
    double dv, vc, psf_fwhm, lsf_fwhm;
    int32_t lsf_mode;
    int32_t model;  /* 0 intensity cube (arctan curve); 1 velocity field,
                       arctan curve; 2 velocity field, Epinat curve */
    double halo_sigmas;
} og_geom;

/* Sizes of the fine, extended grid for one geometry. */
typedef struct {
    int u, nxf, nyf, nzf;      /* fine data grid: u * (nx, ny, nz) */
    int rxy, rz;               /* kernel radii on the fine grid */
    int exf, eyf, ezf;         /* fine extended grid */
    double sig_xy, sig_z;      /* kernel sigmas in fine pixels / channels */
} og_dims;

/* ------------------------------------------------------------------ */
/* Kernel taps: Eq. 9 is separable; each axis is a 1-D Gaussian sampled at
 * integer offsets and normalised to unit sum. */
int og_radius(double sigma, double halo)
{
    if (!(sigma > 0.0)) return 0;
    return (int)ceil(halo * sigma);
}

void og_taps(double sigma, int R, double *w)
{
    if (R == 0) { w[0] = 1.0; return; }
    double s = 0.0;
    for (int j = -R; j <= R; ++j) {
        w[j + R] = exp(-(double)j * (double)j / (2.0 * sigma * sigma));
        s += w[j + R];
    }
    for (int j = 0; j <= 2 * R; ++j) w[j] /= s;
}

void og_get_dims(const og_geom *g, og_dims *d)
{
    int u = g->upsample;
    d->u = u;
    d->nxf = u * g->nx; d->nyf = u * g->ny; d->nzf = u * g->nz;
    d->sig_xy = u * g->psf_fwhm / OG_FWHM_PER_SIGMA;
    d->rxy = og_radius(d->sig_xy, g->halo_sigmas);
    if (g->lsf_mode == 0) {
        d->sig_z = u * (g->lsf_fwhm / OG_FWHM_PER_SIGMA) / g->dv;
        d->rz = og_radius(d->sig_z, g->halo_sigmas);
    } else {
        d->sig_z = 0.0;
        d->rz = 0;
    }
    d->exf = d->nxf + 2 * d->rxy;
    d->eyf = d->nyf + 2 * d->rxy;
    d->ezf = d->nzf + 2 * d->rz;
}

/* Exposed for ctypes: [u, nxf, nyf, nzf, rxy, rz, exf, eyf, ezf]. */
void og_dims_array(const og_geom *g, int32_t *out)
{
    og_dims d; og_get_dims(g, &d);
    out[0] = d.u; out[1] = d.nxf; out[2] = d.nyf; out[3] = d.nzf;
    out[4] = d.rxy; out[5] = d.rz; out[6] = d.exf; out[7] = d.eyf; out[8] = d.ezf;
}

/* ------------------------------------------------------------------ */
/* Sec. 2.1.1, Eqs. 1-3: disc-plane coordinate x_e, deprojected radius r
 * and sin(i) for sky position (x, y), in data-pixel units. */
static void og_disc_coords(const double *p, double x, double y, double *xe_out, double *r_out, double *sin_i)
{
    double pa = p[OG_PA] * OG_PI / 180.0;
    double inc = p[OG_INCL] * OG_PI / 180.0;
    double dx = x - p[OG_X0], dy = y - p[OG_Y0];
    double xe = -dx * sin(pa) + dy * cos(pa);                 /* Eq. 1 */
    double ye = -dx * cos(pa) - dy * sin(pa);                 /* Eq. 2 */
    double yd = ye / cos(inc);
    *xe_out = xe;
    *r_out = sqrt(xe * xe + yd * yd);                         /* Eq. 3 */
    *sin_i = sin(inc);
}

/* Vrot(r) / r for the arctan curve (Eq. 6; r -> 0 limit 2 Vmax / (pi r_t))
 * or the Epinat curve (Eq. 7, V_t (r/r_t)^g / (1 + (r/r_t)^a) with a = p[8],
 * g = p[9]; 0 at r = 0, where x_e = 0 and cos(theta) has no limit).  Times
 * x_e it gives Vrot(r) cos(theta) with cos(theta) = x_e / r (Eq. 4). */
static double og_vrot_over_r(int epinat, const double *p, double r)
{
    if (epinat) {
        if (!(r > 0.0)) return 0.0;
        double q = r / p[OG_RT];
        return p[OG_VMAX] * pow(q, p[OG_H]) / (1.0 + pow(q, p[OG_I0])) / r;
    }
    if (r > 0.0) return (2.0 / OG_PI) * p[OG_VMAX] * atan(r / p[OG_RT]) / r;
    return (2.0 / OG_PI) * p[OG_VMAX] / p[OG_RT];
}

/* Sec. 2.1: line-of-sight velocity (Eq. 8, arctan curve) and surface
 * brightness (Eq. 5) at sky position (x, y), in data-pixel units. */
void og_los(const double *p, double x, double y, double *v_los, double *bright)
{
    double xe, r, si;
    og_disc_coords(p, x, y, &xe, &r, &si);
    *v_los = p[OG_VSYS] + og_vrot_over_r(0, p, r) * xe * si;  /* Eq. 8 */
    *bright = p[OG_I0] * exp(-r / p[OG_H]);                   /* Eq. 5 */
}

void og_los_grid(const double *p, int n, const double *x, const double *y,
                 double *v_los, double *bright)
{
    for (int i = 0; i < n; ++i) og_los(p, x[i], y[i], &v_los[i], &bright[i]);
}

static double og_line_sigma(const og_geom *g, const double *p)
{
    if (g->lsf_mode == 0) return p[OG_SIG0];
    double sl = g->lsf_fwhm / OG_FWHM_PER_SIGMA;
    return sqrt(p[OG_SIG0] * p[OG_SIG0] + sl * sl);
}

/* Velocity of fine channel kf (may lie in the extended band). */
static double og_fine_velocity(const og_geom *g, int u, int kf)
{
    double kc = ((double)kf + 0.5) / u - 0.5;
    return g->vc + (kc - 0.5 * (g->nz - 1)) * g->dv;
}

/* Sec. 2.2.2: the model cube on the fine extended grid, layout [z][y][x],
 * ezf * eyf * exf values. */
void og_model_cube(const og_geom *g, const double *p, double *ext)
{
    og_dims d; og_get_dims(g, &d);
    double s = og_line_sigma(g, p);
    double norm = g->dv / (s * sqrt(2.0 * OG_PI));
    double *vl = (double *)malloc(sizeof(double) * d.exf * d.eyf);
    double *br = (double *)malloc(sizeof(double) * d.exf * d.eyf);
    for (int ye = 0; ye < d.eyf; ++ye) {
        double y = ((double)(ye - d.rxy) + 0.5) / d.u - 0.5;
        for (int xe = 0; xe < d.exf; ++xe) {
            double x = ((double)(xe - d.rxy) + 0.5) / d.u - 0.5;
            og_los(p, x, y, &vl[ye * d.exf + xe], &br[ye * d.exf + xe]);
        }
    }
    for (int ze = 0; ze < d.ezf; ++ze) {
        double v = og_fine_velocity(g, d.u, ze - d.rz);
        for (int i = 0; i < d.exf * d.eyf; ++i) {
            double t = (v - vl[i]) / s;
            ext[(size_t)ze * d.exf * d.eyf + i] = br[i] * norm * exp(-0.5 * t * t);
        }
    }
    free(vl); free(br);
}

/* Sec. 2.2.3 with Eq. 9: direct 3-D "valid" convolution of the extended cube
 * with the product kernel wz(c) wy(b) wx(a).  No factorisation. */
void og_conv3d_direct(const double *ext, int ex, int ey, int ez,
                      const double *wx, int rx, const double *wy, int ry,
                      const double *wz, int rz, double *out)
{
    int ox = ex - 2 * rx, oy = ey - 2 * ry, oz = ez - 2 * rz;
    for (int k = 0; k < oz; ++k)
        for (int j = 0; j < oy; ++j)
            for (int i = 0; i < ox; ++i) {
                double acc = 0.0;
                for (int c = -rz; c <= rz; ++c)
                    for (int b = -ry; b <= ry; ++b)
                        for (int a = -rx; a <= rx; ++a) {
                            double w = wz[c + rz] * wy[b + ry] * wx[a + rx];
                            size_t src = ((size_t)(k + rz + c) * ey + (j + ry + b)) * ex + (i + rx + a);
                            acc += w * ext[src];
                        }
                out[((size_t)k * oy + j) * ox + i] = acc;
            }
}

/* The same valid convolution done as three 1-D passes (x, then y, then z).
 * Kept only as a second, independent check of the direct form. */
void og_conv3d_separable(const double *ext, int ex, int ey, int ez,
                         const double *wx, int rx, const double *wy, int ry,
                         const double *wz, int rz, double *out)
{
    int ox = ex - 2 * rx, oy = ey - 2 * ry, oz = ez - 2 * rz;
    double *t1 = (double *)malloc(sizeof(double) * (size_t)ez * ey * ox);
    double *t2 = (double *)malloc(sizeof(double) * (size_t)ez * oy * ox);
    for (int k = 0; k < ez; ++k)
        for (int j = 0; j < ey; ++j)
            for (int i = 0; i < ox; ++i) {
                double acc = 0.0;
                for (int a = -rx; a <= rx; ++a)
                    acc += wx[a + rx] * ext[((size_t)k * ey + j) * ex + i + rx + a];
                t1[((size_t)k * ey + j) * ox + i] = acc;
            }
    for (int k = 0; k < ez; ++k)
        for (int j = 0; j < oy; ++j)
            for (int i = 0; i < ox; ++i) {
                double acc = 0.0;
                for (int b = -ry; b <= ry; ++b)
                    acc += wy[b + ry] * t1[((size_t)k * ey + j + ry + b) * ox + i];
                t2[((size_t)k * oy + j) * ox + i] = acc;
            }
    for (int k = 0; k < oz; ++k)
        for (int j = 0; j < oy; ++j)
            for (int i = 0; i < ox; ++i) {
                double acc = 0.0;
                for (int c = -rz; c <= rz; ++c)
                    acc += wz[c + rz] * t2[((size_t)(k + rz + c) * oy + j) * ox + i];
                out[((size_t)k * oy + j) * ox + i] = acc;
            }
    free(t1); free(t2);
}

/* Sec. 2.2.4: each output voxel is the mean of its u x u x u fine block. */
void og_downsample(const double *fine, int u, int nx, int ny, int nz, double *coarse)
{
    int fx = u * nx, fy = u * ny;
    double inv = 1.0 / ((double)u * u * u);
    for (int k = 0; k < nz; ++k)
        for (int j = 0; j < ny; ++j)
            for (int i = 0; i < nx; ++i) {
                double acc = 0.0;
                for (int c = 0; c < u; ++c)
                    for (int b = 0; b < u; ++b)
                        for (int a = 0; a < u; ++a)
                            acc += fine[((size_t)(k * u + c) * fy + (j * u + b)) * fx + (i * u + a)];
                coarse[((size_t)k * ny + j) * nx + i] = acc * inv;
            }
}

/* Sec. 2.2.5: moment maps of a data cube [nz][ny][nx].  maps is [3][ny][nx]
 * = (m0, m1, m2).  Two passes: the mean first, then the central second
 * moment.  Spectra with m0 <= 1e-20 * scale are invalid and get
 * (0, v_invalid, 0). */
void og_moments(const double *cube, int nx, int ny, int nz, double dv, double vc,
                double scale, double v_invalid, double *maps)
{
    int np = nx * ny;
    for (int s = 0; s < np; ++s) {
        double s0 = 0.0, s1 = 0.0;
        for (int k = 0; k < nz; ++k) {
            double c = cube[(size_t)k * np + s];
            double v = vc + (k - 0.5 * (nz - 1)) * dv;
            s0 += c;
            s1 += c * v;
        }
        if (!(s0 > OG_INVALID_FRACTION * scale)) {
            maps[s] = 0.0; maps[np + s] = v_invalid; maps[2 * np + s] = 0.0;
            continue;
        }
        double m1 = s1 / s0;
        double s2 = 0.0;
        for (int k = 0; k < nz; ++k) {
            double v = vc + (k - 0.5 * (nz - 1)) * dv;
            s2 += cube[(size_t)k * np + s] * (v - m1) * (v - m1);
        }
        maps[s] = s0;
        maps[np + s] = m1;
        maps[2 * np + s] = sqrt(s2 / s0);
    }
}

/* ------------------------------------------------------------------ */
/* Velocity-field strategy (Sec. 2.2.1 with Sec. 2.1.5): Eq. 8 evaluated at
 * every data pixel -- no cube, no PSF or LSF.  The strategy has no intensity
 * model, so every pixel is valid (m0 = 1); m2 is the constant dispersion
 * model sigma_model = p[SIG0] (Sec. 2.1.4).  Rotation curve: the arctan
 * function (Eq. 6) for model 1; the Epinat function (Eq. 7),
 *   Vrot(r) = V_t (r/r_t)^g / (1 + (r/r_t)^a),
 * for model 2, with a = p[8] and g = p[9] (the intensity slots, unused by a
 * velocity field).  Vrot(r) cos(theta) = [Vrot(r)/r] x_e as in og_los; at
 * r = 0 the Epinat field is Vsys (cos(theta) has no limit there). */
void og_vfield(const og_geom *g, const double *p, double *maps)
{
    const int np = g->nx * g->ny;
    for (int y = 0; y < g->ny; ++y)
        for (int x = 0; x < g->nx; ++x) {
            double xe, r, si;
            og_disc_coords(p, x, y, &xe, &r, &si);
            int s = y * g->nx + x;
            maps[s] = 1.0;
            maps[np + s] = p[OG_VSYS] + og_vrot_over_r(g->model == 2, p, r) * xe * si;  /* Eq. 8 */
            maps[2 * np + s] = p[OG_SIG0];
        }
}

/* Parameter domain (the reading of the parameter ranges shared with the
 * library): 0 <= i < 90 degrees and r_t > 0 for every model; the cube model
 * also needs sigma0, I0, h > 0 and all ten values finite; a velocity field
 * needs sigma0 >= 0 and x0 .. sigma0 finite (and, for the Epinat curve, its
 * slopes a, g).  Outside it the maps and chi2 are NaN. */
int og_param_valid(const og_geom *g, const double *p)
{
    int ok = p[OG_INCL] >= 0.0 && p[OG_INCL] < 90.0 && p[OG_RT] > 0.0;
    if (g->model == 0) {
        ok = ok && p[OG_SIG0] > 0.0 && p[OG_I0] > 0.0 && p[OG_H] > 0.0;
        for (int k = 0; k < OG_NPAR; ++k) ok = ok && isfinite(p[k]);
    } else {
        ok = ok && p[OG_SIG0] >= 0.0;
        for (int k = 0; k <= OG_SIG0; ++k) ok = ok && isfinite(p[k]);
        if (g->model == 2) ok = ok && isfinite(p[OG_I0]) && isfinite(p[OG_H]);
    }
    return ok;
}

/* Which form of the Sec. 2.2.3 convolution og_eval uses: 0 = the direct,
 * unfactored 3-D sum (the default and the definition); 1 = the three 1-D
 * passes of og_conv3d_separable, which equal it up to rounding (the two are
 * compared term by term on small cubes) and cost about 3(2R+1) instead of
 * (2R+1)^3 products per voxel, so that sweeps of 10^5 models finish.  The
 * choice is process-wide and is made before any evaluation starts. */
static int og_conv_form = 0;

void og_set_conv_form(int separable) { og_conv_form = separable ? 1 : 0; }
int og_get_conv_form(void) { return og_conv_form; }

/* Steps 1-5 of one model: cube (optional output, data resolution) and maps. */
void og_eval(const og_geom *g, const double *p, double *cube_out, double *maps_out)
{
    if (!og_param_valid(g, p)) {
        if (maps_out)
            for (int s = 0; s < 3 * g->nx * g->ny; ++s) maps_out[s] = NAN;
        if (cube_out && g->model == 0)
            for (size_t s = 0; s < (size_t)g->nx * g->ny * g->nz; ++s) cube_out[s] = NAN;
        return;
    }
    if (g->model != 0) {  /* velocity field: no cube */
        if (maps_out) og_vfield(g, p, maps_out);
        return;
    }
    og_dims d; og_get_dims(g, &d);
    double *wx = (double *)malloc(sizeof(double) * (2 * d.rxy + 1));
    double *wz = (double *)malloc(sizeof(double) * (2 * d.rz + 1));
    og_taps(d.sig_xy, d.rxy, wx);
    og_taps(d.sig_z, d.rz, wz);
    size_t next = (size_t)d.exf * d.eyf * d.ezf;
    size_t nfine = (size_t)d.nxf * d.nyf * d.nzf;
    size_t ndata = (size_t)g->nx * g->ny * g->nz;
    double *ext = (double *)malloc(sizeof(double) * next);
    double *fine = (double *)malloc(sizeof(double) * nfine);
    double *data = cube_out ? cube_out : (double *)malloc(sizeof(double) * ndata);
    og_model_cube(g, p, ext);
    if (og_conv_form) og_conv3d_separable(ext, d.exf, d.eyf, d.ezf, wx, d.rxy, wx, d.rxy, wz, d.rz, fine);
    else og_conv3d_direct(ext, d.exf, d.eyf, d.ezf, wx, d.rxy, wx, d.rxy, wz, d.rz, fine);
    if (d.u == 1) memcpy(data, fine, sizeof(double) * ndata);
    else og_downsample(fine, d.u, g->nx, g->ny, g->nz, data);
    if (maps_out)
        og_moments(data, g->nx, g->ny, g->nz, g->dv, g->vc, p[OG_I0], p[OG_VSYS], maps_out);
    if (!cube_out) free(data);
    free(ext); free(fine); free(wx); free(wz);
}

/* Neumaier-compensated accumulation. */
typedef struct { double s, c; } og_sum;
static void og_add(og_sum *a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}

/* Eq. 11 over unmasked, valid spaxels.  resid (optional) is [2][ny*nx]:
 * w_v (m1 - v_obs) and w_s (m2 - s_obs), zero where left out. */
double og_chi2_maps(const double *maps, int np, const float *v_obs, const float *s_obs,
                    const float *w_v, const float *w_s, const uint8_t *mask, double *resid)
{
    og_sum acc = {0.0, 0.0};
    for (int s = 0; s < np; ++s) {
        double rv = 0.0, rs = 0.0;
        if (mask[s] != 0 && maps[s] > 0.0) {
            rv = (double)w_v[s] * (maps[np + s] - (double)v_obs[s]);
            rs = (double)w_s[s] * (maps[2 * np + s] - (double)s_obs[s]);
            og_add(&acc, rv * rv);
            og_add(&acc, rs * rs);
        }
        if (resid) { resid[s] = rv; resid[np + s] = rs; }
    }
    return acc.s + acc.c;
}

/* Batched forms (one model per OpenMP iteration).  maps: [n][3][ny][nx]. */
void og_eval_batch(const og_geom *g, int n, const double *params, double *maps, int nthreads)
{
    size_t nm = (size_t)3 * g->nx * g->ny;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int m = 0; m < n; ++m)
        og_eval(g, params + (size_t)m * OG_NPAR, NULL, maps + (size_t)m * nm);
    (void)nthreads;
}

void og_chi2_batch(const og_geom *g, int n, const double *params, const float *v_obs,
                   const float *s_obs, const float *w_v, const float *w_s,
                   const uint8_t *mask, double *chi2, double *resid, int nthreads)
{
    int np = g->nx * g->ny;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int m = 0; m < n; ++m) {
        double *maps = (double *)malloc(sizeof(double) * 3 * np);
        const double *pm = params + (size_t)m * OG_NPAR;
        og_eval(g, pm, NULL, maps);
        if (og_param_valid(g, pm)) {
            chi2[m] = og_chi2_maps(maps, np, v_obs, s_obs, w_v, w_s, mask,
                                   resid ? resid + (size_t)m * 2 * np : NULL);
        } else {  /* outside the domain: NaN, as are the unmasked residuals */
            chi2[m] = NAN;
            if (resid)
                for (int s = 0; s < np; ++s)
                    resid[(size_t)m * 2 * np + s] = resid[(size_t)m * 2 * np + np + s] = mask[s] != 0 ? NAN : 0.0;
        }
        free(maps);
    }
    (void)nthreads;
}

int og_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
