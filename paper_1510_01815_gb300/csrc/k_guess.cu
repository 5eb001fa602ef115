// k_guess.cu -- initial model parameter values measured on an observation's
// maps (Sec. 2.1.9): the optimisers' starting point when no better one is
// known.
//
//   centre (x0, y0): intensity-weighted mean position of the continuum map
//     (negative values count as 0; no light: the image centre);
//   V_sys: mean velocity of the unmasked pixels within 2.5 pixels of that
//     centre (no grid pixel lies at exactly that distance from a pixel
//     centre; if none is that close, of all unmasked pixels; none: 0);
//   PA: with x_e = r sin(phi - PA) (Eqs. 1-2, phi the polar angle about the
//     centre) the receding half x_e > 0 is the polar range (PA, PA + 180);
//     the unmasked pixels are binned by whole degrees of phi and the whole
//     degree PA with the largest mean(x_e > 0) - mean(x_e < 0) is taken
//     (ties to the smaller PA);
//   i: the eigenvalues of the continuum's intensity-weighted second central
//     moments, each less the PSF variance, have the ratio cos^2 i; clipped
//     to [5, 85] degrees (the paper takes a catalogue inclination);
//   r_t: the photometric scale radius, i.e. h (cube models) or the caller's
//     value (velocity fields); V_t = 150, sigma0 = 30 km/s; I0 and h as
//     given (cube), a = g = 1 (Epinat).
// One CTA per galaxy, FP64 arithmetic (a few passes over the maps), fixed-
// order reductions; the per-degree velocity sums are fixed-point integers,
// so their atomic accumulation is exact and the result deterministic.
#include "gbk_api_internal.h"

namespace gbk {

constexpr int kGuessThreads = 256;
constexpr double kVsysRadius = 2.5;
constexpr double kVFix = 1048576.0;  // fixed-point scale of the per-degree velocity sums

// Block sum of one double per thread in a fixed order (warps by shuffles,
// then the warps in order); every thread receives the total.
__device__ double guess_block_sum(double v, double *red)
{
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    const int w = threadIdx.x >> 5;
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    for (int q = 0; q < kGuessThreads / 32; ++q) s += red[q];
    return s;
}

__global__ void __launch_bounds__(kGuessThreads) initial_guess_kernel(Geom g, int n, const float *cont,
                                                                      const gbk_obs *obs_list, const double *fixed,
                                                                      double *out)
{
    __shared__ double red[kGuessThreads / 32];
    __shared__ unsigned long long hv[360];
    __shared__ unsigned int hc[360];
    __shared__ double sd[360];
    __shared__ int sbest[kGuessThreads / 32];
    __shared__ double sbestd[kGuessThreads / 32];
    const int tid = threadIdx.x, nx = g.nx, np = g.nx * g.ny;
    const double kPi = 3.141592653589793;
    for (int gal = blockIdx.x; gal < n; gal += gridDim.x) {
        const gbk_obs ob = obs_list[gal];
        const float *I = cont ? cont + (size_t)gal * np : nullptr;
        // centroid
        double s = 0.0, sx = 0.0, sy = 0.0;
        for (int p = tid; p < np; p += kGuessThreads) {
            const double w = I ? fmax((double)I[p], 0.0) : (ob.mask[p] != 0 ? 1.0 : 0.0);
            const int y = p / nx, x = p - y * nx;
            s += w;
            sx += w * x;
            sy += w * y;
        }
        const double S = guess_block_sum(s, red);
        const double SX = guess_block_sum(sx, red), SY = guess_block_sum(sy, red);
        const bool lit = S > 0.0;
        const double x0 = lit ? SX / S : 0.5 * (nx - 1), y0 = lit ? SY / S : 0.5 * (g.ny - 1);
        // second moments, central velocity, per-degree velocity histogram
        for (int b = tid; b < 360; b += kGuessThreads) {
            hv[b] = 0ull;
            hc[b] = 0u;
        }
        __syncthreads();
        double mxx = 0.0, myy = 0.0, mxy = 0.0, vn = 0.0, cn = 0.0, va = 0.0, ca = 0.0;
        for (int p = tid; p < np; p += kGuessThreads) {
            const int y = p / nx, x = p - y * nx;
            const double dx = x - x0, dy = y - y0;
            const double w = I ? fmax((double)I[p], 0.0) : (ob.mask[p] != 0 ? 1.0 : 0.0);
            mxx += w * dx * dx;
            myy += w * dy * dy;
            mxy += w * dx * dy;
            if (ob.mask[p] == 0) continue;
            const double v = (double)ob.v_obs[p];
            va += v;
            ca += 1.0;
            if (dx * dx + dy * dy <= kVsysRadius * kVsysRadius) {
                vn += v;
                cn += 1.0;
            }
            if (dx == 0.0 && dy == 0.0) continue;
            double phi = atan2(dy, dx) * (180.0 / kPi);
            if (phi < 0.0) phi += 360.0;
            int b = (int)floor(phi);
            b = b < 0 ? 0 : (b > 359 ? 359 : b);
            atomicAdd(&hv[b], (unsigned long long)(long long)llrint(v * kVFix));
            atomicAdd(&hc[b], 1u);
        }
        const double MXX = guess_block_sum(mxx, red), MYY = guess_block_sum(myy, red);
        const double MXY = guess_block_sum(mxy, red);
        const double VN = guess_block_sum(vn, red), CN = guess_block_sum(cn, red);
        const double VA = guess_block_sum(va, red), CA = guess_block_sum(ca, red);
        // (the histogram is complete: guess_block_sum ends with a barrier)
        // PA: the receding half of candidate PA is bins PA .. PA + 179
        long long tot_v = 0;
        unsigned int tot_c = 0;
        for (int b = 0; b < 360; ++b) {
            tot_v += (long long)hv[b];
            tot_c += hc[b];
        }
        for (int pa = tid; pa < 360; pa += kGuessThreads) {
            long long av = 0;
            unsigned int ac = 0;
            for (int k = 0; k < 180; ++k) {
                const int b = pa + k < 360 ? pa + k : pa + k - 360;
                av += (long long)hv[b];
                ac += hc[b];
            }
            const unsigned int bc = tot_c - ac;
            sd[pa] = (ac == 0u || bc == 0u) ? -1e300
                                             : (double)av / kVFix / ac - (double)(tot_v - av) / kVFix / bc;
        }
        __syncthreads();
        // argmax over the 360 candidates, ties to the smaller PA
        int best = -1;
        double bestd = -1e300;
        for (int pa = tid; pa < 360; pa += kGuessThreads)
            if (sd[pa] > bestd) {
                bestd = sd[pa];
                best = pa;
            }
        for (int off = 16; off > 0; off >>= 1) {
            const double od = __shfl_down_sync(0xffffffffu, bestd, off);
            const int ob_ = __shfl_down_sync(0xffffffffu, best, off);
            if (od > bestd || (od == bestd && ob_ >= 0 && (best < 0 || ob_ < best))) {
                bestd = od;
                best = ob_;
            }
        }
        if ((tid & 31) == 0) {
            sbest[tid >> 5] = best;
            sbestd[tid >> 5] = bestd;
        }
        __syncthreads();
        if (tid == 0) {
            int pa = -1;
            double d = -1e300;
            for (int q = 0; q < kGuessThreads / 32; ++q)
                if (sbest[q] >= 0 && (sbestd[q] > d || (sbestd[q] == d && sbest[q] < pa))) {
                    d = sbestd[q];
                    pa = sbest[q];
                }
            // inclination from the PSF-corrected moments
            double incl = 45.0;
            if (lit) {
                const double mx = MXX / S, my = MYY / S, mc = MXY / S;
                const double tr = mx + my, det = mx * my - mc * mc;
                const double disc = sqrt(fmax(0.25 * tr * tr - det, 0.0));
                const double v2 = (double)g.sig_xy * (double)g.sig_xy;
                const double lmax = 0.5 * tr + disc - v2, lmin = 0.5 * tr - disc - v2;
                if (lmax > 0.0 && lmin > 0.0)
                    incl = fmin(fmax(acos(sqrt(fmin(lmin / lmax, 1.0))) * (180.0 / kPi), 5.0), 85.0);
                else if (lmax > 0.0)
                    incl = 85.0;
            }
            const double *f = fixed + (size_t)gal * GBK_NPAR;
            double *o = out + (size_t)gal * GBK_NPAR;
            for (int k = 0; k < GBK_NPAR; ++k) o[k] = f[k];
            o[GBK_X0] = x0;
            o[GBK_Y0] = y0;
            o[GBK_PA] = pa >= 0 ? (double)pa : 0.0;
            o[GBK_INCL] = incl;
            o[GBK_VSYS] = CN > 0.0 ? VN / CN : (CA > 0.0 ? VA / CA : 0.0);
            o[GBK_VMAX] = 150.0;
            o[GBK_SIG0] = 30.0;
            if (g.model == GBK_MODEL_VFIELD_EPINAT) {
                o[GBK_EPI_A] = 1.0;
                o[GBK_EPI_G] = 1.0;
            } else if (g.model == GBK_MODEL_CUBE) {
                o[GBK_RT] = f[GBK_H];
            }
        }
        __syncthreads();  // the shared tables are rewritten for the next galaxy
    }
}

}  // namespace gbk

using namespace gbk;

extern "C" gbk_status gbk_initial_guess(const gbk_geom *gin, int32_t n_gal, const float *continuum,
                                        const gbk_obs *obs, const double *fixed, double *params_out, void *stream)
{
    Geom g;
    gbk_status s = derive_geom(gin, &g);
    if (s) return s;
    if (n_gal < 0) return fail(GBK_EINVAL, "n_gal must be >= 0");
    if (n_gal == 0) return ok();
    if ((long)g.nx * g.ny > (1L << 26)) return fail(GBK_EINVAL, "maps too large for the fixed-point velocity sums");
    if (continuum && (s = check_device_ptr(continuum, "continuum", 4))) return s;
    if ((s = check_device_ptr(obs, "obs", 8)) || (s = check_device_ptr(fixed, "fixed", 8)) ||
        (s = check_device_ptr(params_out, "params_out", 8)))
        return s;
    const int blocks = n_gal < 152 * 8 ? n_gal : 152 * 8;
    initial_guess_kernel<<<blocks, kGuessThreads, 0, (cudaStream_t)stream>>>(g, n_gal, continuum, obs, fixed,
                                                                             params_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "initial-guess launch");
    return ok();
}
