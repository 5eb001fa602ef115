// k_vfield.cu -- the velocity-field modelling strategy (Sec. 2.2.1): Eq. 8
// evaluated at every data pixel directly, with the arctan (Eq. 6) or the
// Epinat (Eq. 7) rotation curve, then the residuals and chi-squared of
// Eq. 11.  There is no cube and no PSF or LSF; m0 = 1 (every pixel valid)
// and m2 = sigma0, the constant dispersion model of Sec. 2.1.4.
//
// One CTA per model (grid-stride over models), consecutive pixels on
// consecutive threads (coalesced map reads and writes, as the paper's
// evaluation kernel does), Kahan sums per thread and a fixed-order FP64
// block reduction, so chi2 is bitwise reproducible.
#include "gbk_api_internal.h"
#include "k_fused.h"

namespace gbk {

constexpr int kVfThreads = 256;

struct VfConst {
    float x0, y0, sin_pa, cos_pa, sin_i, inv_cos_i, vsys, sig0;
    float vk, inv_rt;   // arctan: (2/pi) Vmax and 1/r_t; Epinat: V_t and 1/r_t
    float a, g;         // Epinat slopes
    int epinat, valid;
};

__device__ inline VfConst vf_const(const double *p, int model)
{
    VfConst c;
    c.epinat = model == GBK_MODEL_VFIELD_EPINAT;
    bool ok = (p[GBK_INCL] >= 0.0) && (p[GBK_INCL] < 90.0) && (p[GBK_RT] > 0.0) && (p[GBK_SIG0] >= 0.0);
    for (int k = 0; k <= GBK_SIG0; ++k) ok = ok && isfinite(p[k]);
    if (c.epinat) ok = ok && isfinite(p[GBK_EPI_A]) && isfinite(p[GBK_EPI_G]);
    c.valid = ok ? 1 : 0;
    float sp, cp, si, ci;
    sincospif((float)(p[GBK_PA] * (1.0 / 180.0)), &sp, &cp);
    sincospif((float)(p[GBK_INCL] * (1.0 / 180.0)), &si, &ci);
    c.x0 = (float)p[GBK_X0];
    c.y0 = (float)p[GBK_Y0];
    c.sin_pa = sp;
    c.cos_pa = cp;
    c.sin_i = si;
    c.inv_cos_i = 1.0f / ci;
    c.vsys = (float)p[GBK_VSYS];
    c.sig0 = (float)p[GBK_SIG0];
    c.vk = c.epinat ? (float)p[GBK_VMAX] : (float)(0.63661977236758134 * p[GBK_VMAX]);
    c.inv_rt = 1.0f / (float)p[GBK_RT];
    c.a = c.epinat ? (float)p[GBK_EPI_A] : 0.f;
    c.g = c.epinat ? (float)p[GBK_EPI_G] : 0.f;
    return c;
}

// Eq. 8 at pixel (x, y): Vsys + [Vrot(r)/r] x_e sin i (Eqs. 1-4, 6 or 7).
__device__ __forceinline__ float vf_velocity(const VfConst &c, float x, float y)
{
    float dx = x - c.x0, dy = y - c.y0;
    float xe = -dx * c.sin_pa + dy * c.cos_pa;  // Eq. 1
    float ye = -dx * c.cos_pa - dy * c.sin_pa;  // Eq. 2
    float yd = ye * c.inv_cos_i;
    float r = sqrtf(xe * xe + yd * yd);         // Eq. 3
    float f;
    if (c.epinat) {
        float q = r * c.inv_rt;
        f = (r > 0.f) ? c.vk * powf(q, c.g) / ((1.f + powf(q, c.a)) * r) : 0.f;  // Eq. 7 / r
    } else {
        f = (r > 0.f) ? c.vk * atanf(r * c.inv_rt) / r : c.vk * c.inv_rt;        // Eq. 6 / r
    }
    return c.vsys + f * xe * c.sin_i;
}

__global__ void __launch_bounds__(kVfThreads) vfield_kernel(FusedArgs a)
{
    __shared__ VfConst s_c;
    __shared__ gbk_obs s_ob;
    __shared__ double red[kVfThreads / 32];
    const int tid = threadIdx.x;
    const int nx = a.g.nx, np = a.g.nx * a.g.ny;
    const int mpg = a.models_per_gal;
    const float nanf_ = __int_as_float(0x7fc00000);
    for (int model = blockIdx.x; model < a.n_models; model += gridDim.x) {
        const int gal = mpg > 0 ? model / mpg : 0;
        if (a.skip && a.skip[gal] != 0) continue;
        if (tid == 0) {
            s_c = vf_const(a.params + (size_t)model * GBK_NPAR, a.g.model);
            s_ob = a.obs_list ? a.obs_list[gal] : a.obs;
        }
        __syncthreads();
        const VfConst c = s_c;
        const bool want_obs = a.chi2 || a.resid;
        float s = 0.f, comp = 0.f;  // Kahan
        for (int pix = tid; pix < np; pix += kVfThreads) {
            const int y = pix / nx, x = pix - y * nx;
            float m1 = c.valid ? vf_velocity(c, (float)x, (float)y) : nanf_;
            float m2 = c.valid ? c.sig0 : nanf_;
            float m0 = c.valid ? 1.f : nanf_;
            if (a.maps) {
                float *mp = a.maps + (size_t)model * 3 * np;
                mp[pix] = m0;
                mp[np + pix] = m1;
                mp[2 * np + pix] = m2;
            }
            if (want_obs) {
                float rv = 0.f, rs = 0.f;
                if (s_ob.mask[pix] != 0) {
                    rv = s_ob.w_v[pix] * (m1 - s_ob.v_obs[pix]);
                    rs = s_ob.w_s[pix] * (m2 - s_ob.s_obs[pix]);
                }
                if (a.resid) {
                    float *rp = a.resid + (size_t)model * 2 * np;
                    rp[pix] = rv;
                    rp[np + pix] = rs;
                }
                float t2 = rv * rv + rs * rs;
                float yk = t2 - comp, tk = s + yk;
                comp = (tk - s) - yk;
                s = tk;
            }
        }
        if (a.chi2) {
            double v = (double)s - (double)comp;
            for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
            if ((tid & 31) == 0) red[tid >> 5] = v;
            __syncthreads();
            if (tid == 0) {
                double tot = 0.0;
                for (int w = 0; w < kVfThreads / 32; ++w) tot += red[w];
                a.chi2[model] = c.valid ? tot : (double)nanf_;
            }
        }
        __syncthreads();  // s_c, s_ob and red are rewritten by the next model
    }
}

gbk_status launch_vfield(const FusedArgs &a, cudaStream_t st)
{
    if (a.geoms) return fail(GBK_EUNSUPPORTED, "survey batches serve the intensity-cube model");
    if (a.n_models <= 0) return GBK_OK;
    int blocks = a.n_models < 152 * 16 ? a.n_models : 152 * 16;
    vfield_kernel<<<blocks, kVfThreads, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "velocity-field kernel launch");
    return GBK_OK;
}

}  // namespace gbk
