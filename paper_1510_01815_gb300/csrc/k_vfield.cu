// k_vfield.cu -- the velocity-field modelling strategy (Sec. 2.2.1): Eq. 8
// evaluated at every data pixel directly, with the arctan (Eq. 6) or the
// Epinat (Eq. 7) rotation curve, then the residuals and chi-squared of
// Eq. 11.  There is no cube and no PSF or LSF; m0 = 1 (every pixel valid)
// and m2 = sigma0, the constant dispersion model of Sec. 2.1.4.
//
// One CTA per model (grid-stride over models), consecutive pixels on
// consecutive threads (coalesced map reads and writes, as the paper's
// evaluation kernel does), Kahan sums per thread, FP32 warp sums and a
// fixed-order FP64 sum over the warps, so chi2 is bitwise reproducible.
#include "gbk_api_internal.h"
#include "k_fused.h"
#include "k_tangent.h"

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
            // each warp's sum in FP32 (a fixed shuffle tree), the warps in FP64
            float v = s - comp;
            for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
            if ((tid & 31) == 0) red[tid >> 5] = (double)v;
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

// ---------------------------------------------------------------------------
// Analytic Jacobian of the velocity-field residuals.  With F(r) = Vrot(r) / r,
// m1 = Vsys + F(r) x_e sin i and m2 = sigma0; by the chain rule through
// Eqs. 1-4 (angles in degrees):
//   d x_e = (sin PA, -cos PA, y_e k)  and  d y_e = (cos PA, sin PA, -x_e k)
//   for (x0, y0, PA), k = pi / 180;  d y_d = d y_e / cos i, and for the
//   inclination d y_d / di = y_d tan i k;  d r = (x_e dx_e + y_d dy_d) / r;
//   dm1 = sin i (F'(r) dr x_e + F dx_e) for (x0, y0, PA),
//   dm1/di = F x_e cos i k + sin i F'(r) dr_i x_e,  dm1/dVsys = 1,
//   dm1/dtheta = sin i x_e dF/dtheta for the curve's parameters;
//   arctan (Eq. 6, c = 2 Vmax / pi, u = r / r_t):
//     F' = c (u / (1 + u^2) - atan u) / r^2 (series for small u),
//     dF/dVmax = (2 / pi) atan(u) / r,  dF/dr_t = -c / (r_t^2 + r^2);
//   Epinat (Eq. 7, q = r / r_t, D = 1 + q^a):
//     F' = (F / r) ((g - 1) - a q^a / D),  dF/dV_t = q^g / (D r),
//     dF/dr_t = -(F / r_t) (g - a q^a / D),  dF/da = -F q^a ln q / D,
//     dF/dg = F ln q;
//   dm2/dsigma0 = 1.  At r = 0 the cusp of r gets the one-sided value 0 (and
//   the Epinat curve, whose F is 0 there, zero derivatives).  Rows are
//   J_v = w_v dm1, J_s = w_s dm2 on unmasked pixels.  Every thread keeps its
//   pixels' J^T J, J^T v and sum r^2 for all ten parameters in registers;
//   the CTA reduces them (FP32 within a warp, FP64 over the warps) in a
//   fixed order.
constexpr int kVfEnt = GBK_NPAR * (GBK_NPAR + 1) / 2 + GBK_NPAR + 1;

__global__ void __launch_bounds__(kVfThreads) vfield_tangent_kernel(TangentArgs a)
{
    __shared__ VfConst s_c;
    __shared__ gbk_obs s_ob;
    __shared__ float wred[kVfThreads / 32][kVfEnt];
    __shared__ double s_part[kVfEnt];
    const int tid = threadIdx.x;
    const int nx = a.g.nx, np = a.g.nx * a.g.ny;
    const int mpg = a.models_per_gal;
    const float kdeg = 0.017453292519943295f;
    for (int model = blockIdx.x; model < a.n_models; model += gridDim.x) {
        const int gal = mpg > 0 ? model / mpg : 0;
        if (a.skip && a.skip[gal] != 0) continue;
        if (tid == 0) {
            s_c = vf_const(a.params + (size_t)model * GBK_NPAR, a.g.model);
            s_ob = a.obs_list ? a.obs_list[gal] : a.obs;
        }
        __syncthreads();
        const VfConst c = s_c;
        const float si = c.sin_i, ci = 1.f / c.inv_cos_i, ti = si * c.inv_cos_i;
        const float vmax = (float)a.params[(size_t)model * GBK_NPAR + GBK_VMAX];
        float E[kVfEnt];
#pragma unroll
        for (int e = 0; e < kVfEnt; ++e) E[e] = 0.f;
        for (int pix = tid; pix < np; pix += kVfThreads) {
            const int y = pix / nx, x = pix - y * nx;
            float dx = (float)x - c.x0, dy = (float)y - c.y0;
            float xe = -dx * c.sin_pa + dy * c.cos_pa;
            float ye = -dx * c.cos_pa - dy * c.sin_pa;
            float yd = ye * c.inv_cos_i;
            float r = sqrtf(xe * xe + yd * yd);
            float F, Fr, Fv, Frt, Fa = 0.f, Fg = 0.f;
            if (c.epinat) {
                if (r > 0.f) {
                    float q = r * c.inv_rt, lq = logf(q);
                    float qg = expf(c.g * lq), qa = expf(c.a * lq), D = 1.f + qa;
                    Fv = qg / (D * r);
                    F = c.vk * Fv;
                    float aq = c.a * qa / D;
                    Fr = F / r * ((c.g - 1.f) - aq);
                    Frt = -F * c.inv_rt * (c.g - aq);
                    Fa = -F * qa * lq / D;
                    Fg = F * lq;
                } else {
                    F = Fr = Fv = Frt = 0.f;
                }
            } else {
                float u = r * c.inv_rt, at = atanf(u);
                Fv = 0.63661977f * ((r > 0.f) ? at / r : c.inv_rt);
                F = vmax * Fv;
                if (r <= 0.f) Fr = 0.f;
                else if (u < 0.1f) Fr = c.vk * c.inv_rt * c.inv_rt * u * (-2.f / 3.f + 0.8f * u * u);
                else Fr = c.vk * (u / (1.f + u * u) - at) / (r * r);
                float rt = 1.f / c.inv_rt;
                Frt = -c.vk / (rt * rt + r * r);
            }
            float m1 = c.vsys + F * xe * si;
            float rx = 0.f, ry = 0.f, ri = 0.f;  // dr per unit dx_e, dy_e; dr/di
            if (r > 0.f) {
                rx = xe / r;
                ry = yd * c.inv_cos_i / r;
                ri = yd * yd * ti * kdeg / r;
            }
            float jv[GBK_NPAR], js[GBK_NPAR];
#pragma unroll
            for (int k = 0; k < GBK_NPAR; ++k) { jv[k] = 0.f; js[k] = 0.f; }
            float rv = 0.f, rs = 0.f, cv = 0.f, cs = 0.f;
            if (c.valid && s_ob.mask[pix] != 0) {
                const float wv = s_ob.w_v[pix], ws = s_ob.w_s[pix];
                const float dxe[3] = {c.sin_pa, -c.cos_pa, ye * kdeg};
                const float dye[3] = {c.cos_pa, c.sin_pa, -xe * kdeg};
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    float dr = rx * dxe[k] + ry * dye[k];
                    jv[k] = wv * si * (Fr * dr * xe + F * dxe[k]);
                }
                jv[GBK_INCL] = wv * (F * xe * ci * kdeg + si * Fr * ri * xe);
                jv[GBK_VSYS] = wv;
                jv[GBK_VMAX] = wv * si * xe * Fv;
                jv[GBK_RT] = wv * si * xe * Frt;
                jv[GBK_EPI_A] = wv * si * xe * Fa;
                jv[GBK_EPI_G] = wv * si * xe * Fg;
                js[GBK_SIG0] = ws;
                rv = wv * (m1 - s_ob.v_obs[pix]);
                rs = ws * (c.sig0 - s_ob.s_obs[pix]);
                if (a.cot) {
                    cv = a.cot[(size_t)model * 2 * np + pix];
                    cs = a.cot[(size_t)model * 2 * np + np + pix];
                } else {
                    cv = rv;
                    cs = rs;
                }
            }
            if (a.jac) {
                float *J = a.jac + (size_t)model * GBK_NPAR * 2 * np;
#pragma unroll
                for (int k = 0; k < GBK_NPAR; ++k) {
                    J[((size_t)k * 2) * np + pix] = jv[k];
                    J[((size_t)k * 2 + 1) * np + pix] = js[k];
                }
            }
            int e = 0;
#pragma unroll
            for (int j = 0; j < GBK_NPAR; ++j)
#pragma unroll
                for (int k = j; k < GBK_NPAR; ++k, ++e) E[e] = fmaf(jv[j], jv[k], fmaf(js[j], js[k], E[e]));
#pragma unroll
            for (int j = 0; j < GBK_NPAR; ++j, ++e) E[e] = fmaf(jv[j], cv, fmaf(js[j], cs, E[e]));
            E[e] = fmaf(rv, rv, fmaf(rs, rs, E[e]));
        }
        // CTA sum: each warp's in FP32 by a reduce-scatter, then the warps in
        // FP64 in order
        const int warp = tid >> 5, lane = tid & 31;
        warp_sum_scatter<kVfEnt>(E, lane, wred[warp]);
        __syncthreads();
        for (int e = tid; e < kVfEnt; e += kVfThreads) {
            double v = 0.0;
            for (int q = 0; q < kVfThreads / 32; ++q) v += (double)wred[q][e];
            s_part[e] = v;
        }
        __syncthreads();
        const int nf = a.np, ntri = nf * (nf + 1) / 2;
        if (tid < ntri + nf + 1) {
            int src, j = 0, k = 0;
            if (tid < ntri) {
                int t = tid;
                while (t >= nf - j) { t -= nf - j; ++j; }
                k = j + t;
                int p = a.free_idx[j], q = a.free_idx[k];
                if (p > q) { int w = p; p = q; q = w; }
                src = p * GBK_NPAR - p * (p - 1) / 2 + (q - p);
            } else if (tid < ntri + nf) {
                src = GBK_NPAR * (GBK_NPAR + 1) / 2 + a.free_idx[tid - ntri];
            } else {
                src = kVfEnt - 1;
            }
            double v = c.valid ? s_part[src] : (double)__int_as_float(0x7fc00000);
            if (tid < ntri) {
                if (a.jtj) {
                    a.jtj[(size_t)model * nf * nf + j * nf + k] = v;
                    a.jtj[(size_t)model * nf * nf + k * nf + j] = v;
                }
            } else if (tid < ntri + nf) {
                if (a.jtv) a.jtv[(size_t)model * nf + (tid - ntri)] = v;
            } else if (a.chi2) {
                a.chi2[model] = v;
            }
        }
        __syncthreads();  // s_c, s_ob, wred and s_part are rewritten by the next model
    }
}

gbk_status launch_vfield_tangent(const TangentArgs &a, cudaStream_t st)
{
    if (a.geoms) return fail(GBK_EUNSUPPORTED, "survey batches serve the intensity-cube model");
    if (a.np < 1 || a.np > GBK_NPAR) return fail(GBK_EINVAL, "velocity-field Jacobian: bad free-parameter count");
    if (a.n_models <= 0) return GBK_OK;
    int blocks = a.n_models < 152 * 8 ? a.n_models : 152 * 8;
    vfield_tangent_kernel<<<blocks, kVfThreads, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "velocity-field Jacobian launch");
    return GBK_OK;
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
