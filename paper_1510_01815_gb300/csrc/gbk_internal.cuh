// gbk_internal.cuh -- device-side pieces shared by the library's kernels.
//
// Model: Bekiaris et al. 2015, Sec. 2.1 (Eqs. 1-8).  Everything here runs on
// the GPU; the host side only validates arguments and launches.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gbk.h"

namespace gbk {

constexpr double kFwhmPerSigma = 2.3548200450309493;  // 2 sqrt(2 ln 2)
constexpr float kInvalidFraction = 1e-20f;            // m0 <= this * I0: invalid spectrum

// Line-sampling window of the fused evaluator, in u =
// alpha (v_e - v_los), the Gaussian being 2^(-u^2).  For a line centred in
// the band, channels with |u| > kUCut (beyond 7.06 sigma, below 2^-36 of the
// peak) are left out: the terms fall off geometrically beyond, so the dropped
// tails change the spectrum's sums by under 1e-9 of their values, far below
// their FP32 resolution (6e-8); a one-channel margin keeps the channel
// nearest the centre in the window for any width.  A line centred outside
// the band keeps every channel whose Gaussian is not an exact FP32 zero
// (|u| <= kUFlush): its in-band tail may be all the spaxel has, and whether
// that is above the invalid-spectrum threshold must not change.
constexpr float kUCut = 6.0f;
constexpr float kUFlush = 11.25f;  // beyond it ex2(-u^2) < 2^-126 flushes to +0
constexpr int kMaxRadius = 64;                        // largest kernel radius served

// Geometry after host-side derivation of kernel radii and sizes.
struct Geom {
    int nx, ny, nz;        // data cube
    int u;                 // upsampling factor
    int R, Rz;             // kernel radii on the (fine) model grid
    int nxf, nyf, nzf;     // fine data grid = u * (nx, ny, nz)
    int ex, ey, ez;        // fine extended grid
    float dv, vc;
    float sig_xy;          // PSF sigma, fine pixels
    float sig_z;           // LSF sigma, fine channels (mode 0)
    float sig_lsf_kms;     // LSF sigma, km/s (mode 1 folds it into the line)
    int lsf_mode;
    int model;             // GBK_MODEL_*
};

// Per-model constants, derived once per block.
struct ModelConst {
    float x0, y0, sin_pa, cos_pa, sin_i, inv_cos_i;
    float vsys, vrot_k;    // vrot_k = (2/pi) Vmax
    float inv_rt, i0, inv_h;
    float sigma;           // line sigma, km/s
    float amp;             // dv / (sigma sqrt(2 pi))
    float alpha;           // sqrt(log2 e) / (sigma sqrt 2): exp(-d^2/2s^2) = 2^-(alpha d)^2
    int valid;             // 0 if a parameter is outside its domain
};

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Packed FP32 pairs (f32x2): one instruction performs two lane operations,
// which halves the issue slots of the FP32 loops.
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 pk2(float lo, float hi)
{
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ void upk2(f32x2 v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c)
{
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ float hsum2(f32x2 v)
{
    float lo, hi;
    upk2(v, lo, hi);
    return lo + hi;
}

__device__ inline ModelConst model_const(const double *p, const Geom &g)
{
    ModelConst c;
    bool ok = (p[GBK_INCL] >= 0.0) && (p[GBK_INCL] < 90.0) && (p[GBK_RT] > 0.0) &&
              (p[GBK_SIG0] > 0.0) && (p[GBK_I0] > 0.0) && (p[GBK_H] > 0.0);
    for (int k = 0; k < GBK_NPAR; ++k) ok = ok && isfinite(p[k]);
    c.valid = ok ? 1 : 0;
    float s0 = (float)p[GBK_SIG0];
    float sig = s0;
    if (g.lsf_mode == 1) sig = sqrtf(s0 * s0 + g.sig_lsf_kms * g.sig_lsf_kms);
    float sp, cp, si, ci;
    // sin/cos of (degrees / 180) * pi with exact argument reduction.
    sincospif((float)(p[GBK_PA] * (1.0 / 180.0)), &sp, &cp);
    sincospif((float)(p[GBK_INCL] * (1.0 / 180.0)), &si, &ci);
    c.x0 = (float)p[GBK_X0];
    c.y0 = (float)p[GBK_Y0];
    c.sin_pa = sp;
    c.cos_pa = cp;
    c.sin_i = si;
    c.inv_cos_i = 1.0f / ci;
    c.vsys = (float)p[GBK_VSYS];
    c.vrot_k = (float)(0.63661977236758134 * p[GBK_VMAX]);
    c.inv_rt = 1.0f / (float)p[GBK_RT];
    c.i0 = (float)p[GBK_I0];
    c.inv_h = 1.0f / (float)p[GBK_H];
    c.sigma = sig;
    c.amp = g.dv / (sig * 2.5066282746310002f);
    c.alpha = 0.84932180028801904f / sig;  // sqrt(log2(e) / 2) / sigma
    return c;
}

// Line-of-sight velocity (Eq. 8) and surface brightness (Eq. 5) at sky
// position (x, y) in data pixels.  Vrot(r) cos(theta) is computed as
// [Vrot(r)/r] x_e (Eqs. 4, 6), whose r -> 0 limit is (2/pi) Vmax / r_t.
__device__ __forceinline__ void los(const ModelConst &c, float x, float y, float &v, float &bright)
{
    float dx = x - c.x0, dy = y - c.y0;
    float xe = -dx * c.sin_pa + dy * c.cos_pa;  // Eq. 1
    float ye = -dx * c.cos_pa - dy * c.sin_pa;  // Eq. 2
    float yd = ye * c.inv_cos_i;
    float r = sqrtf(xe * xe + yd * yd);         // Eq. 3
    float f = (r > 0.f) ? c.vrot_k * atanf(r * c.inv_rt) / r : c.vrot_k * c.inv_rt;
    v = c.vsys + f * xe * c.sin_i;              // Eq. 8
    bright = c.i0 * expf(-r * c.inv_h);         // Eq. 5
}

// Unnormalised Gaussian tap exp(-j^2 / (2 sigma^2)) (sigma > 0).
__device__ __forceinline__ float gauss_tap(int j, float sigma)
{
    float t = (float)j / sigma;
    return expf(-0.5f * t * t);
}

// Block-wide: taps w[0..2R] = normalised Gaussian of width sigma.  `scratch`
// holds at least 2R+1 floats.  Must be called by every thread of the block;
// ends with __syncthreads().
__device__ inline void block_taps(float sigma, int R, float *w)
{
    for (int j = threadIdx.x; j <= 2 * R; j += blockDim.x)
        w[j] = (R == 0) ? 1.f : gauss_tap(j - R, sigma);
    __syncthreads();
    __shared__ float s_norm;
    if (threadIdx.x == 0) {
        float s = 0.f;
        for (int j = 0; j <= 2 * R; ++j) s += w[j];
        s_norm = 1.f / s;
    }
    __syncthreads();
    for (int j = threadIdx.x; j <= 2 * R; j += blockDim.x) w[j] *= s_norm;
    __syncthreads();
}

// Warp reduce-scatter of N per-lane FP32 values: at each of five levels a
// lane keeps one half of its values and receives the partner's copy of that
// half (shuffle distance 16, 8, .., 1), so every sum over the 32 lanes ends
// on one lane after about N shuffles instead of 5 N.  Afterwards a[0..cnt)
// hold the warp sums of entries base .. base + cnt - 1; the tree is fixed,
// so the result does not depend on timing.  Whole warps.
template <int N, int OFF>
struct WarpScatter {
    static constexpr int M = (N + 1) / 2;  // values kept at this level
    static constexpr int MF = WarpScatter<M, OFF / 2>::MF;
    __device__ __forceinline__ static void run(float *a, int lane, int &base, int &cnt)
    {
        const bool hi = (lane & OFF) != 0;
#pragma unroll
        for (int i = 0; i < M; ++i) {
            const float lo = a[i], up = (i + M < N) ? a[i + M] : 0.f;
            const float keep = hi ? up : lo, send = hi ? lo : up;
            a[i] = keep + __shfl_xor_sync(0xffffffffu, send, OFF);
        }
        if (hi) {
            base += M;
            cnt -= M;
        }
        cnt = cnt < 0 ? 0 : (cnt > M ? M : cnt);
        WarpScatter<M, OFF / 2>::run(a, lane, base, cnt);
    }
};
template <int N>
struct WarpScatter<N, 0> {
    static constexpr int MF = N;
    __device__ __forceinline__ static void run(float *, int, int &, int &) {}
};

// Sums N values per lane over the warp into red[0..N) (one slot per entry,
// written once by the lane that ends with it).  a[] is clobbered.
template <int N>
__device__ __forceinline__ void warp_sum_scatter(float (&a)[N], int lane, float *red)
{
    int base = 0, cnt = N;
    WarpScatter<N, 16>::run(a, lane, base, cnt);
#pragma unroll
    for (int i = 0; i < WarpScatter<N, 16>::MF; ++i)
        if (i < cnt) red[base + i] = a[i];
}

}  // namespace gbk
