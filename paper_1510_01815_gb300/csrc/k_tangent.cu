// k_tangent.cu -- analytic Jacobian of the residual maps (forward-mode
// derivatives through the whole forward model of Sec. 2.1-2.2.6).
//
// For a spaxel with line centre v, brightness I and line width sigma the
// model cube is c_e = A g_e, A = I dv / (sigma sqrt(2 pi)),
// g_e = exp(-d_e^2 / 2 sigma^2), d_e = v_e - v.  For any parameter theta
//   dc_e/dtheta = c_e [ dlnA/dtheta + d_e/sigma^2 dv/dtheta + d_e^2/sigma^3 dsigma/dtheta ],
// so the derivatives of the spaxel's moment sums q_m = sum_e c_e T_m(e) (the
// z-folded weights of the fused kernel, taken about a fixed centre a) are
//   dq_m = A [ dlnA B_0m + dv/sigma^2 B_1m + dsigma/sigma^3 B_2m ],
//   B_km = sum_e g_e d_e^k T_m(e),  k, m = 0..2.
// The channel loop accumulates the twelve sums needed for the nine B_km
// (powers 0..4 of d against the LSF tap moments G0, H1, H2 of each channel);
// the geometry supplies dv, dlnI and dsigma per spaxel by the chain rule
// through Eqs. 1-8.  The PSF passes are linear, so the derivative triplets go
// through the same re-centred x and y passes as the values; the moments'
// quotient rule then gives dm1, dm2 and the Jacobian rows
// J_v = w_v dm1, J_s = w_s dm2 of the residual maps.  Per model the kernel
// reduces J^T J and J^T v (v = the residuals, or a caller's cotangent maps)
// in a fixed order and can also write J itself.
//
// Where a parameter's derivative is not defined -- the brightness cusp at
// r = 0 -- the one-sided value 0 is used for dr.  The centre a is held fixed
// (the moments do not depend on it).  Sums are taken about the line centre
// and shifted to a afterwards; that is exact algebra, and the small FP32
// cancellation it allows for lines far outside the band only affects the
// Jacobian (chi2 values for LM decisions come from the fused kernel).
#include <cooperative_groups.h>

#include "fused_line.cuh"
#include "gbk_api_internal.h"
#include "gbk_internal.cuh"
#include "k_tangent.h"

namespace cg = cooperative_groups;

namespace gbk {

// NP = derivatives carried: every parameter (GBK_NPAR), or the first eight
// (x0 .. sigma0) when I0 and h are held fixed, as in every fit of the paper.
// A spaxel record holds kTrip = NP + 1 moment triplets (x0, x1, x2) -- the
// values (triplet 0) and the NP derivatives -- and the centre a.  Triplets
// 2q and 2q + 1 are packed as pairs, (x0, x0'), (x1, x1'), (x2, x2') at
// floats 6q .. 6q + 5, so the spatial passes treat two triplets per packed
// f32x2 operation; an odd last triplet follows unpaired, then a.
template <int NP>
struct TgDims {
    static constexpr int kTrip = NP + 1;
    static constexpr int kPairs = kTrip / 2;
    static constexpr int kSingle = 6 * kPairs;               // the unpaired triplet
    static constexpr int kA = kSingle + 3 * (kTrip & 1);     // the centre a
    static constexpr int kRec = kA + 1;                      // floats per record
    // record stride in floats, 2 mod 4: records start 8-byte aligned and a
    // half-warp's 8-byte loads of consecutive records fall on distinct banks
    static constexpr int RS = ((kRec + 1) & ~3) + 2;
    static constexpr int kTri = NP * (NP + 1) / 2;
    static constexpr int kEnt = kTri + NP + 1;  // J^T J upper triangle, J^T v, sum r^2
    // float offset of component m of triplet t
    __host__ __device__ static constexpr int off(int t, int m)
    {
        return t < 2 * kPairs ? 6 * (t >> 1) + 2 * m + (t & 1) : kSingle + m;
    }
};

__host__ __device__ inline int tg_band_begin(int rank, int ey, int cs) { return (int)(((long)rank * ey) / cs); }
__device__ inline int tg_band_owner(int er, int ey, int cs) { return (int)((((long)er + 1) * cs - 1) / ey); }

// Shared memory of one CTA.  direct = 0: the y pass reads the 2R halo rows
// from copies in Q (Q holds the larger of the band's extended records and
// the halo rows); direct = 1: it reads them in the neighbours' P through
// distributed shared memory and Q holds the band's extended records only.
// Records are rs floats; Q and P start on 16-byte boundaries.
__host__ __device__ inline size_t tg_align4(size_t f) { return (f + 3) & ~(size_t)3; }

__host__ __device__ inline size_t tangent_smem_bytes_np(const Geom &g, int band, int threads, int rs, int direct)
{
    size_t q = (size_t)band * g.ex, h = direct ? 0 : (size_t)2 * g.R * g.nx;
    size_t b = tg_align4((q > h ? q : h) * rs) * 4;       // Q records / halo rows
    b += tg_align4((size_t)band * g.nx * rs) * 4;          // P records
    b += (size_t)(g.ez + 2) * 16;                         // per-channel G0, H1, H2 (three padded arrays)
    b += (size_t)((2 * g.R + 1 + 3) & ~3) * 4;            // PSF taps
    b += (size_t)((band + 2 * g.R + 1) & ~1) * 8;         // y-pass row pointers
    b += (size_t)TgDims<GBK_NPAR>::kEnt * (threads / 32) * 8;  // per-warp reduction slots
    return b;
}

// The size of a launch carrying eight (narrow) or ten derivatives.
__host__ __device__ inline size_t tangent_smem_bytes(const Geom &g, int band, int threads, int direct, bool narrow)
{
    return tangent_smem_bytes_np(g, band, threads, narrow ? TgDims<GBK_I0>::RS : TgDims<GBK_NPAR>::RS, direct);
}

size_t tangent_smem_bytes_host(const Geom &g, int band, int threads, int direct, bool narrow)
{
    return tangent_smem_bytes(g, band, threads, direct, narrow);
}

// Accumulated triplets of one output spaxel, in the record's pairing.
template <int NP>
struct TgAcc {
    f32x2 p[3 * TgDims<NP>::kPairs];  // pair q: x0, x1, x2 of triplets 2q, 2q + 1
    float s[3];                       // the unpaired triplet
    __device__ __forceinline__ void zero()
    {
#pragma unroll
        for (int i = 0; i < 3 * TgDims<NP>::kPairs; ++i) p[i] = pk2(0.f, 0.f);
        s[0] = s[1] = s[2] = 0.f;
    }
    // component m of triplet t
    __device__ __forceinline__ float get(int t, int m) const
    {
        if (t < 2 * TgDims<NP>::kPairs) {
            float lo, hi;
            upk2(p[3 * (t >> 1) + m], lo, hi);
            return (t & 1) ? hi : lo;
        }
        return s[m];
    }
    // the accumulated triplets and the centre c as a record at out
    __device__ __forceinline__ void store(float *out, float c) const
    {
#pragma unroll
        for (int i = 0; i < 3 * TgDims<NP>::kPairs; ++i) *reinterpret_cast<f32x2 *>(out + 2 * i) = p[i];
        if (TgDims<NP>::kTrip & 1) {
            out[TgDims<NP>::kSingle] = s[0];
            out[TgDims<NP>::kSingle + 1] = s[1];
            out[TgDims<NP>::kSingle + 2] = s[2];
        }
        out[TgDims<NP>::kA] = c;
    }
};

// Re-centres the record at rec (centre a at rec[kA]) to centre c and adds it
// with weight w: x0 += w x0, x1 += w (x1 + D x0), x2 += w (x2 + D (2 x1 +
// D x0)), D = a - c, two triplets per packed operation.
template <int NP>
__device__ __forceinline__ void accum_rec(const float *rec, float c, float w, TgAcc<NP> &acc)
{
    using Dm = TgDims<NP>;
    const float D = rec[Dm::kA] - c;
    const f32x2 W = pk2(w, w), DD = pk2(D, D);
#pragma unroll
    for (int q = 0; q < Dm::kPairs; ++q) {
        const f32x2 X0 = *reinterpret_cast<const f32x2 *>(rec + 6 * q);
        const f32x2 X1 = *reinterpret_cast<const f32x2 *>(rec + 6 * q + 2);
        const f32x2 X2 = *reinterpret_cast<const f32x2 *>(rec + 6 * q + 4);
        const f32x2 T0 = mul2(W, X0), T1 = mul2(W, X1);
        acc.p[3 * q] = add2(acc.p[3 * q], T0);
        acc.p[3 * q + 1] = add2(acc.p[3 * q + 1], fma2(DD, T0, T1));
        acc.p[3 * q + 2] = add2(acc.p[3 * q + 2], fma2(W, X2, mul2(DD, fma2(DD, T0, add2(T1, T1)))));
    }
    if (Dm::kTrip & 1) {
        const float x0 = rec[Dm::kSingle], x1 = rec[Dm::kSingle + 1], x2 = rec[Dm::kSingle + 2];
        const float t0 = w * x0, t1 = w * x1;
        acc.s[0] += t0;
        acc.s[1] += fmaf(D, t0, t1);
        acc.s[2] += fmaf(w, x2, D * fmaf(D, t0, 2.f * t1));
    }
}

// The eight-derivative build fits 128 registers without spills, so two
// CTAs share an SM when their shared memory allows; the ten-derivative
// build keeps one.
template <int NP>
__global__ void __launch_bounds__(kTangentThreads, NP == GBK_I0 ? 2 : 1) tangent_kernel(TangentArgs a)
{
    constexpr int NPT = NP;
    constexpr int kEnt = TgDims<NP>::kEnt;
    constexpr int RS = TgDims<NP>::RS;  // record stride (2 mod 4)
    cg::cluster_group cluster = cg::this_cluster();
    const int cs = a.cs;
    const int rank = (int)cluster.block_rank();
    const int w = blockIdx.x / cs;
    // ragged batches: one model per galaxy, geometry from the table
    const int model = a.geoms ? (a.order ? a.order[w] : w) : w;
    const Geom g = a.geoms ? a.geoms[model] : a.g;
    const int band = a.geoms ? (g.ey + cs - 1) / cs : a.band;
    const int row0 = tg_band_begin(rank, g.ey, cs), row1 = tg_band_begin(rank + 1, g.ey, cs);
    const int nrows = row1 - row0;
    const int R = g.R;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int gal = a.geoms ? model : (a.models_per_gal > 0 ? model / a.models_per_gal : 0);
    if (a.skip && a.skip[gal] != 0) return;  // the whole cluster returns together

    extern __shared__ __align__(16) unsigned char smem[];
    size_t qn = (size_t)band * g.ex, hn = a.direct ? 0 : (size_t)2 * R * g.nx;
    float *Q = reinterpret_cast<float *>(smem);                        // records, stride RS
    float *P = Q + tg_align4((qn > hn ? qn : hn) * RS);
    // per-channel LSF tap moments, three arrays of ezp (even) floats so that
    // (channel e, e + 1) pairs load as one aligned 8-byte word
    const int ezp = (g.ez + 1) & ~1;
    float *tzx = P + tg_align4((size_t)band * g.nx * RS);
    float *tzy = tzx + ezp, *tzz = tzy + ezp;
    float *wxy = tzx + ((3 * ezp + 3) & ~3);
    const float **rowptr = reinterpret_cast<const float **>(wxy + ((2 * R + 1 + 3) & ~3));
    float *wred = reinterpret_cast<float *>(rowptr + ((band + 2 * R + 1) & ~1));  // [warps][kEnt]

    __shared__ ModelConst mc;
    __shared__ gbk_obs s_ob;
    __shared__ float s_norm_xy, s_norm_z;
    __shared__ double s_part[TgDims<GBK_NPAR>::kEnt];

    if (tid == 0) {
        mc = model_const(a.params + (size_t)model * GBK_NPAR, g);
        s_ob = a.obs_list ? a.obs_list[gal] : a.obs;
        float sx = 0.f, sz = 0.f;
        for (int j = -R; j <= R; ++j) sx += (R == 0) ? 1.f : gauss_tap(j, g.sig_xy);
        for (int j = -g.Rz; j <= g.Rz; ++j) sz += (g.Rz == 0) ? 1.f : gauss_tap(j, g.sig_z);
        s_norm_xy = 1.f / sx;
        s_norm_z = 1.f / sz;
    }
    __syncthreads();
    for (int j = tid; j <= 2 * R; j += nthr) wxy[j] = ((R == 0) ? 1.f : gauss_tap(j - R, g.sig_xy)) * s_norm_xy;
    for (int e = tid; e < g.ez; e += nthr) {
        int kd = e - g.Rz;
        int jlo = max(0, kd - g.Rz) - kd, jhi = min(g.nz - 1, kd + g.Rz) - kd;
        float G0 = 0.f, H1 = 0.f, H2 = 0.f;
        for (int j = jlo; j <= jhi; ++j) {
            float w = ((g.Rz == 0) ? 1.f : gauss_tap(j, g.sig_z)) * s_norm_z;
            G0 += w;
            H1 = fmaf(w, (float)j, H1);
            H2 = fmaf(w, (float)(j * j), H2);
        }
        tzx[e] = G0;
        tzy[e] = g.dv * H1;
        tzz[e] = g.dv * g.dv * H2;
        if (e + 1 == g.ez && g.ez < ezp) tzx[e + 1] = tzy[e + 1] = tzz[e + 1] = 0.f;  // pad of an odd ez
    }
    // first record of extended row row0 - R + k for the y pass: own rows in
    // P; halo rows in their copies in Q, or (direct) in the owner's P
    for (int k = tid; k < nrows + 2 * R; k += nthr) {
        int er = row0 - R + k;
        const float *ptr;
        if (er >= row0 && er < row1) ptr = P + (size_t)(er - row0) * g.nx * RS;
        else if (!a.direct) ptr = Q + (size_t)(er < row0 ? k : R + (er - row1)) * g.nx * RS;
        else if (er < 0 || er >= g.ey) ptr = nullptr;  // never read: outside the image
        else {
            int owner = tg_band_owner(er, g.ey, cs);
            ptr = cluster.map_shared_rank(P, owner) + (size_t)(er - tg_band_begin(owner, g.ey, cs)) * g.nx * RS;
        }
        rowptr[k] = ptr;
    }
    __syncthreads();
    const ModelConst &c = mc;

    // ---- phase 1: records (a, q, dq) of the band's extended spaxels ----
    const float kdeg = 0.017453292519943295f;  // radians per degree
    const float vz0 = g.vc - ((float)g.Rz + 0.5f * (float)(g.nz - 1)) * g.dv;
    const float v_lo = g.vc - 0.5f * (float)(g.nz - 1) * g.dv, v_hi = g.vc + 0.5f * (float)(g.nz - 1) * g.dv;
    const int elo = edge_lo_end(g), ehi = edge_hi_begin(g);  // the band's interior channels
    const float var_z = lsf_var(g);                          // and the LSF variance there
    const float sig = c.sigma, isig2 = 1.f / (sig * sig), isig3 = isig2 / sig;
    const float s0p = (float)a.params[(size_t)model * GBK_NPAR + GBK_SIG0];
    const float dsig_ds0 = (g.lsf_mode == 1) ? s0p / sig : 1.f;
    const float vmax = (float)a.params[(size_t)model * GBK_NPAR + GBK_VMAX];
    const float rtv = (float)a.params[(size_t)model * GBK_NPAR + GBK_RT];
    const float hv = (float)a.params[(size_t)model * GBK_NPAR + GBK_H];
    const float ci = 1.f / c.inv_cos_i;
    for (int idx = tid; idx < nrows * g.ex; idx += nthr) {
        int rr = idx / g.ex, xe_i = idx - rr * g.ex;
        float x = (float)(xe_i - R), y = (float)(row0 + rr - R);
        // geometry and its derivatives (Eqs. 1-8)
        float dx = x - c.x0, dy = y - c.y0;
        float xe = -dx * c.sin_pa + dy * c.cos_pa;
        float ye = -dx * c.cos_pa - dy * c.sin_pa;
        float yd = ye * c.inv_cos_i;
        float r = sqrtf(xe * xe + yd * yd);
        float u = r * c.inv_rt;
        float at = atanf(u);
        float fv = (r > 0.f) ? 0.63661977f * at / r : 0.63661977f * c.inv_rt;  // f / Vmax
        float f = vmax * fv;
        float w = xe * c.sin_i;
        float vl = c.vsys + f * w;
        float br = c.i0 * expf(-r * c.inv_h);
        float fp;  // df/dr
        if (u < 0.1f) fp = vmax * 0.63661977f * c.inv_rt * c.inv_rt * u * (-2.f / 3.f + 0.8f * u * u);
        else fp = vmax * 0.63661977f * (u / (1.f + u * u) - at) / (r * r);
        float rx = 0.f, ry = 0.f, ri = 0.f;
        if (r > 0.f) {
            rx = xe / r;
            ry = ye * c.inv_cos_i * c.inv_cos_i / r;
            ri = yd * yd * (c.sin_i * c.inv_cos_i) / r * kdeg;
        }
        float dxe[3] = {c.sin_pa, -c.cos_pa, ye * kdeg};   // d x_e / d(x0, y0, PA)
        float dye[3] = {c.cos_pa, c.sin_pa, -xe * kdeg};   // d y_e / d(x0, y0, PA)
        float dv[NPT], dlnA[NPT];
#pragma unroll
        for (int k = 0; k < NPT; ++k) { dv[k] = 0.f; dlnA[k] = 0.f; }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float drk = rx * dxe[k] + ry * dye[k];
            dv[k] = f * c.sin_i * dxe[k] + fp * drk * w;
            dlnA[k] = -drk * c.inv_h;
        }
        dv[GBK_INCL] = kdeg * f * xe * ci + fp * ri * w;
        dlnA[GBK_INCL] = -ri * c.inv_h;
        dv[GBK_VSYS] = 1.f;
        dv[GBK_VMAX] = fv * w;
        dv[GBK_RT] = -0.63661977f * vmax / (rtv * rtv + r * r) * w;
        dlnA[GBK_SIG0] = -dsig_ds0 / sig;
        if constexpr (NP > GBK_I0) dlnA[GBK_I0] = 1.f / c.i0;
        if constexpr (NP > GBK_H) dlnA[GBK_H] = r / (hv * hv);
        (void)hv;
        // channel sums: S_k^G = sum g d^k G0 (k <= 4), S_k^1 = sum g d^k H1 (k <= 3), S_k^2 = sum g d^k H2 (k <= 2)
        float a_c = fminf(fmaxf(vl, v_lo), v_hi);
        float sh = vl - a_c;
        float base = vz0 - vl;
        // The warp's channel window: the union of its lanes' |u| <= cut (the
        // evaluators' rule: beyond it the Gaussian is below 2^-36 of its
        // peak, or flushed to zero for a line centred outside the band), in
        // whole channel pairs.
        int e0, e1;
        {
            const unsigned am = __activemask();
            const float cut = (sh != 0.f) ? kUFlush : kUCut;
            const float inv_adv = 1.f / (c.alpha * g.dv);
            float flo = (-cut - c.alpha * base) * inv_adv - 1.f, fhi = (cut - c.alpha * base) * inv_adv + 2.f;
            if (!(flo > -1e6f)) flo = -1e6f;
            if (!(fhi < 1e6f)) fhi = 1e6f;
            e0 = __reduce_min_sync(am, (int)floorf(flo));
            e1 = __reduce_max_sync(am, (int)ceilf(fhi));
            e0 = max(0, e0) & ~1;
            e1 = min(ezp, (e1 + 1) & ~1);
        }
        // Channels in pairs (e, e + 1) on packed FP32 lanes: per pair one
        // argument, two ex2, the powers of d as a shallow tree and twelve
        // packed accumulations; an odd last channel pairs with the padding,
        // whose tap moments are 0.  The two lanes are added at the end.
        // Interior channels (the LSF window inside the band: G0 = 1, H1 = 0,
        // H2 = the LSF variance) need no table and only the sums of g d^k;
        // the segments keep whole pairs inside [elo, ehi), the edge loops
        // take the rest (their tables hold every channel).
        float SG[5], S1[4], S2[3];
        {
            const f32x2 Z2 = pk2(0.f, 0.f), AL = pk2(c.alpha, c.alpha), DV = pk2(g.dv, g.dv);
            const f32x2 BASE = pk2(base, base), TWO = pk2(2.f, 2.f);
            f32x2 A0 = Z2, A1 = Z2, A2 = Z2, A3 = Z2, A4 = Z2, B0 = Z2, B1 = Z2, B2 = Z2, B3 = Z2, C0 = Z2, C1 = Z2,
                  C2 = Z2;
            f32x2 I0 = Z2, I1 = Z2, I2 = Z2, I3 = Z2, I4 = Z2;
            const int eil = max(e0, min(e1, (elo + 1) & ~1)), eih = max(eil, min(e1, ehi & ~1));
            f32x2 FE = pk2((float)e0, (float)(e0 + 1));
            auto edge_pair = [&](int e) {
                const f32x2 D = fma2(FE, DV, BASE);
                const f32x2 T = mul2(D, AL);
                const f32x2 W = mul2(T, T);
                float w0, w1;
                upk2(W, w0, w1);
                const f32x2 G0 = pk2(ex2_approx(-w0), ex2_approx(-w1));
                const f32x2 D2 = mul2(D, D);
                const f32x2 G1 = mul2(G0, D), G2 = mul2(G0, D2);
                const f32x2 G3 = mul2(G1, D2), G4 = mul2(G2, D2);
                const f32x2 TX = *reinterpret_cast<const f32x2 *>(tzx + e);
                const f32x2 TY = *reinterpret_cast<const f32x2 *>(tzy + e);
                const f32x2 TZ = *reinterpret_cast<const f32x2 *>(tzz + e);
                A0 = fma2(G0, TX, A0); A1 = fma2(G1, TX, A1); A2 = fma2(G2, TX, A2);
                A3 = fma2(G3, TX, A3); A4 = fma2(G4, TX, A4);
                B0 = fma2(G0, TY, B0); B1 = fma2(G1, TY, B1); B2 = fma2(G2, TY, B2); B3 = fma2(G3, TY, B3);
                C0 = fma2(G0, TZ, C0); C1 = fma2(G1, TZ, C1); C2 = fma2(G2, TZ, C2);
                FE = add2(FE, TWO);
            };
            int e = e0;
            for (; e < eil; e += 2) edge_pair(e);
#pragma unroll 2
            for (; e < eih; e += 2) {
                const f32x2 D = fma2(FE, DV, BASE);
                const f32x2 T = mul2(D, AL);
                const f32x2 W = mul2(T, T);
                float w0, w1;
                upk2(W, w0, w1);
                const f32x2 G0 = pk2(ex2_approx(-w0), ex2_approx(-w1));
                const f32x2 D2 = mul2(D, D);
                const f32x2 G1 = mul2(G0, D), G2 = mul2(G0, D2);
                I0 = add2(I0, G0); I1 = add2(I1, G1); I2 = add2(I2, G2);
                I3 = fma2(G1, D2, I3); I4 = fma2(G2, D2, I4);
                FE = add2(FE, TWO);
            }
            for (; e < e1; e += 2) edge_pair(e);
            const float i0 = hsum2(I0), i1 = hsum2(I1), i2 = hsum2(I2);
            SG[0] = hsum2(A0) + i0; SG[1] = hsum2(A1) + i1; SG[2] = hsum2(A2) + i2;
            SG[3] = hsum2(A3) + hsum2(I3); SG[4] = hsum2(A4) + hsum2(I4);
            S1[0] = hsum2(B0); S1[1] = hsum2(B1); S1[2] = hsum2(B2); S1[3] = hsum2(B3);
            S2[0] = fmaf(var_z, i0, hsum2(C0)); S2[1] = fmaf(var_z, i1, hsum2(C1));
            S2[2] = fmaf(var_z, i2, hsum2(C2));
        }
        // B_km (k: power of d from the derivative; m: moment weight about a)
        float B[3][3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            B[k][0] = SG[k];
            B[k][1] = SG[k + 1] + sh * SG[k] + S1[k];
            B[k][2] = SG[k + 2] + 2.f * sh * SG[k + 1] + 2.f * S1[k + 1] + sh * sh * SG[k] + 2.f * sh * S1[k] + S2[k];
        }
        float A = c.amp * br;
        float *rec = Q + (size_t)idx * RS;
        rec[TgDims<NP>::kA] = a_c;
        rec[TgDims<NP>::off(0, 0)] = A * B[0][0];
        rec[TgDims<NP>::off(0, 1)] = A * B[0][1];
        rec[TgDims<NP>::off(0, 2)] = A * B[0][2];
#pragma unroll
        for (int k = 0; k < NPT; ++k) {
            float ds = (k == GBK_SIG0) ? dsig_ds0 : 0.f;
            float cA = dlnA[k], cv = dv[k] * isig2, cs3 = ds * isig3;
#pragma unroll
            for (int m = 0; m < 3; ++m)
                rec[TgDims<NP>::off(k + 1, m)] = A * (cA * B[0][m] + cv * B[1][m] + cs3 * B[2][m]);
        }
    }
    __syncthreads();

    // ---- phase 2: x pass on every triplet ----
    for (int idx = tid; idx < nrows * g.nx; idx += nthr) {
        int rr = idx / g.nx, xx = idx - rr * g.nx;
        const float *row = Q + ((size_t)rr * g.ex + xx) * RS;
        float cen = row[(size_t)R * RS + TgDims<NP>::kA];
        TgAcc<NP> acc;
        acc.zero();
        for (int j = 0; j <= 2 * R; ++j) accum_rec<NP>(row + (size_t)j * RS, cen, wxy[j], acc);
        acc.store(P + (size_t)idx * RS, cen);
    }
    cluster.sync();

    // ---- phase 3a: halo records from the neighbours (copy mode) ----
    for (int k = 0; k < 2 * R && !a.direct; ++k) {
        int er = (k < R) ? row0 - R + k : row1 + (k - R);
        if (er < 0 || er >= g.ey) continue;
        int owner = tg_band_owner(er, g.ey, cs);
        const float *src = cluster.map_shared_rank(P, owner) + (size_t)(er - tg_band_begin(owner, g.ey, cs)) * g.nx * RS;
        float *dst = Q + (size_t)k * g.nx * RS;
        for (int i = tid; i < g.nx * RS; i += nthr) dst[i] = src[i];
    }
    __syncthreads();

    // ---- phase 3b: y pass, moments, Jacobian rows; J^T J, J^T v and
    // sum r^2 accumulated per thread, then reduced in a fixed order ----
    const int ylo = max(row0 - R, 0), yhi = min(row1 - R, g.ny);
    const int nout = max(0, yhi - ylo) * g.nx;
    const size_t np = (size_t)g.nx * g.ny;
    const float thr = kInvalidFraction * c.i0;
    float E[kEnt];
#pragma unroll
    for (int e = 0; e < kEnt; ++e) E[e] = 0.f;
    for (int idx = tid; idx < nout; idx += nthr) {
        float jv[NPT], js[NPT], rv = 0.f, rs = 0.f, cv_ = 0.f, cs_ = 0.f;
#pragma unroll
        for (int k = 0; k < NPT; ++k) { jv[k] = 0.f; js[k] = 0.f; }
        int yy = idx / g.nx, xx = idx - yy * g.nx;
        int y = ylo + yy;
        size_t pix = (size_t)y * g.nx + xx;
        int k0 = y - (row0 - R);
        float cen = rowptr[k0 + R][(size_t)xx * RS + TgDims<NP>::kA];
        TgAcc<NP> acc;
        acc.zero();
        for (int j = 0; j <= 2 * R; ++j) accum_rec<NP>(rowptr[k0 + j] + (size_t)xx * RS, cen, wxy[j], acc);
        float S0 = acc.get(0, 0), S1v = acc.get(0, 1), S2v = acc.get(0, 2);
        bool use = c.valid && S0 > thr && s_ob.mask[pix] != 0;
        if (use) {
            float inv = 1.f / S0;
            float mu = S1v * inv;
            float var = fmaxf(fmaf(-mu, mu, S2v * inv), 0.f);
            float m2 = sqrtf(var);
            float wv = s_ob.w_v[pix], ws = s_ob.w_s[pix];
            rv = wv * (cen + mu - s_ob.v_obs[pix]);
            rs = ws * (m2 - s_ob.s_obs[pix]);
            float inv2m2 = m2 > 0.f ? 0.5f / m2 : 0.f;
#pragma unroll
            for (int k = 0; k < NPT; ++k) {
                float d0 = acc.get(k + 1, 0), d1 = acc.get(k + 1, 1), d2 = acc.get(k + 1, 2);
                float dmu = (d1 - mu * d0) * inv;
                float dvar = (d2 - S2v * inv * d0) * inv - 2.f * mu * dmu;
                jv[k] = wv * dmu;
                js[k] = ws * dvar * inv2m2;
            }
            if (a.cot) {
                cv_ = a.cot[(size_t)model * 2 * np + pix];
                cs_ = a.cot[(size_t)model * 2 * np + np + pix];
            } else {
                cv_ = rv;
                cs_ = rs;
            }
        }
        if (a.jac) {
            float *J = a.jac + (size_t)model * GBK_NPAR * 2 * np;
#pragma unroll
            for (int k = 0; k < GBK_NPAR; ++k) {
                J[((size_t)k * 2) * np + pix] = k < NPT ? jv[k < NPT ? k : 0] : 0.f;
                J[((size_t)k * 2 + 1) * np + pix] = k < NPT ? js[k < NPT ? k : 0] : 0.f;
            }
        }
        // both rows (velocity and dispersion) of this spaxel
        int e = 0;
#pragma unroll
        for (int j = 0; j < NPT; ++j)
#pragma unroll
            for (int k = j; k < NPT; ++k, ++e) E[e] = fmaf(jv[j], jv[k], fmaf(js[j], js[k], E[e]));
#pragma unroll
        for (int j = 0; j < NPT; ++j, ++e) E[e] = fmaf(jv[j], cv_, fmaf(js[j], cs_, E[e]));
        E[e] = fmaf(rv, rv, fmaf(rs, rs, E[e]));
    }
    // CTA sum: each warp's in FP32 by a reduce-scatter, then the warps in
    // FP64 in order
    {
        const int warp = tid >> 5, lane = tid & 31, nw = nthr >> 5;
        warp_sum_scatter<kEnt>(E, lane, wred + warp * kEnt);
        __syncthreads();
        for (int e = tid; e < kEnt; e += nthr) {
            double v = 0.0;
            for (int q = 0; q < nw; ++q) v += (double)wred[q * kEnt + e];
            s_part[e] = v;
        }
    }
    cluster.sync();
    // entry t of the free-parameter output: (j, k) of the upper triangle of
    // J^T J, then J^T v, then sum r^2, gathered from the carried entries
    const int nf = a.np;
    const int nent = nf * (nf + 1) / 2 + nf + 1;
    if (rank == 0 && tid < nent) {
        int ntri = nf * (nf + 1) / 2;
        int src, j = 0, k = 0;
        if (tid < ntri) {
            int t = tid;
            while (t >= nf - j) { t -= nf - j; ++j; }
            k = j + t;
            int p = a.free_idx[j], q = a.free_idx[k];
            if (p > q) { int x = p; p = q; q = x; }
            src = p * NPT - p * (p - 1) / 2 + (q - p);
        } else if (tid < ntri + nf) {
            src = TgDims<NP>::kTri + a.free_idx[tid - ntri];
        } else {
            src = kEnt - 1;
        }
        double s = 0.0;
        for (int q = 0; q < cs; ++q) {
            const double *p = (q == 0) ? s_part : cluster.map_shared_rank(s_part, q);
            s += p[src];
        }
        if (!c.valid) s = (double)__int_as_float(0x7fc00000);
        if (tid < ntri) {
            if (a.jtj) {
                a.jtj[(size_t)model * nf * nf + j * nf + k] = s;
                a.jtj[(size_t)model * nf * nf + k * nf + j] = s;
            }
        } else if (tid < ntri + nf) {
            if (a.jtv) a.jtv[(size_t)model * nf + (tid - ntri)] = s;
        } else {
            if (a.chi2) a.chi2[model] = s;
        }
    }
    cluster.sync();
}

template <int NP>
static gbk_status launch_np(const TangentArgs &args, size_t smem, cudaStream_t stream)
{
    static KernelAttrMemo memo;
    auto kern = tangent_kernel<NP>;
    gbk_status s0 = ensure_kernel_attrs((const void *)kern, smem, true, memo,
                                        "tangent kernel: setting its shared memory and cluster attributes");
    if (s0) return s0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(args.n_models * args.cs), 1, 1);
    cfg.blockDim = dim3(kTangentThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)args.cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, args);
    if (e != cudaSuccess) return cuda_fail(e, "tangent kernel launch");
    return GBK_OK;
}

gbk_status launch_tangent(const TangentArgs &args, cudaStream_t stream)
{
    if (!args.geoms && args.g.model != GBK_MODEL_CUBE) return launch_vfield_tangent(args, stream);
    if (args.geoms && args.jac) return fail(GBK_EINVAL, "ragged tangent launches do not write J");
    if (args.np < 1 || args.np > GBK_NPAR) return fail(GBK_EINVAL, "tangent launch: bad free-parameter count");
    // carry only x0 .. sigma0 when I0 and h are fixed and J is not written
    const bool narrow = tangent_narrow(args);
    if (args.geoms && !narrow)
        return fail(GBK_EUNSUPPORTED, "ragged Jacobian launches carry the eight parameters x0 .. sigma0");
    size_t smem = args.geoms ? args.smem : tangent_smem_bytes(args.g, args.band, kTangentThreads, args.direct, narrow);
    return narrow ? launch_np<GBK_I0>(args, smem, stream) : launch_np<GBK_NPAR>(args, smem, stream);
}

bool tangent_narrow(const TangentArgs &a)
{
    bool narrow = !a.jac;
    for (int k = 0; k < a.np; ++k) narrow = narrow && a.free_idx[k] < GBK_I0;
    return narrow;
}

int tangent_cluster_for(const Geom &g)
{
    int cs, band, direct;
    return tangent_config(g, &cs, &band, &direct, true) ? cs + 32 * direct : 0;
}

// Halo copies while they fit -- first two CTAs per SM (narrow launches: 110 KB
// per CTA), then one (200 KB) -- otherwise direct reads of the neighbours'
// records, up to 220 KB per CTA.  The smallest cluster of the first shape
// that fits.
bool tangent_config(const Geom &g, int *cs, int *band, int *direct, bool narrow)
{
    if (g.u != 1) return false;
    const size_t caps[3] = {(size_t)110 * 1024, (size_t)200 * 1024, (size_t)220 * 1024};
    for (int pass = narrow ? 0 : 1; pass < 3; ++pass) {
        const int d = pass == 2 ? 1 : 0;
        for (int c = 1; c <= 16; ++c) {
            int b = (g.ey + c - 1) / c;
            if (c > g.ey) break;
            if (tangent_smem_bytes(g, b, kTangentThreads, d, narrow) <= caps[pass]) {
                *cs = c;
                *band = b;
                *direct = d;
                return true;
            }
        }
    }
    return false;
}

}  // namespace gbk
