// fused_line.cuh -- the per-spaxel pieces of the folded forward model that
// both fused evaluators use (k_fused.cu: one thread-block cluster per model;
// k_split.cu: line sampling and PSF passes as separate stages).
//
// Model: Bekiaris et al. 2015, Sec. 2.2.2 (cube), Sec. 2.1.7 / Eq. 9 and
// Sec. 2.2.3 (PSF x LSF convolution), Sec. 2.2.5 (moments).  The identities
// that fold the LSF convolution and the channel sums of the moments into
// per-channel weights, and that re-centre moment sums exactly, are stated
// in k_fused.cu's header.
#pragma once

#include "gbk_internal.cuh"

namespace gbk {

__host__ __device__ inline int pad4(int n) { return (n + 3) & ~3; }

// Edge channels of the extended band: the lower block [0, elo) and the upper
// block [ehi, ez) have part of their LSF window outside the data band.
__host__ __device__ inline int edge_lo_end(const Geom &g) { return g.ez < 2 * g.Rz ? g.ez : 2 * g.Rz; }
__host__ __device__ inline int edge_hi_begin(const Geom &g)
{
    int elo = edge_lo_end(g);
    return g.nz > elo ? g.nz : elo;
}
// Floats per edge table: both blocks, each padded to an even length.
__host__ __device__ inline int edge_table_len(const Geom &g)
{
    int lo = edge_lo_end(g), hi = g.ez - edge_hi_begin(g);
    return pad4(((lo + 1) & ~1) + ((hi + 1) & ~1));
}

// Moves a (q0, q1, q2) triple centred on q.w to centre c and accumulates it
// with weight w (exact re-centring of moment sums).
// With t0 = w q0, t1 = w q1 and u = t1 + D t0 the three contributions are
// t0, u and w q2 + D (u + t1): nine FP32 operations.
__device__ __forceinline__ void accum_shift(float4 q, float c, float w, float &s0, float &s1, float &s2)
{
    const float D = q.w - c;
    const float t0 = w * q.x;
    const float t1 = w * q.y;
    const float u = fmaf(D, t0, t1);
    s0 += t0;
    s1 += u;
    s2 = fmaf(w, q.z, s2);
    s2 = fmaf(D, u + t1, s2);
}

// Accumulates input (q0, q1, q2 about a; l1 = q1 + a q0, h1 = 2 q1
// precomputed per input) into output sums with weight w: s0 and s1 about 0,
// s2 about the output's centre c, exactly re-centred (D = a - c): six FP32
// operations.  The caller moves s1 to c once at the end (s1 - c s0).
__device__ __forceinline__ void accum_lin(float q0, float l1, float h1, float q2, float a, float c, float w,
                                          float &s0, float &s1, float &s2)
{
    const float D = a - c;
    s0 = fmaf(w, q0, s0);
    s1 = fmaf(w, l1, s1);
    const float i1 = fmaf(D, q0, h1);
    const float i2 = fmaf(D, i1, q2);
    s2 = fmaf(w, i2, s2);
}

// An input (q0, q1, q2 about its centre a) moved exactly to a reference
// velocity r shared by a thread's outputs (d = a - r): l1 = q1 + d q0 and
// l2 = q2 + d (2 q1 + d q0), both sums of non-negative or centred terms.
// Each output then accumulates w q0, w l1, w l2 (three FMAs per tap) and
// moves its sums from r to its own centre once at the end (shift_sums).
__device__ __forceinline__ void about_ref(float q0, float q1, float q2, float a, float r, float &l1, float &l2)
{
    const float d = a - r;
    l1 = fmaf(d, q0, q1);
    l2 = fmaf(d, fmaf(d, q0, q1 + q1), q2);
}

// Sums about r moved to centre c (delta = c - r): s1 - delta s0 and
// s2 - 2 delta s1 + delta^2 s0 (exact re-centring of moment sums).
__device__ __forceinline__ void shift_sums(float delta, float s0, float &s1, float &s2)
{
    s2 = fmaf(delta, fmaf(delta, s0, -2.f * s1), s2);
    s1 = fmaf(-delta, s0, s1);
}

// Unnormalised tap and the full normalisation sum (computed by each thread
// that needs it, so no serial section or extra barrier is required).
__device__ __forceinline__ float tap_raw(int j, float sigma, int R)
{
    return (R == 0) ? 1.f : gauss_tap(j, sigma);
}

__device__ __forceinline__ float tap_sum(float sigma, int R)
{
    if (R == 0) return 1.f;
    float s = 0.f;
    for (int j = -R; j <= R; ++j) s += gauss_tap(j, sigma);
    return s;
}

// Kahan-compensated FP32 accumulation (a thread adds a handful of terms).
struct KahanF {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x)
    {
        float y = x - c;
        float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

// LSF variance dv^2 sum_j j^2 L_j (normalised taps).
__device__ __forceinline__ float lsf_var(const Geom &g)
{
    float S = tap_sum(g.sig_z, g.Rz), V = 0.f;
    for (int j = -g.Rz; j <= g.Rz; ++j) V = fmaf(tap_raw(j, g.sig_z, g.Rz), (float)(j * j), V);
    return g.dv * g.dv * (V / S);
}

// Edge tables.  For an edge channel e with in-band LSF tap sums
// G0 = sum L_j, H1 = dv sum L_j j, H2 = dv^2 sum L_j j^2 (j = k - e over
// data channels k) and delta = (e - e_ref) dv from its block's middle
// channel e_ref:  A1 = delta G0 + H1,  A2 = delta^2 G0 + 2 delta H1 + H2,
// so that the moment weights are T0 = G0, T1 = d_ref G0 + A1 and
// T2 = d_ref^2 G0 + 2 d_ref A1 + A2 with d_ref = v(e_ref) - a.
// Entries are written by threads first, first + step, ... (disjoint).
__device__ inline void edge_tables(const Geom &g, float *eG0, float *eA1, float *eA2, int first, int step)
{
    const int elo = edge_lo_end(g), ehi = edge_hi_begin(g);
    const int hi_off = (elo + 1) & ~1;  // table slot of channel ehi
    for (int ee = first; ee < g.ez; ee += step) {
        if (ee < 0 || (ee >= elo && ee < ehi)) continue;
        int kd = ee - g.Rz;  // data channel of extended channel ee
        int jlo = max(0, kd - g.Rz) - kd, jhi = min(g.nz - 1, kd + g.Rz) - kd;
        float S = tap_sum(g.sig_z, g.Rz);
        float G0 = 0.f, H1 = 0.f, H2 = 0.f;
        for (int j = jlo; j <= jhi; ++j) {
            float w = tap_raw(j, g.sig_z, g.Rz);
            G0 += w;
            H1 = fmaf(w, (float)j, H1);
            H2 = fmaf(w, (float)(j * j), H2);
        }
        G0 /= S;
        H1 = g.dv * (H1 / S);
        H2 = g.dv * g.dv * (H2 / S);
        bool lower = ee < elo;
        float eref = lower ? 0.5f * (float)(elo - 1) : 0.5f * (float)(ehi + g.ez - 1);
        float delta = ((float)ee - eref) * g.dv;
        int slot = lower ? ee : hi_off + (ee - ehi);
        eG0[slot] = G0;
        eA1[slot] = fmaf(delta, G0, H1);
        eA2[slot] = fmaf(delta, fmaf(delta, G0, 2.f * H1), H2);
    }
}

// Per-model constants of the line sampling (one set per thread and model).
struct LineCtx {
    int elo, ehi, hi_off;
    float vz0, al, adv, inv_al, inv_adv, v_lo, v_hi, eref_lo, eref_hi, var_z;
};

__device__ __forceinline__ LineCtx line_ctx(const Geom &g, const ModelConst &c, float var_z)
{
    LineCtx L;
    L.elo = edge_lo_end(g);
    L.ehi = edge_hi_begin(g);
    L.hi_off = (L.elo + 1) & ~1;
    L.vz0 = g.vc - ((float)g.Rz + 0.5f * (float)(g.nz - 1)) * g.dv;  // v of e = 0
    L.al = c.alpha;
    L.adv = c.alpha * g.dv;
    L.inv_al = 1.f / c.alpha;
    L.inv_adv = 1.f / L.adv;
    L.v_lo = g.vc - 0.5f * (float)(g.nz - 1) * g.dv;  // first and last data channel
    L.v_hi = g.vc + 0.5f * (float)(g.nz - 1) * g.dv;
    L.eref_lo = 0.5f * (float)(L.elo - 1);
    L.eref_hi = 0.5f * (float)(L.ehi + g.ez - 1);
    L.var_z = var_z;
    return L;
}

// Line-of-sight velocity (Eq. 8) and surface brightness (Eq. 5) at sky
// position (x, y), as los() in gbk_internal.cuh but with one reciprocal
// square root in place of the square root and the division by r, and the
// exponential as a power of two: [Vrot(r)/r] x_e = (2/pi) Vmax atan(r/r_t)
// (1/r) x_e with the r -> 0 limit (2/pi) Vmax / r_t.  Agrees with los() to a
// few FP32 ulps.
__device__ __forceinline__ void los_line(const ModelConst &c, float x, float y, float &v, float &bright)
{
    const float dx = x - c.x0, dy = y - c.y0;
    const float xe = -dx * c.sin_pa + dy * c.cos_pa;  // Eq. 1
    const float ye = -dx * c.cos_pa - dy * c.sin_pa;  // Eq. 2
    const float yd = ye * c.inv_cos_i;
    const float r2 = xe * xe + yd * yd;
    const float ri = rsqrtf(r2);                       // +inf at the centre
    const float r = (r2 > 0.f) ? r2 * ri : 0.f;        // Eq. 3
    const float f = (r2 > 0.f) ? c.vrot_k * atanf(r * c.inv_rt) * ri : c.vrot_k * c.inv_rt;
    v = c.vsys + f * xe * c.sin_i;                     // Eq. 8
    bright = c.i0 * exp2f(-1.4426950408889634f * c.inv_h * r);  // Eq. 5
}

// The moment sums of one extended spaxel at sky position (x, y): its
// Gaussian line (Sec. 2.2.2) sampled in every extended channel, the LSF
// convolution and the channel sums of the moments folded into per-channel
// weights (interior channels: none needed; the 2 Rz channels at each band
// edge: the tables eG0, eA1, eA2).  Returns (A q0, A q1, A q2, a): the sums
// of weight, weight * (v - a) and weight * (v - a)^2 about a = v_los clamped
// into the band, A the line amplitude times the surface brightness.
//
// The Gaussian is 2^(-u^2) with u = alpha (v_e - v_los); a warp samples only
// the union of its lanes' channel windows (|u| <= kUCut for a line centred
// in the band, <= kUFlush for one centred outside it, one channel of margin),
// two channels per packed FP32 instruction, stepping u by additions that are
// re-anchored by one FMA every six channel pairs.
// Must be called by whole warps (the lanes of a warp share the channel
// window); inactive lanes are allowed.
__device__ __forceinline__ float4 line_sums(const Geom &g, const ModelConst &c, const LineCtx &L,
                                            const float *eG0, const float *eA1, const float *eA2, float x, float y)
{
    const f32x2 ADV = pk2(L.adv, L.adv), ADV2 = pk2(2.f * L.adv, 2.f * L.adv), Z2 = pk2(0.f, 0.f);
    const f32x2 TWELVE = pk2(12.f, 12.f);
    float vl, br;
    los_line(c, x, y, vl, br);
    // Sums are taken about a = v_los clamped into the band: for a line
    // inside the band a = v_los; for a line outside it the band edge keeps
    // the FP32 second moment of the truncated spectrum free of
    // cancellation.  (The moments do not depend on this choice.)
    const float a_c = fminf(fmaxf(vl, L.v_lo), L.v_hi);
    const float sh = vl - a_c;
    const float ub = L.al * (L.vz0 - vl);  // u = alpha (v_e - v_los) at e = 0
    const f32x2 UB = pk2(ub, ub);
    const unsigned am = __activemask();
    const bool outside = __any_sync(am, sh != 0.f);

    // channel window of the warp: the union of the lanes' |u| <= cut
    const float cut = (sh != 0.f) ? kUFlush : kUCut;
    float flo = (-cut - ub) * L.inv_adv - 1.f, fhi = (cut - ub) * L.inv_adv + 1.f;
    if (!(flo > -1e6f)) flo = -1e6f;
    if (!(fhi < 1e6f)) fhi = 1e6f;
    const int wlo = __reduce_min_sync(am, (int)floorf(flo));
    const int whi = __reduce_max_sync(am, (int)ceilf(fhi));

    // interior channels [elo, ehi): sums of g, g m, g m^2 with m = alpha (v_e - a)
    int e = L.elo, e_stop = L.ehi;
    if (wlo > L.elo) e = min(L.ehi, L.elo + ((wlo - L.elo) & ~1));  // an even offset keeps the pairing
    if (whi < L.ehi) e_stop = max(e, whi);
    f32x2 S0 = Z2, S1 = Z2, S2 = Z2;
    f32x2 FE = pk2((float)e, (float)(e + 1));
    if (!outside) {
        // m = u: the Gaussian argument is also the moment variable
        for (; e + 12 <= e_stop; e += 12) {
            f32x2 U = fma2(FE, ADV, UB);
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                const f32x2 W = mul2(U, U);
                float w0, w1;
                upk2(W, w0, w1);
                const f32x2 G = pk2(ex2_approx(-w0), ex2_approx(-w1));
                S0 = add2(S0, G); S1 = fma2(G, U, S1); S2 = fma2(G, W, S2);
                U = add2(U, ADV2);
            }
            FE = add2(FE, TWELVE);
        }
        f32x2 U = fma2(FE, ADV, UB);
        for (; e + 2 <= e_stop; e += 2) {
            const f32x2 W = mul2(U, U);
            float w0, w1;
            upk2(W, w0, w1);
            const f32x2 G = pk2(ex2_approx(-w0), ex2_approx(-w1));
            S0 = add2(S0, G); S1 = fma2(G, U, S1); S2 = fma2(G, W, S2);
            U = add2(U, ADV2);
        }
    } else {
        // some lane of the warp has its line outside the band: m = u + alpha sh
        const float su = L.al * sh;
        const f32x2 SU = pk2(su, su);
        for (; e + 12 <= e_stop; e += 12) {
            f32x2 U = fma2(FE, ADV, UB);
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                const f32x2 W = mul2(U, U);
                float w0, w1;
                upk2(W, w0, w1);
                const f32x2 G = pk2(ex2_approx(-w0), ex2_approx(-w1));
                const f32x2 M = add2(U, SU);
                const f32x2 T = mul2(G, M);
                S0 = add2(S0, G); S1 = add2(S1, T); S2 = fma2(T, M, S2);
                U = add2(U, ADV2);
            }
            FE = add2(FE, TWELVE);
        }
        f32x2 U = fma2(FE, ADV, UB);
        for (; e + 2 <= e_stop; e += 2) {
            const f32x2 W = mul2(U, U);
            float w0, w1;
            upk2(W, w0, w1);
            const f32x2 G = pk2(ex2_approx(-w0), ex2_approx(-w1));
            const f32x2 M = add2(U, SU);
            const f32x2 T = mul2(G, M);
            S0 = add2(S0, G); S1 = add2(S1, T); S2 = fma2(T, M, S2);
            U = add2(U, ADV2);
        }
    }
    float s0 = hsum2(S0), s1 = hsum2(S1), s2 = hsum2(S2);
    if (e < e_stop) {  // an odd channel left over
        const float u0 = fmaf((float)e, L.adv, ub);
        const float m0 = outside ? u0 + L.al * sh : u0;
        const float g0 = ex2_approx(-u0 * u0);
        const float t0 = g0 * m0;
        s0 += g0; s1 += t0; s2 = fmaf(t0, m0, s2);
    }
    float q0 = s0, q1 = s1 * L.inv_al, q2 = fmaf(s2, L.inv_al * L.inv_al, L.var_z * s0);

    // edge blocks: E0 = sum g G0, B1 = sum g A1, B2 = sum g A2 over the part
    // of the block inside the warp's window
    for (int blk = 0; blk < 2; ++blk) {
        int eb = blk ? L.ehi : 0, ee = blk ? g.ez : L.elo;
        if (wlo > eb) eb += (min(wlo, ee) - eb) & ~1;  // an even offset keeps the table pairs aligned
        if (whi < ee) ee = max(eb, whi);
        if (eb >= ee) continue;
        const int toff = blk ? L.hi_off - L.ehi : 0;  // table slot = e + toff
        f32x2 E0 = Z2, B1 = Z2, B2 = Z2;
        f32x2 U = fma2(pk2((float)eb, (float)(eb + 1)), ADV, UB);
        int k = eb;
#pragma unroll 3
        for (; k + 2 <= ee; k += 2) {
            const f32x2 W = mul2(U, U);
            float w0, w1;
            upk2(W, w0, w1);
            const f32x2 G = pk2(ex2_approx(-w0), ex2_approx(-w1));
            const int t = k + toff;
            E0 = fma2(G, *reinterpret_cast<const f32x2 *>(eG0 + t), E0);
            B1 = fma2(G, *reinterpret_cast<const f32x2 *>(eA1 + t), B1);
            B2 = fma2(G, *reinterpret_cast<const f32x2 *>(eA2 + t), B2);
            U = add2(U, ADV2);
        }
        float e0 = hsum2(E0), b1 = hsum2(B1), b2 = hsum2(B2);
        if (k < ee) {
            const float u0 = fmaf((float)k, L.adv, ub);
            const float g0 = ex2_approx(-u0 * u0);
            e0 = fmaf(g0, eG0[k + toff], e0);
            b1 = fmaf(g0, eA1[k + toff], b1);
            b2 = fmaf(g0, eA2[k + toff], b2);
        }
        const float dref = fmaf(blk ? L.eref_hi : L.eref_lo, g.dv, L.vz0) - a_c;
        q0 += e0;
        q1 += fmaf(dref, e0, b1);
        q2 += fmaf(dref, fmaf(dref, e0, 2.f * b1), b2);
    }
    const float A = c.amp * br;
    return make_float4(A * q0, A * q1, A * q2, a_c);
}

}  // namespace gbk
