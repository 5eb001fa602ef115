// k_fused.cu -- fused forward model: cube -> PSF x LSF convolution -> moments
// -> masked chi-squared in one kernel, with the cube never written to HBM.
//
// What it computes is exactly Sec. 2.2.2-2.2.6 of Bekiaris et al. 2015 at
// u = 1 (the GPU parity tests compare its maps against the direct FP64
// definition).  How it computes it differs from the paper's FFT pipeline,
// using three exact identities of finite sums:
//
//  1. The moments are linear in the cube and the convolution is linear, so
//     the z (LSF) convolution followed by the channel sums of the moments
//     equals one weighted sum over the extended channels e of the model
//     cube, with weights T_m(e) = sum_{k in band} L(k-e) (v_k - a)^m.  With
//     d = v_e - a these are  T_0 = G0(e),  T_1 = d G0 + dv H1(e),
//     T_2 = d^2 G0 + 2 d dv H1 + dv^2 H2(e), where G0, H1, H2 are the zeroth
//     to second moments of the LSF taps that land inside the band.  Inside
//     the band interior G0 = 1, H1 = 0, H2 = Var(LSF taps).
//  2. Likewise the spatial (PSF) convolution commutes with those channel
//     sums, so it can be applied to the three per-spaxel sums (q0, q1, q2)
//     instead of to every channel.
//  3. Sums about a centre a are re-centred exactly when they are moved to a
//     neighbour with centre a':  q1' = q1 + D q0,  q2' = q2 + 2 D q1 + D^2 q0,
//     D = a - a'.  Centring each spectrum on its own line-of-sight velocity
//     (clamped into the band) keeps the FP32 second moment free of
//     cancellation.
//
// Work decomposition: one thread-block cluster per model; the CTAs of the
// cluster split the extended rows into balanced bands.  Each CTA
//   phase 1  samples the Gaussian line of every extended spaxel of its band
//            (the hot loop: one ex2 and five FP32 operations per extended
//            voxel) into per-spaxel sums Q = (q0, q1, q2, a);
//   phase 2  applies the PSF along x in shared memory (Q -> P);
//   phase 3  copies the R rows above and below its band from its neighbours'
//            shared memory (DSMEM, once, coalesced) so that no halo row is
//            evaluated twice, applies the PSF along y, takes the moments, the
//            residuals and this CTA's part of chi2;
// and cluster rank 0 adds the CTAs' parts in rank order.  The reduction order
// is fixed, so results are bitwise reproducible.
#include <cooperative_groups.h>

#include "gbk_api_internal.h"
#include "gbk_internal.cuh"
#include "k_fused.h"

namespace cg = cooperative_groups;

namespace gbk {

__host__ __device__ inline int pad4(int n) { return (n + 3) & ~3; }

// Extended rows [band_begin(r), band_begin(r+1)) belong to cluster rank r.
__host__ __device__ inline int band_begin(int rank, int ey, int cs) { return (int)(((long)rank * ey) / cs); }

// Rank owning extended row er: the largest r with band_begin(r) <= er.
__device__ inline int band_owner(int er, int ey, int cs) { return (int)((((long)er + 1) * cs - 1) / ey); }

__host__ __device__ inline size_t fused_q_floats4(const Geom &g, int band)
{
    // Q holds the band's extended spaxels during phases 1-2 and the halo
    // rows (R above, R below) during phase 3.
    size_t q = (size_t)band * g.ex, h = (size_t)2 * g.R * g.nx;
    return q > h ? q : h;
}

__host__ __device__ inline size_t fused_smem_bytes(const Geom &g, int band)
{
    size_t b = 0;
    b += fused_q_floats4(g, band) * sizeof(float4);  // Q / halo rows
    b += (size_t)band * g.nx * sizeof(float4);        // P: band rows after the x pass
    b += (size_t)g.ez * sizeof(float4);               // z edge table (G0, dv H1, dv^2 H2, -)
    b += (size_t)pad4(2 * g.R + 1) * sizeof(float);   // PSF taps
    b += (size_t)pad4(band + 2 * g.R) * sizeof(int);  // row offsets of the y pass
    b += 64 * sizeof(double);                         // reduction scratch
    return b;
}

size_t fused_smem_bytes_host(const Geom &g, int band) { return fused_smem_bytes(g, band); }

// Moves a (q0, q1, q2) triple centred on q.w to centre c and accumulates it
// with weight w (identity 3 above).
__device__ __forceinline__ void accum_shift(float4 q, float c, float w, float &s0, float &s1, float &s2)
{
    float D = q.w - c;
    float t0 = w * q.x;
    float t1 = w * q.y;
    s0 += t0;
    s1 += fmaf(D, t0, t1);
    s2 += fmaf(w, q.z, D * fmaf(D, t0, 2.f * t1));
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

__global__ void __launch_bounds__(kFusedThreads, 2) fused_eval_kernel(FusedArgs a)
{
    cg::cluster_group cluster = cg::this_cluster();
    const Geom &g = a.g;
    const int cs = a.cs;
    const int rank = (int)cluster.block_rank();
    const int model = blockIdx.x / cs;
    const int band = a.band;                          // max rows of any CTA
    const int row0 = band_begin(rank, g.ey, cs);
    const int row1 = band_begin(rank + 1, g.ey, cs);
    const int nrows = row1 - row0;
    const int R = g.R;
    const int tid = threadIdx.x, nthr = blockDim.x;

    extern __shared__ __align__(16) unsigned char smem[];
    float4 *Q = reinterpret_cast<float4 *>(smem);
    float4 *P = Q + fused_q_floats4(g, band);
    float4 *ztab = P + (size_t)band * g.nx;
    float *wxy = reinterpret_cast<float *>(ztab + g.ez);
    int *rowoff = reinterpret_cast<int *>(wxy + pad4(2 * R + 1));
    double *red = reinterpret_cast<double *>(rowoff + pad4(band + 2 * R));

    __shared__ ModelConst mc;
    __shared__ float s_var_z;  // dv^2 * sum_j j^2 L_j

    // ---- set-up, all in parallel, one barrier ----
    if (tid == 0) mc = model_const(a.params + (size_t)model * GBK_NPAR, g);
    if (tid >= nthr - 32) {  // last warp: PSF taps
        for (int j = tid - (nthr - 32); j <= 2 * R; j += 32)
            wxy[j] = tap_raw(j - R, g.sig_xy, R) / tap_sum(g.sig_xy, R);
    }
    if (tid == nthr - 64) {
        float S = tap_sum(g.sig_z, g.Rz), V = 0.f;
        for (int j = -g.Rz; j <= g.Rz; ++j) V = fmaf(tap_raw(j, g.sig_z, g.Rz), (float)(j * j), V);
        s_var_z = g.dv * g.dv * (V / S);
    }
    for (int ee = tid - 32; ee < g.ez; ee += nthr) {  // warps 1.. : z edge table
        if (ee < 0) continue;
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
        ztab[ee] = make_float4(G0 / S, g.dv * (H1 / S), g.dv * g.dv * (H2 / S), 0.f);
    }
    // y-pass row offsets (in float4 units from Q) of extended rows [row0 - R, row1 + R)
    for (int k = tid; k < nrows + 2 * R; k += nthr) {
        int er = row0 - R + k;
        int off;
        if (er < row0) off = k * g.nx;                                        // top halo
        else if (er < row1) off = (int)(P - Q) + (er - row0) * g.nx;          // own rows
        else off = (R + (er - row1)) * g.nx;                                  // bottom halo
        rowoff[k] = off;
    }
    __syncthreads();

    const ModelConst c = mc;
    const float var_z = s_var_z;

    // ---- phase 1: Gaussian line of every extended spaxel of the band ----
    // Interior channels [elo, ehi) have their whole LSF window inside the band.
    const int elo = min(2 * g.Rz, g.ez);
    const int ehi = max(g.nz, elo);
    const float vz0 = g.vc - ((float)g.Rz + 0.5f * (float)(g.nz - 1)) * g.dv;  // v of e = 0
    const float al = c.alpha, adv = c.alpha * g.dv, inv_al = 1.f / c.alpha;
    const float adv2 = 2.f * adv, adv3 = 3.f * adv;
    const float v_lo = g.vc - 0.5f * (float)(g.nz - 1) * g.dv;  // first and last data channel
    const float v_hi = g.vc + 0.5f * (float)(g.nz - 1) * g.dv;
    const int nsp = nrows * g.ex;
    int r = tid / g.ex, xe = tid - r * g.ex;
    const int dr_e = nthr / g.ex, dx_e = nthr - dr_e * g.ex;  // (row, col) step of idx += nthr
    for (int idx = tid; idx < nsp; idx += nthr) {
        float x = (float)(xe - R), y = (float)(row0 + r - R);
        float vl, br;
        los(c, x, y, vl, br);
        // Sums are taken about a = v_los clamped into the band: for a line
        // inside the band a = v_los; for a line outside it the band edge keeps
        // the FP32 second moment of the truncated spectrum free of
        // cancellation.  (The moments do not depend on this choice.)
        float a_c = fminf(fmaxf(vl, v_lo), v_hi);
        float base = vz0 - vl;      // d = v_e - v_los at e = 0 (Gaussian argument)
        float sh = vl - a_c;        // d' = d + sh = v_e - a (moment weight)
        float ub = al * base;
        float s0, s1, s2;           // in units of u = alpha d: sum g, sum g u, sum g u^2
        if (sh == 0.f) {
            float s0a = 0.f, s1a = 0.f, s2a = 0.f, s0b = 0.f, s1b = 0.f, s2b = 0.f;
            int e = elo;
            float fe = (float)elo;
            for (; e + 4 <= ehi; e += 4, fe += 4.f) {
                float u0 = fmaf(fe, adv, ub);
                float u1 = u0 + adv, u2 = u0 + adv2, u3 = u0 + adv3;
                float w0 = u0 * u0, w1 = u1 * u1, w2 = u2 * u2, w3 = u3 * u3;
                float g0 = ex2_approx(-w0), g1 = ex2_approx(-w1);
                float g2 = ex2_approx(-w2), g3 = ex2_approx(-w3);
                s0a += g0; s1a = fmaf(g0, u0, s1a); s2a = fmaf(g0, w0, s2a);
                s0b += g1; s1b = fmaf(g1, u1, s1b); s2b = fmaf(g1, w1, s2b);
                s0a += g2; s1a = fmaf(g2, u2, s1a); s2a = fmaf(g2, w2, s2a);
                s0b += g3; s1b = fmaf(g3, u3, s1b); s2b = fmaf(g3, w3, s2b);
            }
            for (; e < ehi; ++e, fe += 1.f) {
                float u0 = fmaf(fe, adv, ub);
                float w0 = u0 * u0;
                float g0 = ex2_approx(-w0);
                s0a += g0; s1a = fmaf(g0, u0, s1a); s2a = fmaf(g0, w0, s2a);
            }
            s0 = s0a + s0b; s1 = s1a + s1b; s2 = s2a + s2b;
        } else {
            float ubs = al * (base + sh);
            s0 = s1 = s2 = 0.f;
            float fe = (float)elo;
            for (int e = elo; e < ehi; ++e, fe += 1.f) {
                float u0 = fmaf(fe, adv, ub);
                float w0 = fmaf(fe, adv, ubs);
                float g0 = ex2_approx(-u0 * u0);
                float t0 = g0 * w0;
                s0 += g0; s1 += t0; s2 = fmaf(t0, w0, s2);
            }
        }
        float E0 = 0.f, E1 = 0.f, E2 = 0.f;
        for (int pass = 0; pass < 2; ++pass) {
            int eb = pass ? ehi : 0, ee = pass ? g.ez : elo;
            float fk = (float)eb;
            for (int k = eb; k < ee; ++k, fk += 1.f) {
                float d = fmaf(fk, g.dv, base);
                float u = al * d;
                float gg = ex2_approx(-u * u);
                float dp = d + sh;
                float4 T = ztab[k];
                float t0 = gg * T.x;
                float h = gg * T.y;
                E0 += t0;
                E1 = fmaf(t0, dp, E1 + h);
                E2 = fmaf(t0 * dp, dp, fmaf(h, 2.f * dp, fmaf(gg, T.z, E2)));
            }
        }
        float A = c.amp * br;
        float4 q;
        q.x = A * (s0 + E0);
        q.y = A * fmaf(s1, inv_al, E1);
        q.z = A * (fmaf(s2, inv_al * inv_al, var_z * s0) + E2);
        q.w = a_c;
        Q[idx] = q;
        xe += dx_e; r += dr_e;
        if (xe >= g.ex) { xe -= g.ex; ++r; }
    }
    __syncthreads();

    // ---- phase 2: x pass (PSF along x), band rows, data columns ----
    const int nout = nrows * g.nx;
    const int dr_x = nthr / g.nx, dx_x = nthr - dr_x * g.nx;
    r = tid / g.nx;
    int x = tid - r * g.nx;
    for (int idx = tid; idx < nout; idx += nthr) {
        const float4 *row = Q + (size_t)r * g.ex + x;  // row[j] = extended column x + j
        float cen = row[R].w;
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
        for (int j = 0; j <= 2 * R; ++j) accum_shift(row[j], cen, wxy[j], s0, s1, s2);
        P[idx] = make_float4(s0, s1, s2, cen);
        x += dx_x; r += dr_x;
        if (x >= g.nx) { x -= g.nx; ++r; }
    }

    cluster.sync();  // every CTA's P is complete and visible cluster-wide; Q is free

    // ---- phase 3a: copy the halo rows of the y pass from the neighbours ----
    for (int k = 0; k < 2 * R; ++k) {
        int er = (k < R) ? row0 - R + k : row1 + (k - R);
        if (er < 0 || er >= g.ey) continue;
        int owner = band_owner(er, g.ey, cs);
        const float4 *src = cluster.map_shared_rank(P, owner) + (size_t)(er - band_begin(owner, g.ey, cs)) * g.nx;
        float4 *dst = Q + (size_t)k * g.nx;
        for (int xx = tid; xx < g.nx; xx += nthr) dst[xx] = src[xx];
    }
    __syncthreads();

    // ---- phase 3b: y pass, moments, residuals, chi2 ----
    // Output data rows y whose extended row y + R lies in this CTA's band.
    const int ylo = max(row0 - R, 0);
    const int yhi = min(row1 - R, g.ny);
    const int nyout = max(0, yhi - ylo);
    KahanF acc;
    const bool want_chi2 = (a.chi2 != nullptr);
    const size_t np = (size_t)g.nx * g.ny;
    const float thr = kInvalidFraction * c.i0;
    const float nanf_ = __int_as_float(0x7fc00000);
    r = tid / g.nx;
    x = tid - r * g.nx;
    for (int idx = tid; idx < nyout * g.nx; idx += nthr) {
        int y = ylo + r;
        int k0 = y - (row0 - R);  // row-offset index of extended row y (tap j = 0)
        float cen = Q[rowoff[k0 + R] + x].w;
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
        for (int j = 0; j <= 2 * R; ++j) accum_shift(Q[rowoff[k0 + j] + x], cen, wxy[j], s0, s1, s2);
        float m0, m1, m2;
        bool valid = s0 > thr;
        if (!c.valid) {
            m0 = m1 = m2 = nanf_;
        } else if (valid) {
            float mu = s1 / s0;
            float var = fmaf(-mu, mu, s2 / s0);
            m0 = s0;
            m1 = cen + mu;
            m2 = sqrtf(fmaxf(var, 0.f));
        } else {
            m0 = 0.f; m1 = c.vsys; m2 = 0.f;
        }
        size_t pix = (size_t)y * g.nx + x;
        if (a.maps) {
            float *mp = a.maps + (size_t)model * 3 * np;
            mp[pix] = m0; mp[np + pix] = m1; mp[2 * np + pix] = m2;
        }
        if (want_chi2 || a.resid) {
            float rv = 0.f, rs = 0.f;
            if (a.obs.mask[pix] != 0 && (valid || !c.valid)) {
                rv = a.obs.w_v[pix] * (m1 - a.obs.v_obs[pix]);
                rs = a.obs.w_s[pix] * (m2 - a.obs.s_obs[pix]);
            }
            acc.add(rv * rv);
            acc.add(rs * rs);
            if (a.resid) {
                float *rp = a.resid + (size_t)model * 2 * np;
                rp[pix] = rv; rp[np + pix] = rs;
            }
        }
        x += dx_x; r += dr_x;
        if (x >= g.nx) { x -= g.nx; ++r; }
    }

    if (want_chi2) {
        double v = (double)acc.s - (double)acc.c;
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        int warp = tid >> 5, lane = tid & 31;
        if (lane == 0) red[warp] = v;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int w = 0; w < (nthr >> 5); ++w) s += red[w];
            red[32] = s;
        }
    }
    cluster.sync();  // halo copies done everywhere; CTA parts visible
    if (want_chi2 && rank == 0 && tid == 0) {
        double s = 0.0;
        for (int rr = 0; rr < cs; ++rr) {
            const double *p = (rr == 0) ? red : cluster.map_shared_rank(red, rr);
            s += p[32];
        }
        a.chi2[model] = c.valid ? s : (double)nanf_;
    }
    cluster.sync();  // keep every CTA's shared memory alive until rank 0 is done
}

gbk_status launch_fused(const FusedArgs &args, cudaStream_t stream)
{
    size_t smem = fused_smem_bytes(args.g, args.band);
    // Shared-memory opt-in is set to what this launch needs (static shared
    // memory of the kernel counts against the same per-block limit).
    static size_t configured = 0;
    static bool cluster_configured = false;
    if (smem > configured) {
        cudaError_t e = cudaFuncSetAttribute(fused_eval_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return cuda_fail(e, "fused kernel: setting dynamic shared memory");
        configured = smem;
    }
    if (!cluster_configured) {
        cudaError_t e = cudaFuncSetAttribute(fused_eval_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return cuda_fail(e, "fused kernel: allowing 16-CTA clusters");
        cluster_configured = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(args.n_models * args.cs), 1, 1);
    cfg.blockDim = dim3(kFusedThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)args.cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, fused_eval_kernel, args);
    if (e != cudaSuccess) return cuda_fail(e, "fused kernel launch");
    return GBK_OK;
}

}  // namespace gbk
