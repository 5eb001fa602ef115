// k_fused.cu -- fused forward model: cube -> PSF x LSF convolution -> moments
// -> masked chi-squared in one kernel, with the cube never written to HBM.
//
// What it computes is exactly Sec. 2.2.2-2.2.6 of Bekiaris et al. 2015 at
// u = 1 (the GPU parity tests compare it voxel-for-voxel of the maps against
// the direct FP64 definition).  How it computes it differs from the paper's
// FFT pipeline, using three exact identities of finite sums:
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
//  3. Sums about a spaxel-local velocity a are re-centred exactly when they
//     are moved to a neighbour with centre a':  q1' = q1 + D q0,
//     q2' = q2 + 2 D q1 + D^2 q0, D = a - a'.  Centring each spectrum on its
//     own line-of-sight velocity keeps the FP32 second moment free of
//     cancellation.
//
// Work decomposition: one thread-block cluster per model; the CTAs of the
// cluster split the extended rows into bands.  Each CTA evaluates the
// Gaussian line of every extended spaxel of its band (the hot loop: one ex2
// per extended voxel), applies the x pass in shared memory, then reads the
// rows of the y pass from its neighbours' shared memory (DSMEM) so no halo is
// computed twice.  chi2 is reduced in a fixed order: warp shuffles, then
// CTA, then cluster rank 0 over the ranks.
#include <cooperative_groups.h>

#include "gbk_api_internal.h"
#include "gbk_internal.cuh"
#include "k_fused.h"

namespace cg = cooperative_groups;

namespace gbk {

__host__ __device__ inline int pad4(int n) { return (n + 3) & ~3; }

__host__ __device__ inline size_t fused_smem_bytes(const Geom &g, int band)
{
    size_t b = 0;
    b += (size_t)band * g.ex * sizeof(float4);  // Q: per extended spaxel (q0, q1, q2, a)
    b += (size_t)band * g.nx * sizeof(float4);  // P: after the x pass
    b += (size_t)g.ez * sizeof(float4);         // z edge table (G0, dv H1, dv^2 H2, -)
    b += (size_t)pad4(2 * g.R + 1) * sizeof(float);
    b += (size_t)pad4(2 * g.Rz + 1) * sizeof(float);
    b += 64 * sizeof(double);                   // reduction scratch
    return b;
}

size_t fused_smem_bytes_host(const Geom &g, int band) { return fused_smem_bytes(g, band); }

// Moves a (q0, q1, q2) triple centred on a to centre c and accumulates it with
// weight w (identity 3 above).
__device__ __forceinline__ void accum_shift(float4 q, float c, float w, float &s0, float &s1, float &s2)
{
    float D = q.w - c;
    float t0 = w * q.x;
    float t1 = w * q.y;
    s0 += t0;
    s1 += fmaf(D, t0, t1);
    s2 += fmaf(w, q.z, D * fmaf(D, t0, 2.f * t1));
}

__global__ void __launch_bounds__(kFusedThreads, 2) fused_eval_kernel(FusedArgs a)
{
    cg::cluster_group cluster = cg::this_cluster();
    const Geom &g = a.g;
    const int cs = a.cs;
    const int rank = (int)cluster.block_rank();
    const int model = blockIdx.x / cs;
    const int band = a.band;
    const int row0 = rank * band;                       // first extended row of this CTA
    const int nrows = max(0, min(g.ey, row0 + band) - row0);

    extern __shared__ __align__(16) unsigned char smem[];
    float4 *Q = reinterpret_cast<float4 *>(smem);
    float4 *P = Q + (size_t)band * g.ex;
    float4 *ztab = P + (size_t)band * g.nx;
    float *wxy = reinterpret_cast<float *>(ztab + g.ez);
    float *wz = wxy + pad4(2 * g.R + 1);
    double *red = reinterpret_cast<double *>(wz + pad4(2 * g.Rz + 1));

    __shared__ ModelConst mc;
    __shared__ float s_var_z;  // dv^2 * sum_j j^2 L_j
    if (threadIdx.x == 0) mc = model_const(a.params + (size_t)model * GBK_NPAR, g);

    // ---- kernel taps and the z table (per CTA, FP32, parallel) ----
    block_taps(g.sig_xy, g.R, wxy);
    block_taps(g.sig_z, g.Rz, wz);
    for (int e = threadIdx.x; e < g.ez; e += blockDim.x) {
        int kd = e - g.Rz;  // data channel of extended channel e
        int jlo = max(0, kd - g.Rz) - kd, jhi = min(g.nz - 1, kd + g.Rz) - kd;
        float G0 = 0.f, H1 = 0.f, H2 = 0.f;
        for (int j = jlo; j <= jhi; ++j) {
            float w = wz[j + g.Rz];
            G0 += w;
            H1 = fmaf(w, (float)j, H1);
            H2 = fmaf(w, (float)(j * j), H2);
        }
        ztab[e] = make_float4(G0, g.dv * H1, g.dv * g.dv * H2, 0.f);
    }
    if (threadIdx.x == 0) {
        float V = 0.f;
        for (int j = -g.Rz; j <= g.Rz; ++j) V = fmaf(wz[j + g.Rz], (float)(j * j), V);
        s_var_z = g.dv * g.dv * V;
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
    const int nsp = nrows * g.ex;
    const float v_lo = g.vc - 0.5f * (float)(g.nz - 1) * g.dv;  // first and last data channel
    const float v_hi = g.vc + 0.5f * (float)(g.nz - 1) * g.dv;
    for (int idx = threadIdx.x; idx < nsp; idx += blockDim.x) {
        int r = idx / g.ex, xe = idx - r * g.ex;
        float x = (float)(xe - g.R), y = (float)(row0 + r - g.R);
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
        float s0, s1, s2;
        if (sh == 0.f) {
            float s0a = 0.f, s1a = 0.f, s2a = 0.f, s0b = 0.f, s1b = 0.f, s2b = 0.f;
            int e = elo;
            for (; e + 1 < ehi; e += 2) {
                float u0 = fmaf((float)e, adv, ub);
                float u1 = u0 + adv;
                float g0 = ex2_approx(-u0 * u0);
                float g1 = ex2_approx(-u1 * u1);
                float t0 = g0 * u0, t1 = g1 * u1;
                s0a += g0; s1a += t0; s2a = fmaf(t0, u0, s2a);
                s0b += g1; s1b += t1; s2b = fmaf(t1, u1, s2b);
            }
            if (e < ehi) {
                float u0 = fmaf((float)e, adv, ub);
                float g0 = ex2_approx(-u0 * u0);
                float t0 = g0 * u0;
                s0a += g0; s1a += t0; s2a = fmaf(t0, u0, s2a);
            }
            s0 = s0a + s0b; s1 = s1a + s1b; s2 = s2a + s2b;
        } else {
            float ubs = al * (base + sh);
            s0 = s1 = s2 = 0.f;
            for (int e = elo; e < ehi; ++e) {
                float u0 = fmaf((float)e, adv, ub);
                float w0 = fmaf((float)e, adv, ubs);
                float g0 = ex2_approx(-u0 * u0);
                float t0 = g0 * w0;
                s0 += g0; s1 += t0; s2 = fmaf(t0, w0, s2);
            }
        }
        float E0 = 0.f, E1 = 0.f, E2 = 0.f;
        for (int pass = 0; pass < 2; ++pass) {
            int eb = pass ? ehi : 0, ee = pass ? g.ez : elo;
            for (int k = eb; k < ee; ++k) {
                float d = fmaf((float)k, g.dv, base);
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
    }
    __syncthreads();

    // ---- phase 2: x pass (PSF along x), band rows, data columns ----
    const int nout = nrows * g.nx;
    for (int idx = threadIdx.x; idx < nout; idx += blockDim.x) {
        int r = idx / g.nx, x = idx - r * g.nx;
        const float4 *row = Q + (size_t)r * g.ex + x;  // row[j] = extended column x + j
        float cen = row[g.R].w;
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
        for (int j = 0; j <= 2 * g.R; ++j) accum_shift(row[j], cen, wxy[j], s0, s1, s2);
        P[idx] = make_float4(s0, s1, s2, cen);
    }

    cluster.sync();  // every CTA's P is complete and visible cluster-wide

    // ---- phase 3: y pass over DSMEM, moments, residuals, chi2 ----
    // Output data rows y whose extended row y + R lies in this CTA's band.
    const int ylo = max(row0 - g.R, 0);
    const int yhi = min(row0 + nrows - g.R, g.ny);
    double acc = 0.0;
    const bool want_chi2 = (a.chi2 != nullptr);
    const size_t np = (size_t)g.nx * g.ny;
    const float thr = kInvalidFraction * c.i0;
    const float nanf_ = __int_as_float(0x7fc00000);
    for (int idx = threadIdx.x; idx < max(0, yhi - ylo) * g.nx; idx += blockDim.x) {
        int yy = idx / g.nx, x = idx - yy * g.nx;
        int y = ylo + yy;
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
        float cen = 0.f;
        for (int j = 0; j <= 2 * g.R; ++j) {
            int er = y + j;                   // extended row
            int owner = er / band;
            const float4 *Pown = (owner == rank) ? P : cluster.map_shared_rank(P, owner);
            float4 p = Pown[(size_t)(er - owner * band) * g.nx + x];
            if (j == 0) {
                int ec = y + g.R;
                int oc = ec / band;
                const float4 *Pc = (oc == rank) ? P : cluster.map_shared_rank(P, oc);
                cen = Pc[(size_t)(ec - oc * band) * g.nx + x].w;
            }
            accum_shift(p, cen, wxy[j], s0, s1, s2);
        }
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
            acc += (double)(rv * rv) + (double)(rs * rs);
            if (a.resid) {
                float *rp = a.resid + (size_t)model * 2 * np;
                rp[pix] = rv; rp[np + pix] = rs;
            }
        }
    }

    if (want_chi2) {
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, off);
        int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (lane == 0) red[warp] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
            red[32] = s;
        }
    }
    cluster.sync();  // all y-pass DSMEM reads done; CTA partials visible
    if (want_chi2 && rank == 0 && threadIdx.x == 0) {
        double s = 0.0;
        for (int r = 0; r < cs; ++r) {
            const double *rr = (r == 0) ? red : cluster.map_shared_rank(red, r);
            s += rr[32];
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
