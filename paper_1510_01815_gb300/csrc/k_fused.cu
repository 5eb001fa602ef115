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
// Work decomposition: thread-block clusters loop over the models (either one
// resident wave of clusters, as many as fit on the device, or one cluster per
// model -- a tuning choice); the CTAs of a cluster split a model's
// extended rows into balanced bands.  The PSF taps, LSF edge tables and row
// offsets depend only on the geometry and are set up once per CTA.  For each
// model each CTA
//   phase 1  samples the Gaussian line of every extended spaxel of its band
//            (the hot loop: one ex2 and five FP32 lane operations per
//            extended voxel, issued as packed f32x2 pairs) into per-spaxel
//            sums Q = (q0, q1, q2, a); the 2 Rz channels at each band edge
//            use three table-weighted sums referenced to their block's
//            middle channel;
//   phase 2  applies the PSF along x in shared memory (Q -> P);
//   phase 3  copies the R rows above and below its band from its neighbours'
//            shared memory (DSMEM, once, coalesced) so that no halo row is
//            evaluated twice, applies the PSF along y, takes the moments, the
//            residuals and this CTA's part of chi2;
// and cluster rank 0 adds the CTAs' parts in rank order.  The reduction order
// is fixed, so results are bitwise reproducible.
#include <cooperative_groups.h>

#include <mutex>

#include "gbk_api_internal.h"
#include "gbk_internal.cuh"
#include "fused_line.cuh"
#include "k_fused.h"

namespace cg = cooperative_groups;

namespace gbk {

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
    b += (size_t)3 * edge_table_len(g) * sizeof(float);  // edge tables G0, A1, A2
    b += (size_t)pad4(2 * g.R + 1) * sizeof(float);   // PSF taps
    b += (size_t)pad4(band + 2 * g.R) * sizeof(int);  // row offsets of the y pass
    return b;
}

size_t fused_smem_bytes_host(const Geom &g, int band) { return fused_smem_bytes(g, band); }

// Dynamic shared memory of one model's geometry.
struct FusedSmem {
    float4 *Q, *P;
    float *eG0, *eA1, *eA2, *wxy;
    int *rowoff;
};

__device__ __forceinline__ FusedSmem fused_layout(unsigned char *smem, const Geom &g, int band)
{
    FusedSmem L;
    L.Q = reinterpret_cast<float4 *>(smem);
    L.P = L.Q + fused_q_floats4(g, band);
    const int etl = edge_table_len(g);
    L.eG0 = reinterpret_cast<float *>(L.P + (size_t)band * g.nx);
    L.eA1 = L.eG0 + etl;
    L.eA2 = L.eA1 + etl;
    L.wxy = L.eA2 + etl;
    L.rowoff = reinterpret_cast<int *>(L.wxy + pad4(2 * g.R + 1));
    return L;
}

// Geometry-only tables of one CTA: PSF taps, LSF edge tables, the y-pass row
// offsets and the LSF variance, written by disjoint threads (the caller
// places a barrier before they are read).
__device__ void fused_setup(const Geom &g, const FusedSmem &L, int row0, int row1, float *var_z)
{
    const int tid = threadIdx.x, nthr = blockDim.x, R = g.R;
    if (tid >= nthr - 32) {  // last warp: PSF taps
        for (int j = tid - (nthr - 32); j <= 2 * R; j += 32)
            L.wxy[j] = tap_raw(j - R, g.sig_xy, R) / tap_sum(g.sig_xy, R);
    }
    if (tid == nthr - 64) *var_z = lsf_var(g);
    edge_tables(g, L.eG0, L.eA1, L.eA2, tid - 32, nthr);  // warps 1.. (warp 0 holds thread 0)
    // y-pass row offsets (in float4 units from Q) of extended rows [row0 - R, row1 + R)
    const int nrows = row1 - row0;
    for (int k = tid; k < nrows + 2 * R; k += nthr) {
        int er = row0 - R + k;
        int off;
        if (er < row0) off = k * g.nx;                                        // top halo
        else if (er < row1) off = (int)(L.P - L.Q) + (er - row0) * g.nx;      // own rows
        else off = (R + (er - row1)) * g.nx;                                  // bottom halo
        L.rowoff[k] = off;
    }
}

// RAGGED = false: one geometry (a.g) for every model; the tables are set up
// once per CTA.  RAGGED = true: galaxy gal has geometry a.geoms[gal], its
// maps and residuals are packed at pixel offset a.pix_off[gal] * models per
// galaxy, and the tables are rebuilt for every model.
template <int NT, int MINB, bool RAGGED>
__global__ void __launch_bounds__(NT, MINB) fused_eval_kernel(FusedArgs a)
{
    cg::cluster_group cluster = cg::this_cluster();
    const int cs = a.cs;
    const int rank = (int)cluster.block_rank();
    const int cid = blockIdx.x / cs, ncl = gridDim.x / cs;  // this cluster, clusters in the grid
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int mpg = a.models_per_gal;

    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ ModelConst mc;
    __shared__ gbk_obs s_ob;   // observed maps of the current model's galaxy
    __shared__ float s_var_z;  // dv^2 * sum_j j^2 L_j
    __shared__ double red[40]; // chi2 reduction: one slot per warp, the CTA total in [32]
    __shared__ Geom s_g;       // RAGGED: geometry of the current model

    // Uniform geometry: the tables are built once, before the model loop.
    int band = a.band, row0 = 0, row1 = 0;
    FusedSmem L;
    if (!RAGGED) {
        row0 = band_begin(rank, a.g.ey, cs);
        row1 = band_begin(rank + 1, a.g.ey, cs);
        L = fused_layout(smem, a.g, band);
        fused_setup(a.g, L, row0, row1, &s_var_z);
        __syncthreads();
    }

    // The clusters of the grid take the models in turn: statically (w = cid,
    // cid + ncl, ...) or, with a work counter, in the order they become free.
    // Rank 0 takes the next item and the cluster reads it from rank 0's
    // shared memory after one cluster barrier.  Fetch k uses slot k & 1:
    // rank 0 rewrites a slot only at fetch k + 2, after the barrier of fetch
    // k + 1, which no CTA passes before it has read fetch k.
    // The last a.n_solo models (ragged persistent launches only) are served
    // solo: once the cluster's share is exhausted, every CTA takes those
    // models one at a time from the second counter and evaluates each alone
    // (the whole extended grid in its band, block barriers instead of
    // cluster barriers, no distributed shared memory).
    __shared__ int s_work[2], s_solo[2];
    int fetch = 0, fetch_solo = 0;
    bool solo = false;
    const int n_cl = a.n_models - a.n_solo;  // models served by whole clusters
    // next model from counter ctr over [base, base + lim), passing over the
    // models of galaxies the caller skips (one atomic each, no barrier)
    auto take = [&](int *ctr, int base, int lim) -> int {
        int v = atomicAdd(ctr, 1);
        while (a.skip && v < lim) {
            const int gi = mpg > 0 ? (base + v) / mpg : 0;
            if (a.skip[RAGGED && a.order ? a.order[gi] : gi] == 0) break;
            v = atomicAdd(ctr, 1);
        }
        return v < lim ? base + v : a.n_models;
    };
    auto next_item = [&](int prev) -> int {
        if (!a.work) return prev + ncl;
        if (!solo) {
            const int slot = fetch++ & 1;
            if (rank == 0 && tid == 0) s_work[slot] = take(a.work, 0, n_cl);
            cluster.sync();
            const int v = *cluster.map_shared_rank(&s_work[slot], 0);
            if (v < n_cl || a.n_solo == 0) return v;
            solo = true;  // the same decision in every CTA of the cluster
        }
        const int slot = fetch_solo++ & 1;
        if (tid == 0) s_solo[slot] = take(a.work + 1, n_cl, a.n_solo);
        __syncthreads();
        return s_solo[slot];
    };
    // barrier over the CTAs that share the current model
    auto model_sync = [&]() {
        if (solo) __syncthreads();
        else cluster.sync();
    };
    for (int w = a.work ? next_item(0) : cid; w < a.n_models; w = next_item(w)) {
    int gal, model;
    if (RAGGED) {
        const int gi = w / mpg;
        gal = a.order ? a.order[gi] : gi;
        model = gal * mpg + (w - gi * mpg);
    } else {
        model = w;
        gal = mpg > 0 ? model / mpg : 0;
    }
    if (a.skip && a.skip[gal] != 0) continue;  // same decision in every CTA of the cluster
    // CTAs sharing this model and this CTA's rank among them
    const int mcs = solo ? 1 : cs, mrank = solo ? 0 : rank;
    if (RAGGED) {
        // The previous model ended with a cluster (or block) barrier, so
        // nobody still reads s_g or the tables.
        if (tid == 0) s_g = a.geoms[gal];
        __syncthreads();
        band = (s_g.ey + mcs - 1) / mcs;
        row0 = band_begin(mrank, s_g.ey, mcs);
        row1 = band_begin(mrank + 1, s_g.ey, mcs);
        L = fused_layout(smem, s_g, band);
        fused_setup(s_g, L, row0, row1, &s_var_z);
    }
    const Geom &g = RAGGED ? s_g : a.g;
    const int nrows = row1 - row0;
    const int R = g.R;
    float4 *const Q = L.Q, *const P = L.P;
    const float *const eG0 = L.eG0, *const eA1 = L.eA1, *const eA2 = L.eA2, *const wxy = L.wxy;
    const int *const rowoff = L.rowoff;
    // pixel offset of this model's maps and residuals
    const size_t mo = RAGGED ? (size_t)a.pix_off[gal] * mpg + (size_t)(model - gal * mpg) * g.nx * g.ny
                             : (size_t)model * g.nx * g.ny;
    if (tid == 0) {
        mc = model_const(a.params + (size_t)model * GBK_NPAR, g);
        s_ob = a.obs_list ? a.obs_list[gal] : a.obs;
    }
    __syncthreads();
    const float var_z = s_var_z;
    const ModelConst &c = mc;  // read from shared memory (broadcast) to save registers

    // ---- phase 1: Gaussian line of every extended spaxel of the band ----
    // Interior channels [elo, ehi) have their whole LSF window inside the band.
    const LineCtx lc = line_ctx(g, c, var_z);
    const int nsp = nrows * g.ex;
    int r = tid / g.ex, xe = tid - r * g.ex;
    const int dr_e = nthr / g.ex, dx_e = nthr - dr_e * g.ex;  // (row, col) step of idx += nthr
    for (int idx = tid; idx < nsp; idx += nthr) {
        const float x = (float)(xe - R), y = (float)(row0 + r - R);
        Q[idx] = line_sums(g, c, lc, eG0, eA1, eA2, x, y);
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
#pragma unroll 4
        for (int j = 0; j <= 2 * R; ++j) accum_shift(row[j], cen, wxy[j], s0, s1, s2);
        P[idx] = make_float4(s0, s1, s2, cen);
        x += dx_x; r += dr_x;
        if (x >= g.nx) { x -= g.nx; ++r; }
    }

    model_sync();  // every CTA's P is complete and visible cluster-wide; Q is free

    // ---- phase 3a: copy the halo rows of the y pass from the neighbours ----
    // All of a thread's remote loads are issued before its shared stores so
    // the DSMEM latencies overlap.
    {
        const int nh = 2 * R * g.nx;
        constexpr int kU = 4;
        for (int base = tid; base < nh; base += kU * nthr) {
            float4 v[kU];
            int dst[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                int i = base + u * nthr;
                dst[u] = -1;
                if (i < nh) {
                    int k = i / g.nx, xx = i - k * g.nx;
                    int er = (k < R) ? row0 - R + k : row1 + (k - R);
                    if (er >= 0 && er < g.ey) {
                        // (never reached solo: the CTA owns every row)
                        int owner = band_owner(er, g.ey, mcs);
                        const float4 *src = cluster.map_shared_rank(P, owner);
                        v[u] = src[(size_t)(er - band_begin(owner, g.ey, mcs)) * g.nx + xx];
                        dst[u] = i;
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < kU; ++u)
                if (dst[u] >= 0) Q[dst[u]] = v[u];
        }
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
    const bool want_obs = want_chi2 || a.resid;
    for (int idx = tid; idx < nyout * g.nx; idx += nthr) {
        int y = ylo + r;
        size_t pix = (size_t)y * g.nx + x;
        // observed values first, so their latency overlaps the y pass
        uint8_t mk = 0;
        float vo = 0.f, so = 0.f, wv = 0.f, ws = 0.f;
        if (want_obs) {
            mk = s_ob.mask[pix];
            vo = s_ob.v_obs[pix];
            so = s_ob.s_obs[pix];
            wv = s_ob.w_v[pix];
            ws = s_ob.w_s[pix];
        }
        int k0 = y - (row0 - R);  // row-offset index of extended row y (tap j = 0)
        float cen = Q[rowoff[k0 + R] + x].w;
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll 4
        for (int j = 0; j <= 2 * R; ++j) accum_shift(Q[rowoff[k0 + j] + x], cen, wxy[j], s0, s1, s2);
        float m0, m1, m2;
        bool valid = s0 > thr;
        if (!c.valid) {
            m0 = m1 = m2 = nanf_;
        } else if (valid) {
            float inv = __frcp_rn(s0);
            float mu = s1 * inv;
            float var = fmaf(-mu, mu, s2 * inv);
            m0 = s0;
            m1 = cen + mu;
            m2 = sqrtf(fmaxf(var, 0.f));
        } else {
            m0 = 0.f; m1 = c.vsys; m2 = 0.f;
        }
        if (a.maps) {
            float *mp = a.maps + 3 * mo;
            mp[pix] = m0; mp[np + pix] = m1; mp[2 * np + pix] = m2;
        }
        if (want_obs) {
            float rv = 0.f, rs = 0.f;
            if (mk != 0 && (valid || !c.valid)) {
                rv = wv * (m1 - vo);
                rs = ws * (m2 - so);
            }
            acc.add(rv * rv);
            acc.add(rs * rs);
            if (a.resid) {
                float *rp = a.resid + 2 * mo;
                rp[pix] = rv; rp[np + pix] = rs;
            }
        }
        x += dx_x; r += dr_x;
        if (x >= g.nx) { x -= g.nx; ++r; }
    }

    if (want_chi2) {
        // each warp's sum in FP32 (the compensated per-thread sums, a fixed
        // shuffle tree), the warps and the CTAs in FP64
        float v = acc.s - acc.c;
        for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
        int warp = tid >> 5, lane = tid & 31;
        if (lane == 0) red[warp] = (double)v;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int w = 0; w < (nthr >> 5); ++w) s += red[w];
            red[32] = s;
        }
    }
    // Halo reads of every CTA's P are done and the CTA parts of chi2 are
    // visible.  No second barrier is needed before the next model: P and
    // red are next written after that model's first cluster barrier, which
    // rank 0 reaches only once it has read the parts below.
    model_sync();
    if (want_chi2 && mrank == 0 && tid == 0) {
        double s = 0.0;
        for (int rr = 0; rr < mcs; ++rr) {
            const double *p = (rr == 0) ? red : cluster.map_shared_rank(red, rr);
            s += p[32];
        }
        a.chi2[model] = c.valid ? s : (double)nanf_;
    }
    }  // models
    cluster.sync();  // keep every CTA's shared memory alive until rank 0 is done
}

template <int NT, int MINB, bool RAGGED>
static gbk_status launch_variant(const FusedArgs &args, size_t smem, cudaStream_t stream)
{
    // Shared-memory opt-in is set to what this launch needs (static shared
    // memory of the kernel counts against the same per-block limit).
    static KernelAttrMemo memo;
    auto kern = fused_eval_kernel<NT, MINB, RAGGED>;
    gbk_status s0 = ensure_kernel_attrs((const void *)kern, smem, true, memo,
                                        "fused kernel: setting its shared memory and cluster attributes");
    if (s0) return s0;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(NT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)args.cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // One wave of clusters: as many as can be resident at once (cached per
    // device, cluster size and shared-memory size), each looping over models.
    int ncl = args.n_models;
    if (args.persistent) {
        struct Wave { int cs = -1, clusters = 0; size_t smem = 0; };
        static Wave cache[kMaxDevices];
        static std::mutex mu;
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
        if (dev < 0 || dev >= kMaxDevices) return fail(GBK_EUNSUPPORTED, "device ordinal %d out of range", dev);
        std::lock_guard<std::mutex> lk(mu);
        Wave &w = cache[dev];
        if (w.cs != args.cs || w.smem != smem) {
            cfg.gridDim = dim3((unsigned)args.cs, 1, 1);
            int n = 0;
            e = cudaOccupancyMaxActiveClusters(&n, kern, &cfg);
            if (e != cudaSuccess) return cuda_fail(e, "fused kernel: cluster occupancy query");
            if (n < 1) return fail(GBK_EUNSUPPORTED, "no %d-CTA cluster of the fused kernel fits on this device", args.cs);
            w.cs = args.cs;
            w.smem = smem;
            w.clusters = n;
        }
        if (w.clusters < ncl) ncl = w.clusters;
    }
    cfg.gridDim = dim3((unsigned)(ncl * args.cs), 1, 1);
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, args);
    if (e != cudaSuccess) return cuda_fail(e, "fused kernel launch");
    return GBK_OK;
}

gbk_status launch_fused(const FusedArgs &args, cudaStream_t stream)
{
    if (!args.geoms && args.g.model != GBK_MODEL_CUBE) return launch_vfield(args, stream);
    if (args.geoms) {
        if (args.models_per_gal < 1 || args.n_models % args.models_per_gal != 0 || !args.pix_off)
            return fail(GBK_EINVAL, "ragged fused launch: inconsistent batch description");
        switch (args.threads) {
        case 512: return launch_variant<512, 2, true>(args, args.smem, stream);
        case 384: return launch_variant<384, 2, true>(args, args.smem, stream);
        case 256: return launch_variant<256, 4, true>(args, args.smem, stream);
        default: return fail(GBK_EINVAL, "unsupported fused block size %d", args.threads);
        }
    }
    size_t smem = fused_smem_bytes(args.g, args.band);
    switch (args.threads) {
    case 512: return launch_variant<512, 2, false>(args, smem, stream);
    case 384: return launch_variant<384, 2, false>(args, smem, stream);
    case 256: return launch_variant<256, 4, false>(args, smem, stream);
    default: return fail(GBK_EINVAL, "unsupported fused block size %d", args.threads);
    }
}

// Shared memory a ragged launch with cluster size cs needs: the largest of
// its geometries' needs; false if one of them does not fit.
bool fused_config_ragged(const Geom *geoms, int n, int cs, int threads, size_t *smem)
{
    size_t need = 0;
    for (int i = 0; i < n; ++i) {
        const Geom &g = geoms[i];
        if (g.u != 1 || cs > g.ey) return false;
        size_t b = fused_smem_bytes(g, (g.ey + cs - 1) / cs);
        if (b > need) need = b;
    }
    if (need > (size_t)kFusedMaxSmem || (threads != 512 && threads != 384 && threads != 256)) return false;
    *smem = need;
    return true;
}

}  // namespace gbk
