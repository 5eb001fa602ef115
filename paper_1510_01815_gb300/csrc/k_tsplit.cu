// k_tsplit.cu -- the analytic Jacobian of the residual maps (forward-mode
// derivatives through Sec. 2.1-2.2.6 of Bekiaris et al. 2015) in the split
// evaluator's shape: no thread-block cluster, the derivative triplets handed
// from a line stage to a PSF stage through an L2-resident buffer.
//
// What it computes is k_tangent.cu's (the header there states the
// derivative algebra): for every extended spaxel the moment triplet of its
// line and its derivatives with respect to x0, y0, PA, i, Vsys, Vmax, r_t and
// sigma0 (I0 and h held fixed, as in every fit here), through the PSF passes
// (linear: the derivative triplets go through the same passes as the
// values), then the quotient rule of the moments gives each spaxel's two
// Jacobian rows, and J^T J, J^T v (v = the residuals or a caller's
// cotangent) and the sum of squared residuals are reduced per model in a
// fixed order.
//
//  set-up   (tsplit_setup_kernel) per-model constants, the PSF taps and the
//           per-channel LSF tap moments (G0, H1, H2), once per call.
//  stage A  (tsplit_line_kernel<R>) one CTA per few extended rows of a model:
//           each spaxel's value and eight derivative triplets (its channel
//           loop runs over the warp's window of channels where the line is
//           not negligible, |u| <= 6, or up to the FP32 flush for lines
//           centred outside the band), as 28 shared planes; then the PSF pass
//           along x, four outputs per thread, one triplet at a time, written
//           as 28 coalesced planes [model][28][ey][nxp].
//  stage B  (tsplit_psf_kernel<R>) one CTA per 32 x 16 tile of data spaxels
//           of a model: the tile's rows of all 28 planes in one TMA load
//           (bounded mbarrier wait, status bit 3), the PSF pass along y for
//           two outputs per thread, the moments, residuals and Jacobian rows,
//           J^T J, J^T v and sum r^2 per thread, the CTA's sums (FP32 within
//           a warp, FP64 over the warps) in a fixed order; the last tile of
//           a model adds the tiles in order.
//
// The PSF passes accumulate as the split evaluator's (six FP32 operations
// per tap and triplet).  Models go in chunks whose planes stay in L2.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "fused_line.cuh"
#include "gbk_api_internal.h"
#include "k_split.h"
#include "k_tsplit.h"
#include "tma_util.cuh"

namespace gbk {

constexpr int kTsThreads = 256;
constexpr int kTsNP = GBK_I0;                  // derivatives carried: x0 .. sigma0
constexpr int kTsNT = kTsNP + 1;               // triplets: the values and the derivatives
constexpr int kTsPlanes = 3 * kTsNT + 1;       // and the centres
constexpr int kTsTX = 32, kTsTY = 16;          // data spaxels per stage-B tile
constexpr int kTsEnt = kTsNP * (kTsNP + 1) / 2 + kTsNP + 1;  // J^T J upper triangle, J^T v, sum r^2
constexpr size_t kTsL2Budget = (size_t)48 << 20;
constexpr size_t kTsSmemA = (size_t)72 * 1024;   // shared-memory target of a stage-A CTA (three per SM)
constexpr int kTsplitMaxRA = 12;               // most extended rows per stage-A CTA
constexpr long kTsWaitLimit = 1L << 18;        // tries: about one second

__device__ int g_tsplit_status;  // 0 = fine; 1 = a tile's TMA load did not complete in time

// Table layout in the workspace: PSF taps at [4, 4 + 2R + 1), then the three
// per-channel LSF moment arrays of ezp floats each.
constexpr int kTsTabTaps = 4;
constexpr int kTsTabZ = kTsTabTaps + 2 * kTsplitMaxR + 4;

__host__ __device__ inline int ts_rowpitch(int ex) { return ((ex + 3) & ~3) + 4; }
__host__ __device__ inline int ts_ezp(const Geom &g) { return (g.ez + 1) & ~1; }

struct TsArgs {
    Geom g;
    int n_models;             // models of this chunk
    const double *params;     // [n_models][GBK_NPAR]
    const ModelConst *mcs;    // [n_models]
    const float *tab;         // taps and LSF channel moments
    float w1[2 * kTsplitMaxR + 1];  // PSF taps of the launch's models, normalised (host-computed)
    f32x2 w2[2 * kTsplitMaxR + 1];  // the same as (w, w) pairs
    float *pl;                // [n_models][28][ey][nxp]
    int pl_z0;                // first plane of this buffer in the PSF stage's tensor map
    gbk_obs obs;              // every model's galaxy when obs_list is null
    const gbk_obs *obs_list;  // or one per model
    const int32_t *skip;      // per model: non-zero = leave alone (or null)
    const float *cot;         // [n_models][2][ny][nx] cotangent (null: the residuals)
    int np, free_idx[GBK_NPAR];
    double *jtj, *jtv, *chi2; // outputs [n_models][np][np], [n_models][np], [n_models] (each may be null)
    double *part;             // [n_models][tiles][kTsEnt]
    unsigned *arrived;        // [n_models]
    int nxp, ezp, ra, tiles_x, tiles;
    // Ragged batches (a geometry per model; unused in the single-geometry
    // form): model m's geometry, table offset (floats into tab), plane offset
    // (floats into pl, relative to the chunk), rows per stage-A CTA and first
    // part slot; the launch's work items (model, row block or tile).
    const Geom *geo;
    const int *tab_off;
    const long long *pl_off;
    const int *ra_m;
    const int *tile_base;
    const int2 *work;
};

// The tables of one geometry: PSF taps at [kTsTabTaps, + 2R + 1), then the
// per-channel LSF tap moments G0, H1, H2 (ezp floats each) at kTsTabZ.
__device__ void ts_tables(const Geom &g, float *tab, int tid, int nthr)
{
    const int ezp = ts_ezp(g);
    for (int j = tid; j <= 2 * g.R; j += nthr) tab[kTsTabTaps + j] = tap_raw(j - g.R, g.sig_xy, g.R) / tap_sum(g.sig_xy, g.R);
    float *tzx = tab + kTsTabZ, *tzy = tzx + ezp, *tzz = tzy + ezp;
    const float S = tap_sum(g.sig_z, g.Rz);
    for (int e = tid; e < ezp; e += nthr) {
        float G0 = 0.f, H1 = 0.f, H2 = 0.f;
        if (e < g.ez) {
            const int kd = e - g.Rz;  // data channel of extended channel e
            const int jlo = max(0, kd - g.Rz) - kd, jhi = min(g.nz - 1, kd + g.Rz) - kd;
            for (int j = jlo; j <= jhi; ++j) {
                const float w = tap_raw(j, g.sig_z, g.Rz) / S;
                G0 += w;
                H1 = fmaf(w, (float)j, H1);
                H2 = fmaf(w, (float)(j * j), H2);
            }
        }
        tzx[e] = G0;
        tzy[e] = g.dv * H1;
        tzz[e] = g.dv * g.dv * H2;
    }
}

// ---------------------------------------------------------------------------
__global__ void tsplit_setup_kernel(const double *params, int n, Geom g, ModelConst *mcs, float *tab)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) mcs[i] = model_const(params + (size_t)i * GBK_NPAR, g);
    if (blockIdx.x != 0) return;
    ts_tables(g, tab, threadIdx.x, blockDim.x);
}

// Ragged batches: one block per model, its constants and its own tables
// (models with skip[m] != 0 are left alone: a plan over the running
// galaxies gives the others no table slot).
__global__ void tsplit_setup_ragged_kernel(const double *params, const Geom *geo, const int *tab_off,
                                           const int32_t *skip, ModelConst *mcs, float *tab)
{
    const int m = blockIdx.x;
    if (skip && skip[m] != 0) return;
    const Geom g = geo[m];
    if (threadIdx.x == 0) mcs[m] = model_const(params + (size_t)m * GBK_NPAR, g);
    ts_tables(g, tab + tab_off[m], threadIdx.x, blockDim.x);
}

// ---------------------------------------------------------------------------
// The value triplet and the eight derivative triplets of one extended
// spaxel at (x, y) (k_tangent.cu's phase 1, its channel loop limited to the
// warp's window): rec[3 t + m] = component m of triplet t (t = 0: values,
// t = k + 1: d/dp_k), about the centre a (returned).  Whole warps (inactive
// lanes allowed).
__device__ __forceinline__ float tangent_spaxel(const Geom &g, const ModelConst &c, const double *pm, const float *tzx,
                                                const float *tzy, const float *tzz, int ezp, int elo, int ehi,
                                                float var_z, float x, float y, float rec[3 * kTsNT])
{
    const float kdeg = 0.017453292519943295f;  // radians per degree
    const float vz0 = g.vc - ((float)g.Rz + 0.5f * (float)(g.nz - 1)) * g.dv;
    const float v_lo = g.vc - 0.5f * (float)(g.nz - 1) * g.dv, v_hi = g.vc + 0.5f * (float)(g.nz - 1) * g.dv;
    const float sig = c.sigma, isig2 = 1.f / (sig * sig), isig3 = isig2 / sig;
    const float s0p = (float)pm[GBK_SIG0];
    const float dsig_ds0 = (g.lsf_mode == 1) ? s0p / sig : 1.f;
    const float vmax = (float)pm[GBK_VMAX], rtv = (float)pm[GBK_RT];
    const float ci = 1.f / c.inv_cos_i;
    // geometry and its derivatives (Eqs. 1-8)
    const float dx = x - c.x0, dy = y - c.y0;
    const float xe = -dx * c.sin_pa + dy * c.cos_pa;
    const float ye = -dx * c.cos_pa - dy * c.sin_pa;
    const float yd = ye * c.inv_cos_i;
    const float r = sqrtf(xe * xe + yd * yd);
    const float u = r * c.inv_rt;
    const float at = atanf(u);
    const float fv = (r > 0.f) ? 0.63661977f * at / r : 0.63661977f * c.inv_rt;  // f / Vmax
    const float f = vmax * fv;
    const float w = xe * c.sin_i;
    const float vl = c.vsys + f * w;
    const float br = c.i0 * expf(-r * c.inv_h);
    float fp;  // df/dr
    if (u < 0.1f) fp = vmax * 0.63661977f * c.inv_rt * c.inv_rt * u * (-2.f / 3.f + 0.8f * u * u);
    else fp = vmax * 0.63661977f * (u / (1.f + u * u) - at) / (r * r);
    float rx = 0.f, ry = 0.f, ri = 0.f;
    if (r > 0.f) {
        rx = xe / r;
        ry = ye * c.inv_cos_i * c.inv_cos_i / r;
        ri = yd * yd * (c.sin_i * c.inv_cos_i) / r * kdeg;
    }
    const float dxe[3] = {c.sin_pa, -c.cos_pa, ye * kdeg};  // d x_e / d(x0, y0, PA)
    const float dye[3] = {c.cos_pa, c.sin_pa, -xe * kdeg};  // d y_e / d(x0, y0, PA)
    float dv[kTsNP], dlnA[kTsNP];
#pragma unroll
    for (int k = 0; k < kTsNP; ++k) { dv[k] = 0.f; dlnA[k] = 0.f; }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float drk = rx * dxe[k] + ry * dye[k];
        dv[k] = f * c.sin_i * dxe[k] + fp * drk * w;
        dlnA[k] = -drk * c.inv_h;
    }
    dv[GBK_INCL] = kdeg * f * xe * ci + fp * ri * w;
    dlnA[GBK_INCL] = -ri * c.inv_h;
    dv[GBK_VSYS] = 1.f;
    dv[GBK_VMAX] = fv * w;
    dv[GBK_RT] = -0.63661977f * vmax / (rtv * rtv + r * r) * w;
    dlnA[GBK_SIG0] = -dsig_ds0 / sig;
    const float a_c = fminf(fmaxf(vl, v_lo), v_hi);
    const float sh = vl - a_c;
    const float base = vz0 - vl;  // d = v_e - v_los at e = 0

    // the warp's channel window (the union of its lanes' |u| <= cut), whole
    // channel pairs
    const unsigned am = __activemask();
    const float cut = (sh != 0.f) ? kUFlush : kUCut;
    const float inv_adv = 1.f / (c.alpha * g.dv);
    float flo = (-cut - c.alpha * base) * inv_adv - 1.f, fhi = (cut - c.alpha * base) * inv_adv + 2.f;
    if (!(flo > -1e6f)) flo = -1e6f;
    if (!(fhi < 1e6f)) fhi = 1e6f;
    int e0 = __reduce_min_sync(am, (int)floorf(flo)), e1 = __reduce_max_sync(am, (int)ceilf(fhi));
    e0 = max(0, e0) & ~1;
    e1 = min(ezp, (e1 + 1) & ~1);

    // channel sums: SG_k = sum g d^k G0 (k <= 4), S1_k = sum g d^k H1 (k <= 3), S2_k = sum g d^k H2 (k <= 2).
    // Interior channels [elo, ehi) have their whole LSF window in the band:
    // G0 = 1, H1 = 0, H2 = the LSF variance there, so they need no table and
    // only the sums of g d^k; the band-edge channels read the tables.  The
    // segments keep whole channel pairs (the interior starts and stops at
    // even channels inside [elo, ehi); the edge loops take the rest, whose
    // tables are valid for every channel).
    float SG[5], S1[4], S2[3];
    {
        const f32x2 Z2 = pk2(0.f, 0.f), AL2 = pk2(c.alpha * c.alpha, c.alpha * c.alpha);
        const f32x2 DV2 = pk2(2.f * g.dv, 2.f * g.dv);
        f32x2 A0 = Z2, A1 = Z2, A2 = Z2, A3 = Z2, A4 = Z2, B0 = Z2, B1 = Z2, B2 = Z2, B3 = Z2, C0 = Z2, C1 = Z2,
              C2 = Z2;
        f32x2 I0 = Z2, I1 = Z2, I2 = Z2, I3 = Z2, I4 = Z2;
        const int eil = max(e0, min(e1, (elo + 1) & ~1)), eih = max(eil, min(e1, ehi & ~1));
        f32x2 D = pk2(fmaf((float)e0, g.dv, base), fmaf((float)(e0 + 1), g.dv, base));
        auto edge_pair = [&](int e) {
            const f32x2 D2 = mul2(D, D);
            const f32x2 W = mul2(D2, AL2);
            float w0, w1;
            upk2(W, w0, w1);
            const f32x2 G0 = pk2(ex2_approx(-w0), ex2_approx(-w1));
            const f32x2 G1 = mul2(G0, D), G2 = mul2(G0, D2);
            const f32x2 G3 = mul2(G1, D2), G4 = mul2(G2, D2);
            const f32x2 TX = *reinterpret_cast<const f32x2 *>(tzx + e);
            const f32x2 TY = *reinterpret_cast<const f32x2 *>(tzy + e);
            const f32x2 TZ = *reinterpret_cast<const f32x2 *>(tzz + e);
            A0 = fma2(G0, TX, A0); A1 = fma2(G1, TX, A1); A2 = fma2(G2, TX, A2);
            A3 = fma2(G3, TX, A3); A4 = fma2(G4, TX, A4);
            B0 = fma2(G0, TY, B0); B1 = fma2(G1, TY, B1); B2 = fma2(G2, TY, B2); B3 = fma2(G3, TY, B3);
            C0 = fma2(G0, TZ, C0); C1 = fma2(G1, TZ, C1); C2 = fma2(G2, TZ, C2);
            D = add2(D, DV2);
        };
        int e = e0;
        for (; e < eil; e += 2) edge_pair(e);
#pragma unroll 2
        for (; e < eih; e += 2) {
            const f32x2 D2 = mul2(D, D);
            const f32x2 W = mul2(D2, AL2);
            float w0, w1;
            upk2(W, w0, w1);
            const f32x2 G0 = pk2(ex2_approx(-w0), ex2_approx(-w1));
            const f32x2 G1 = mul2(G0, D), G2 = mul2(G0, D2);
            I0 = add2(I0, G0); I1 = add2(I1, G1); I2 = add2(I2, G2);
            I3 = fma2(G1, D2, I3); I4 = fma2(G2, D2, I4);
            D = add2(D, DV2);
        }
        for (; e < e1; e += 2) edge_pair(e);
        const float i0 = hsum2(I0), i1 = hsum2(I1), i2 = hsum2(I2);
        SG[0] = hsum2(A0) + i0; SG[1] = hsum2(A1) + i1; SG[2] = hsum2(A2) + i2;
        SG[3] = hsum2(A3) + hsum2(I3); SG[4] = hsum2(A4) + hsum2(I4);
        S1[0] = hsum2(B0); S1[1] = hsum2(B1); S1[2] = hsum2(B2); S1[3] = hsum2(B3);
        S2[0] = fmaf(var_z, i0, hsum2(C0)); S2[1] = fmaf(var_z, i1, hsum2(C1)); S2[2] = fmaf(var_z, i2, hsum2(C2));
    }
    // B_km (k: power of d from the derivative; m: moment weight about a)
    float B[3][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        B[k][0] = SG[k];
        B[k][1] = SG[k + 1] + sh * SG[k] + S1[k];
        B[k][2] = SG[k + 2] + 2.f * sh * SG[k + 1] + 2.f * S1[k + 1] + sh * sh * SG[k] + 2.f * sh * S1[k] + S2[k];
    }
    const float A = c.amp * br;
#pragma unroll
    for (int m = 0; m < 3; ++m) rec[m] = A * B[0][m];
#pragma unroll
    for (int k = 0; k < kTsNP; ++k) {
        const float ds = (k == GBK_SIG0) ? dsig_ds0 : 0.f;
        const float cA = dlnA[k], cv = dv[k] * isig2, cs3 = ds * isig3;
#pragma unroll
        for (int m = 0; m < 3; ++m) rec[3 * (k + 1) + m] = A * (cA * B[0][m] + cv * B[1][m] + cs3 * B[2][m]);
    }
    return a_c;
}

// ---------------------------------------------------------------------------
// Stage A: triplets of a.ra extended rows, then their x pass.
template <int R, bool RAG>
__global__ void __launch_bounds__(kTsThreads, 3) tsplit_line_kernel(TsArgs a)
{
    constexpr int W = 2 * R + 1;
    constexpr int NIN = 4 + 2 * R;      // inputs of four consecutive outputs
    constexpr int NC4 = (NIN + 3) / 4;  // ... as float4 groups
    extern __shared__ __align__(16) float sm[];
    __shared__ ModelConst mc;
    __shared__ Geom s_g;
    const int tid = threadIdx.x;
    int model, blk;
    if constexpr (RAG) {
        const int2 wk = a.work[blockIdx.x];
        model = wk.x;
        blk = wk.y;
    } else {
        model = blockIdx.y;
        blk = blockIdx.x;
    }
    if (a.skip && a.skip[model] != 0) return;  // the whole CTA
    if constexpr (RAG) {
        if (tid < (int)(sizeof(Geom) / 4))
            reinterpret_cast<int *>(&s_g)[tid] = reinterpret_cast<const int *>(a.geo + model)[tid];
        __syncthreads();
    }
    const Geom &g = RAG ? s_g : a.g;
    const int ra = RAG ? a.ra_m[model] : a.ra;
    const int ezp = RAG ? ts_ezp(g) : a.ezp;
    const int nxp = RAG ? ((g.nx + 3) & ~3) : a.nxp;
    const float *const tab = RAG ? a.tab + a.tab_off[model] : a.tab;
    const int row0 = blk * ra, nrows = min(ra, g.ey - row0);
    const int PA = ts_rowpitch(g.ex);
    const int NPL = ra * PA;
    float *const tz = sm + kTsPlanes * NPL;  // tzx, tzy, tzz
    if (tid < (int)(sizeof(ModelConst) / 4))
        reinterpret_cast<float *>(&mc)[tid] = reinterpret_cast<const float *>(a.mcs + model)[tid];
    for (int i = tid; i < 3 * ezp; i += kTsThreads) tz[i] = tab[kTsTabZ + i];
    __syncthreads();

    // the band's interior channels and the LSF variance there
    const int elo = edge_lo_end(g), ehi = edge_hi_begin(g);
    const float var_z = lsf_var(g);

    // phase 1: triplets of every extended spaxel of the rows.  Layout: the
    // value triplet's three planes, then the derivative triplets in pairs
    // (2P + 1, 2P + 2), each component of a pair one plane of interleaved
    // (first, second) values, then the centres:
    //   value plane m:         sm + m NPL + o
    //   pair P, component m:   sm + 3 NPL + (3 P + m) 2 NPL + 2 o + (0 | 1)
    //   centres:               sm + 27 NPL + o
    const double *pm = a.params + (size_t)model * GBK_NPAR;
    {
        const int nsp = nrows * g.ex;
        int r = tid / g.ex, xe = tid - r * g.ex;
        const int dr = kTsThreads / g.ex, dx = kTsThreads - dr * g.ex;
        for (int idx = tid; idx < nsp; idx += kTsThreads) {
            float rec[3 * kTsNT];
            const float ac = tangent_spaxel(g, mc, pm, tz, tz + ezp, tz + 2 * ezp, ezp, elo, ehi, var_z, (float)(xe - R),
                                            (float)(row0 + r - R), rec);
            const int o = r * PA + xe;
#pragma unroll
            for (int m = 0; m < 3; ++m) sm[m * NPL + o] = rec[m];
#pragma unroll
            for (int P = 0; P < kTsNP / 2; ++P)
#pragma unroll
                for (int m = 0; m < 3; ++m)
                    *reinterpret_cast<float2 *>(sm + 3 * NPL + (3 * P + m) * 2 * NPL + 2 * o) =
                        make_float2(rec[3 * (2 * P + 1) + m], rec[3 * (2 * P + 2) + m]);
            sm[3 * kTsNT * NPL + o] = ac;
            xe += dx; r += dr;
            if (xe >= g.ex) { xe -= g.ex; ++r; }
        }
    }
    __syncthreads();

    // phase 2: x pass; task (triplet, row, outputs 4 gx .. 4 gx + 3), the
    // triplet slowest so that consecutive threads write consecutive outputs
    const int ngx = (g.nx + 3) / 4;
    const size_t pstride = (size_t)g.ey * nxp;  // floats per plane
    float *const P0 = (RAG ? a.pl + a.pl_off[model] : a.pl + (size_t)model * kTsPlanes * pstride) + (size_t)row0 * nxp;
    const float *const QA = sm + 3 * kTsNT * NPL;
    const int ntask = nrows * ngx;
    // units: 0 the value triplet, 1 .. 4 the derivative pairs (f32x2)
    constexpr int kUnits = 1 + kTsNP / 2;
    for (int t = tid; t < ntask * kUnits; t += kTsThreads) {
        const int u = t / ntask, tk = t - u * ntask;
        const int rr = tk / ngx, gx = 4 * (tk - rr * ngx);
        const int ro = rr * PA + gx;
        float av[4 * NC4], cen[4];
#pragma unroll
        for (int c4 = 0; c4 < NC4; ++c4) {
            const float4 v = *reinterpret_cast<const float4 *>(QA + ro + 4 * c4);
            av[4 * c4] = v.x; av[4 * c4 + 1] = v.y; av[4 * c4 + 2] = v.z; av[4 * c4 + 3] = v.w;
        }
#pragma unroll
        for (int o = 0; o < 4; ++o) cen[o] = av[o + R];
        float *const out = P0 + (size_t)rr * nxp + gx;
        // inputs moved exactly to the task's reference velocity (three FMAs
        // a tap), each output's sums moved to its centre at the end
        const float ref = cen[1];
        if (u == 0) {
            const float *Q0 = sm, *Q1 = Q0 + NPL, *Q2 = Q1 + NPL;
            float s[4][3];
#pragma unroll
            for (int o = 0; o < 4; ++o) s[o][0] = s[o][1] = s[o][2] = 0.f;
#pragma unroll
            for (int c4 = 0; c4 < NC4; ++c4) {
                const float4 v0 = *reinterpret_cast<const float4 *>(Q0 + ro + 4 * c4);
                const float4 v1 = *reinterpret_cast<const float4 *>(Q1 + ro + 4 * c4);
                const float4 v2 = *reinterpret_cast<const float4 *>(Q2 + ro + 4 * c4);
                const float q0[4] = {v0.x, v0.y, v0.z, v0.w}, q1[4] = {v1.x, v1.y, v1.z, v1.w};
                const float q2[4] = {v2.x, v2.y, v2.z, v2.w};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int e = 4 * c4 + k;
                    if (e >= NIN) break;
                    float l1, l2;
                    about_ref(q0[k], q1[k], q2[k], av[e], ref, l1, l2);
#pragma unroll
                    for (int o = 0; o < 4; ++o) {
                        const int j = e - o;
                        if (j >= 0 && j < W) {
                            s[o][0] = fmaf(a.w1[j], q0[k], s[o][0]);
                            s[o][1] = fmaf(a.w1[j], l1, s[o][1]);
                            s[o][2] = fmaf(a.w1[j], l2, s[o][2]);
                        }
                    }
                }
            }
#pragma unroll
            for (int o = 0; o < 4; ++o) shift_sums(cen[o] - ref, s[o][0], s[o][1], s[o][2]);
            *reinterpret_cast<float4 *>(out) = make_float4(s[0][0], s[1][0], s[2][0], s[3][0]);
            *reinterpret_cast<float4 *>(out + pstride) = make_float4(s[0][1], s[1][1], s[2][1], s[3][1]);
            *reinterpret_cast<float4 *>(out + 2 * pstride) = make_float4(s[0][2], s[1][2], s[2][2], s[3][2]);
            *reinterpret_cast<float4 *>(out + (size_t)(3 * kTsNT) * pstride) =
                make_float4(cen[0], cen[1], cen[2], cen[3]);
        } else {
            // derivative triplets 2P + 1 and 2P + 2 side by side in f32x2
            // lanes: the same centres, taps and arithmetic as one triplet
            const int P = u - 1;
            const float *B0 = sm + 3 * NPL + (3 * P) * 2 * NPL, *B1 = B0 + 2 * NPL, *B2 = B1 + 2 * NPL;
            const f32x2 Z2 = pk2(0.f, 0.f);
            f32x2 s0[4], s1[4], s2[4];
#pragma unroll
            for (int o = 0; o < 4; ++o) s0[o] = s1[o] = s2[o] = Z2;
#pragma unroll
            for (int c4 = 0; c4 < NC4; ++c4) {
                const float *b0 = B0 + 2 * (ro + 4 * c4), *b1 = B1 + 2 * (ro + 4 * c4), *b2 = B2 + 2 * (ro + 4 * c4);
                const ulonglong2 x0 = *reinterpret_cast<const ulonglong2 *>(b0);
                const ulonglong2 y0 = *reinterpret_cast<const ulonglong2 *>(b0 + 4);
                const ulonglong2 x1 = *reinterpret_cast<const ulonglong2 *>(b1);
                const ulonglong2 y1 = *reinterpret_cast<const ulonglong2 *>(b1 + 4);
                const ulonglong2 x2 = *reinterpret_cast<const ulonglong2 *>(b2);
                const ulonglong2 y2 = *reinterpret_cast<const ulonglong2 *>(b2 + 4);
                const f32x2 q0[4] = {x0.x, x0.y, y0.x, y0.y}, q1[4] = {x1.x, x1.y, y1.x, y1.y};
                const f32x2 q2[4] = {x2.x, x2.y, y2.x, y2.y};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int e = 4 * c4 + k;
                    if (e >= NIN) break;
                    const float d = av[e] - ref;
                    const f32x2 D = pk2(d, d);
                    const f32x2 l1 = fma2(D, q0[k], q1[k]);
                    const f32x2 l2 = fma2(D, fma2(D, q0[k], add2(q1[k], q1[k])), q2[k]);
#pragma unroll
                    for (int o = 0; o < 4; ++o) {
                        const int j = e - o;
                        if (j >= 0 && j < W) {
                            s0[o] = fma2(a.w2[j], q0[k], s0[o]);
                            s1[o] = fma2(a.w2[j], l1, s1[o]);
                            s2[o] = fma2(a.w2[j], l2, s2[o]);
                        }
                    }
                }
            }
            float r[3][2][4];  // [component][triplet of the pair][output]
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                float a0, b0, a1, b1, a2, b2;
                upk2(s0[o], a0, b0);
                upk2(s1[o], a1, b1);
                upk2(s2[o], a2, b2);
                const float dl = cen[o] - ref;
                shift_sums(dl, a0, a1, a2);
                shift_sums(dl, b0, b1, b2);
                r[0][0][o] = a0; r[1][0][o] = a1; r[2][0][o] = a2;
                r[0][1][o] = b0; r[1][1][o] = b1; r[2][1][o] = b2;
            }
#pragma unroll
            for (int h = 0; h < 2; ++h)
#pragma unroll
                for (int m = 0; m < 3; ++m)
                    *reinterpret_cast<float4 *>(out + (size_t)(3 * (2 * P + 1 + h) + m) * pstride) =
                        make_float4(r[m][h][0], r[m][h][1], r[m][h][2], r[m][h][3]);
        }
    }
}

// ---------------------------------------------------------------------------
// Stage B: y pass, moments, Jacobian rows and the per-model reductions.
template <int R, bool RAG>
__global__ void __launch_bounds__(kTsThreads, 2)
    tsplit_psf_kernel(const __grid_constant__ CUtensorMap tmap, TsArgs a)
{
    constexpr int W = 2 * R + 1;
    constexpr int NR = kTsTY + 2 * R;   // rows of the tile's planes
    constexpr int NPL = NR * kTsTX;     // floats per plane
    constexpr int NIN = 2 + 2 * R;      // inputs of two consecutive outputs
    extern __shared__ __align__(128) unsigned char sraw[];
    float *const sp = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(sraw) + 127) & ~(uintptr_t)127);
    __shared__ ModelConst mc;
    __shared__ gbk_obs s_ob;
    __shared__ float red[kTsThreads / 32][kTsEnt];
    __shared__ double s_part[kTsEnt];
    __shared__ bool s_last;
    __shared__ __align__(8) uint64_t bar;

    __shared__ Geom s_g;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int model, tile;
    if constexpr (RAG) {
        const int2 wk = a.work[blockIdx.x];
        model = wk.x;
        tile = wk.y;
    } else {
        model = blockIdx.y;
        tile = blockIdx.x;
    }
    if (a.skip && a.skip[model] != 0) return;  // the whole CTA
    if constexpr (RAG) {
        if (tid < (int)(sizeof(Geom) / 4))
            reinterpret_cast<int *>(&s_g)[tid] = reinterpret_cast<const int *>(a.geo + model)[tid];
        __syncthreads();
    }
    const Geom &g = RAG ? s_g : a.g;
    const int tiles_x = RAG ? (g.nx + kTsTX - 1) / kTsTX : a.tiles_x;
    const int tiles = RAG ? tiles_x * ((g.ny + kTsTY - 1) / kTsTY) : a.tiles;
    double *const part0 = a.part + (RAG ? (size_t)a.tile_base[model] : (size_t)model * a.tiles) * kTsEnt;
    const int tx0 = (tile % tiles_x) * kTsTX, ty0 = (tile / tiles_x) * kTsTY;
    const int nxo = min(kTsTX, g.nx - tx0), nyo = min(kTsTY, g.ny - ty0);
    bool loaded = true;
    if constexpr (RAG) {
        // the tile's rows of all 28 planes by untiled bulk copies, one per
        // plane row inside the model's planes (ncol floats from column tx0:
        // the plane pitch nxp and tx0 are multiples of four, so every address
        // and size is a multiple of 16 bytes), completion on the mbarrier;
        // rows past the planes and columns past nxp are zeroed by stores
        const int nxp = (g.nx + 3) & ~3;
        const size_t pstride = (size_t)g.ey * nxp;
        const float *const src = a.pl + a.pl_off[model];
        const int ncol = min(kTsTX, nxp - tx0);  // >= 4: tx0 < nx <= nxp
        const int nrv = min(NR, g.ey - ty0);     // >= 1: ty0 < ny <= ey
        if (tid == 0) {
            mbar_init(&bar, 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            tma_expect(&bar, (uint32_t)(kTsPlanes * nrv * ncol * sizeof(float)));
        }
        __syncthreads();
        for (int i = tid; i < kTsPlanes * nrv; i += kTsThreads) {
            const int pl = i / nrv, rr = i - pl * nrv;
            bulk_load(sp + pl * NPL + rr * kTsTX, src + pl * pstride + (size_t)(ty0 + rr) * nxp + tx0,
                      (uint32_t)(ncol * sizeof(float)), &bar);
        }
        constexpr int C4 = kTsTX / 4;
        if (nrv < NR || ncol < kTsTX)
            for (int i = tid; i < kTsPlanes * NR * C4; i += kTsThreads) {
                const int c4 = i % C4, rr = (i / C4) % NR, pl = i / (C4 * NR);
                if (rr >= nrv || 4 * c4 >= ncol)
                    *reinterpret_cast<float4 *>(sp + pl * NPL + rr * kTsTX + 4 * c4) = make_float4(0.f, 0.f, 0.f, 0.f);
            }
    } else {
        if (tid == 0) {
            mbar_init(&bar, 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
        if (tid == 0) {
            // the tile's rows of all 28 planes in one box (beyond the buffer: zeros)
            tma_expect(&bar, (uint32_t)(kTsPlanes * NPL * sizeof(float)));
            tma_load_3d(&tmap, sp, &bar, tx0, ty0, a.pl_z0 + kTsPlanes * model);
        }
    }
    if (tid < (int)(sizeof(ModelConst) / 4))
        reinterpret_cast<float *>(&mc)[tid] = reinterpret_cast<const float *>(a.mcs + model)[tid];
    if (tid == 32) s_ob = a.obs_list ? a.obs_list[model] : a.obs;
    loaded = mbar_wait(&bar, 0, kTsWaitLimit);
    if (__syncthreads_or(!loaded)) {  // the same decision in every thread
        if (tid == 0) {
            atomicExch(&g_tsplit_status, 1);
            mbar_wait(&bar, 0, kTsWaitLimit);  // a bounded chance for the copy in flight to land
        }
        return;
    }

    const ModelConst &c = mc;
    const size_t np = (size_t)g.nx * g.ny;
    const float thr = kInvalidFraction * c.i0;
    float E[kTsEnt];
#pragma unroll
    for (int e = 0; e < kTsEnt; ++e) E[e] = 0.f;
    // task: column x, outputs gy, gy + 1
    const int x = tid % kTsTX, gy = 2 * (tid / kTsTX);
    if (x < nxo && gy < nyo) {
        const float *const SA = sp + 3 * kTsNT * NPL;
        float av[NIN], cen[2];
#pragma unroll
        for (int e = 0; e < NIN; ++e) av[e] = SA[(gy + e) * kTsTX + x];
        cen[0] = av[R];
        cen[1] = av[R + 1];
        // the inputs' offsets from the task's reference velocity (the first
        // output's centre), shared by the nine triplets
#pragma unroll
        for (int e = 0; e < NIN; ++e) av[e] -= cen[0];
        // y pass of triplet tr for both outputs: inputs moved exactly to the
        // reference (three FMAs a tap), then each output to its centre
        auto ypass = [&](int tr, float s[2][3]) {
            const float *Q0 = sp + (3 * tr) * NPL, *Q1 = Q0 + NPL, *Q2 = Q1 + NPL;
#pragma unroll
            for (int o = 0; o < 2; ++o) s[o][0] = s[o][1] = s[o][2] = 0.f;
#pragma unroll
            for (int e = 0; e < NIN; ++e) {
                const int oi = (gy + e) * kTsTX + x;
                const float q0 = Q0[oi], q1 = Q1[oi], q2 = Q2[oi], d = av[e];
                const float l1 = fmaf(d, q0, q1), l2 = fmaf(d, fmaf(d, q0, q1 + q1), q2);
#pragma unroll
                for (int o = 0; o < 2; ++o) {
                    const int j = e - o;
                    if (j >= 0 && j < W) {
                        s[o][0] = fmaf(a.w1[j], q0, s[o][0]);
                        s[o][1] = fmaf(a.w1[j], l1, s[o][1]);
                        s[o][2] = fmaf(a.w1[j], l2, s[o][2]);
                    }
                }
            }
            shift_sums(0.f, s[0][0], s[0][1], s[0][2]);
            shift_sums(cen[1] - cen[0], s[1][0], s[1][1], s[1][2]);
        };
        float v[2][3];
        ypass(0, v);
        bool use[2];
        float inv[2], mu[2], inv2m2[2], s2i[2], wv[2], ws[2], cv[2], cs[2];
#pragma unroll
        for (int o = 0; o < 2; ++o) {
            use[o] = false;
            inv[o] = mu[o] = inv2m2[o] = s2i[o] = wv[o] = ws[o] = cv[o] = cs[o] = 0.f;
            if (gy + o >= nyo) continue;
            const size_t pix = (size_t)(ty0 + gy + o) * g.nx + (tx0 + x);
            use[o] = c.valid && v[o][0] > thr && s_ob.mask[pix] != 0;
            if (!use[o]) continue;
            inv[o] = 1.f / v[o][0];
            mu[o] = v[o][1] * inv[o];
            s2i[o] = v[o][2] * inv[o];
            const float m2 = sqrtf(fmaxf(fmaf(-mu[o], mu[o], s2i[o]), 0.f));
            wv[o] = s_ob.w_v[pix];
            ws[o] = s_ob.w_s[pix];
            const float rv = wv[o] * (cen[o] + mu[o] - s_ob.v_obs[pix]);
            const float rs = ws[o] * (m2 - s_ob.s_obs[pix]);
            inv2m2[o] = m2 > 0.f ? 0.5f / m2 : 0.f;
            if (a.cot) {
                cv[o] = a.cot[(size_t)model * 2 * np + pix];
                cs[o] = a.cot[(size_t)model * 2 * np + np + pix];
            } else {
                cv[o] = rv;
                cs[o] = rs;
            }
            E[kTsEnt - 1] = fmaf(rv, rv, fmaf(rs, rs, E[kTsEnt - 1]));
        }
        // the Jacobian rows (quotient rule of the moments), one parameter at a time
        float jv[2][kTsNP], js[2][kTsNP];
#pragma unroll
        for (int k = 0; k < kTsNP; ++k) {
            float d[2][3];
            ypass(k + 1, d);
#pragma unroll
            for (int o = 0; o < 2; ++o) {
                const float dmu = (d[o][1] - mu[o] * d[o][0]) * inv[o];
                const float dvar = (d[o][2] - s2i[o] * d[o][0]) * inv[o] - 2.f * mu[o] * dmu;
                jv[o][k] = use[o] ? wv[o] * dmu : 0.f;
                js[o][k] = use[o] ? ws[o] * dvar * inv2m2[o] : 0.f;
            }
        }
#pragma unroll
        for (int o = 0; o < 2; ++o) {
            int e = 0;
#pragma unroll
            for (int j = 0; j < kTsNP; ++j)
#pragma unroll
                for (int k = j; k < kTsNP; ++k, ++e) E[e] = fmaf(jv[o][j], jv[o][k], fmaf(js[o][j], js[o][k], E[e]));
#pragma unroll
            for (int j = 0; j < kTsNP; ++j, ++e) E[e] = fmaf(jv[o][j], cv[o], fmaf(js[o][j], cs[o], E[e]));
        }
    }
    // the CTA's sums: each warp's in FP32 by a reduce-scatter, then the warps
    // in FP64 in order
    warp_sum_scatter<kTsEnt>(E, lane, red[warp]);
    __syncthreads();
    if (tid < kTsEnt) {
        double sum = 0.0;
        for (int q = 0; q < kTsThreads / 32; ++q) sum += (double)red[q][tid];
        part0[(size_t)tile * kTsEnt + tid] = sum;
    }
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(&a.arrived[model], 1u);
        s_last = (prev == (unsigned)tiles - 1);
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    if (tid < kTsEnt) {
        const volatile double *p = part0 + tid;
        double sum = 0.0;
        for (int k = 0; k < tiles; ++k) sum += p[(size_t)k * kTsEnt];
        s_part[tid] = sum;
    }
    __syncthreads();
    // entry t of the free-parameter output: (j, k) of the upper triangle of
    // J^T J, then J^T v, then sum r^2, gathered from the carried entries
    const int nf = a.np;
    const int ntri = nf * (nf + 1) / 2, nent = ntri + nf + 1;
    if (tid < nent) {
        int src, j = 0, k = 0;
        if (tid < ntri) {
            int t = tid;
            while (t >= nf - j) { t -= nf - j; ++j; }
            k = j + t;
            int p = a.free_idx[j], q = a.free_idx[k];
            if (p > q) { const int x2 = p; p = q; q = x2; }
            src = p * kTsNP - p * (p - 1) / 2 + (q - p);
        } else if (tid < ntri + nf) {
            src = kTsNP * (kTsNP + 1) / 2 + a.free_idx[tid - ntri];
        } else {
            src = kTsEnt - 1;
        }
        double sv = s_part[src];
        if (!c.valid) sv = (double)__int_as_float(0x7fc00000);
        if (tid < ntri) {
            if (a.jtj) {
                a.jtj[(size_t)model * nf * nf + j * nf + k] = sv;
                a.jtj[(size_t)model * nf * nf + k * nf + j] = sv;
            }
        } else if (tid < ntri + nf) {
            if (a.jtv) a.jtv[(size_t)model * nf + (tid - ntri)] = sv;
        } else if (a.chi2) {
            a.chi2[model] = sv;
        }
    }
    if (tid == 0) a.arrived[model] = 0u;  // ready for the next chunk or call
}

// ---------------------------------------------------------------------------
// Host side.
struct TsLayout {
    int chunk, nbuf, nxp, ezp, ra, tiles_x, tiles;
    size_t mc_off, tab_off, pl_off, pl_bytes, part_off, arr_off, total;  // pl_bytes: one buffer
};

static size_t ts_al256(size_t b) { return (b + 255) & ~(size_t)255; }

// Normalised PSF taps exp(-j^2 / (2 sigma^2)) / sum of a launch (every model
// of a launch has the same PSF), as floats and as (w, w) pairs.
static void ts_taps(int R, float sigma, TsArgs &a)
{
    double v[2 * kTsplitMaxR + 1], sum = 0.0;
    for (int j = -R; j <= R; ++j) {
        const double t = (R == 0) ? 0.0 : (double)j / (double)sigma;
        v[j + R] = std::exp(-0.5 * t * t);
        sum += v[j + R];
    }
    for (int j = 0; j <= 2 * R; ++j) {
        const float f = (float)(v[j] / sum);
        uint32_t b;
        std::memcpy(&b, &f, 4);
        a.w1[j] = f;
        a.w2[j] = ((f32x2)b << 32) | (f32x2)b;
    }
}

static size_t ts_smem_a(const Geom &g, int ra)
{
    return (size_t)(kTsPlanes * ra * ts_rowpitch(g.ex) + 3 * ts_ezp(g)) * sizeof(float);
}
static size_t ts_smem_b(int R) { return 128 + (size_t)kTsPlanes * (kTsTY + 2 * R) * kTsTX * sizeof(float); }

// Rows per stage-A CTA: within the shared-memory target, the count whose
// extended spaxels fill the most of whole rounds of the CTA's threads (the
// larger on a tie).
static int ts_rows_a(const Geom &g)
{
    int ra_max = kTsplitMaxRA;
    while (ra_max > 1 && ts_smem_a(g, ra_max) > kTsSmemA) --ra_max;
    int best_ra = ra_max;
    double best = 0.0;
    for (int ra = ra_max; ra >= 1; --ra) {
        const int nsp = ra * g.ex, rounds = (nsp + kTsThreads - 1) / kTsThreads;
        const double use = (double)nsp / (double)(rounds * kTsThreads);
        if (use > best + 1e-9) {
            best = use;
            best_ra = ra;
        }
    }
    return best_ra;
}

static TsLayout ts_layout(const Geom &g, int n_models)
{
    TsLayout L = {};
    L.nxp = (g.nx + 3) & ~3;
    L.ezp = ts_ezp(g);
    L.ra = ts_rows_a(g);
    const size_t plb = (size_t)kTsPlanes * g.ey * L.nxp * sizeof(float);
    size_t chunk = kTsL2Budget / plb;
    if (chunk < 1) chunk = 1;
    if (chunk > (size_t)n_models) chunk = (size_t)n_models;
    const size_t nchunks = ((size_t)n_models + chunk - 1) / chunk;
    chunk = ((size_t)n_models + nchunks - 1) / nchunks;  // balanced chunks
    L.chunk = (int)chunk;
    L.nbuf = nchunks > 1 ? 2 : 1;  // chunk k + 1's line stage runs beside chunk k's PSF stage
    L.tiles_x = (g.nx + kTsTX - 1) / kTsTX;
    L.tiles = L.tiles_x * ((g.ny + kTsTY - 1) / kTsTY);
    L.mc_off = 0;
    L.tab_off = ts_al256((size_t)n_models * sizeof(ModelConst));
    L.pl_off = L.tab_off + ts_al256((size_t)(kTsTabZ + 3 * L.ezp) * sizeof(float));
    L.pl_bytes = chunk * plb;  // a multiple of 16 bytes (nxp is a multiple of 4)
    L.part_off = L.pl_off + ts_al256(L.nbuf * L.pl_bytes);
    L.arr_off = L.part_off + ts_al256(chunk * L.tiles * kTsEnt * sizeof(double));
    L.total = L.arr_off + ts_al256(chunk * sizeof(unsigned));
    return L;
}

bool tsplit_supported(const Geom &g, int np, const int *free_idx)
{
    if (g.model != GBK_MODEL_CUBE || g.u != 1 || g.R > kTsplitMaxR || g.ex > 1024) return false;
    if (np < 1 || np > kTsNP) return false;
    for (int k = 0; k < np; ++k)
        if (free_idx[k] < 0 || free_idx[k] >= kTsNP) return false;
    return ts_smem_a(g, 1) <= 200 * 1024 && ts_smem_b(g.R) <= 200 * 1024;
}

size_t tsplit_workspace_bytes(const Geom &g, int n_models)
{
    if (g.model != GBK_MODEL_CUBE || g.u != 1 || g.R > kTsplitMaxR || n_models < 1) return 0;
    return ts_layout(g, n_models).total;
}

gbk_status tsplit_status_read(int *v)
{
    int zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(v, g_tsplit_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_tsplit_status, &zero, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "reading the split Jacobian's status");
    return GBK_OK;
}

template <int R>
static gbk_status ts_launch_stage(int stage, const CUtensorMap &tm, const TsArgs &a, cudaStream_t st)
{
    static KernelAttrMemo memo_a, memo_b;
    const size_t sa = ts_smem_a(a.g, a.ra), sb = ts_smem_b(R);
    gbk_status s;
    if ((s = ensure_kernel_attrs((const void *)tsplit_line_kernel<R, false>, sa, false, memo_a,
                                 "split Jacobian: setting the line stage's shared memory")) ||
        (s = ensure_kernel_attrs((const void *)tsplit_psf_kernel<R, false>, sb, false, memo_b,
                                 "split Jacobian: setting the PSF stage's shared memory")))
        return s;
    cudaError_t e;
    if (stage == 0) {
        const unsigned blocks_a = (unsigned)((a.g.ey + a.ra - 1) / a.ra);
        tsplit_line_kernel<R, false><<<dim3(blocks_a, (unsigned)a.n_models), kTsThreads, sa, st>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "split Jacobian: line stage launch");
    } else {
        tsplit_psf_kernel<R, false><<<dim3((unsigned)a.tiles, (unsigned)a.n_models), kTsThreads, sb, st>>>(tm, a);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "split Jacobian: PSF stage launch");
    }
    return GBK_OK;
}

static gbk_status ts_launch_stage_r(int stage, const CUtensorMap &tm, const TsArgs &a, cudaStream_t st)
{
    switch (a.g.R) {
    case 0: return ts_launch_stage<0>(stage, tm, a, st);
    case 1: return ts_launch_stage<1>(stage, tm, a, st);
    case 2: return ts_launch_stage<2>(stage, tm, a, st);
    case 3: return ts_launch_stage<3>(stage, tm, a, st);
    case 4: return ts_launch_stage<4>(stage, tm, a, st);
    case 5: return ts_launch_stage<5>(stage, tm, a, st);
    case 6: return ts_launch_stage<6>(stage, tm, a, st);
    case 7: return ts_launch_stage<7>(stage, tm, a, st);
    case 8: return ts_launch_stage<8>(stage, tm, a, st);
    default: return fail(GBK_EUNSUPPORTED, "split Jacobian: PSF radius %d > %d", a.g.R, kTsplitMaxR);
    }
}

gbk_status launch_tsplit(const TsplitCall &call, void *ws, size_t ws_bytes, cudaStream_t st)
{
    const Geom &g = call.g;
    const int n = call.n_models;
    if (!tsplit_supported(g, call.np, call.free_idx))
        return fail(GBK_EUNSUPPORTED, "the split Jacobian serves the cube model at u = 1, PSF radius <= %d, with "
                    "free parameters among x0 .. sigma0", kTsplitMaxR);
    if (n == 0) return GBK_OK;
    const TsLayout L = ts_layout(g, n);
    if (!ws || ws_bytes < L.total)
        return fail(GBK_EWORKSPACE, "the split Jacobian needs %zu bytes of workspace (got %zu)", L.total, ws_bytes);
    if (!split_encode_fn()) return fail(GBK_EUNSUPPORTED, "cuTensorMapEncodeTiled is not available from the driver");
    char *base = (char *)ws;
    ModelConst *mcs = (ModelConst *)(base + L.mc_off);
    float *tab = (float *)(base + L.tab_off);
    cudaError_t e = cudaMemsetAsync(base + L.arr_off, 0, (size_t)L.chunk * sizeof(unsigned), st);
    if (e != cudaSuccess) return cuda_fail(e, "split Jacobian: clearing the arrival counters");
    // the buffers' planes as one 3-D tensor [nbuf * 28 * chunk][ey][nxp] for the tile loads
    CUtensorMap tm;
    {
        const cuuint64_t dims[3] = {(cuuint64_t)L.nxp, (cuuint64_t)g.ey, (cuuint64_t)kTsPlanes * L.chunk * L.nbuf};
        const cuuint64_t strides[2] = {(cuuint64_t)L.nxp * sizeof(float), (cuuint64_t)L.nxp * g.ey * sizeof(float)};
        const cuuint32_t box[3] = {(cuuint32_t)kTsTX, (cuuint32_t)(kTsTY + 2 * g.R), (cuuint32_t)kTsPlanes};
        const cuuint32_t estr[3] = {1, 1, 1};
        CUresult r = split_encode_fn()(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base + L.pl_off, dims, strides, box,
                                       estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                       CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(GBK_ECUDA, "split Jacobian: cuTensorMapEncodeTiled failed (%d)", (int)r);
    }
    tsplit_setup_kernel<<<(n + 127) / 128, 128, 0, st>>>(call.params, n, g, mcs, tab);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "split Jacobian: set-up launch");
    const size_t npix = (size_t)g.nx * g.ny;
    // Two plane buffers: chunk c fills buffer c % 2; chunk c's PSF stage
    // runs on the auxiliary stream beside chunk c + 1's line stage, and
    // chunk c + 2's line stage waits for it.
    const bool overlap = L.nbuf == 2;
    SplitAux *aux = nullptr;
    if (overlap) {
        gbk_status s = split_aux(&aux);
        if (s) return s;
    }
    cudaStream_t sb = overlap ? aux->s : st;
    int c = 0;
    for (int m0 = 0; m0 < n; m0 += L.chunk, ++c) {
        const int b = c & (L.nbuf - 1);
        TsArgs a = {};
        a.g = g;
        a.n_models = std::min(L.chunk, n - m0);
        a.params = call.params + (size_t)m0 * GBK_NPAR;
        a.mcs = mcs + m0;
        a.tab = tab;
        a.pl = (float *)(base + L.pl_off + (size_t)b * L.pl_bytes);
        a.pl_z0 = kTsPlanes * L.chunk * b;
        a.obs = call.obs;
        a.obs_list = call.obs_list ? call.obs_list + m0 : nullptr;
        a.skip = call.skip ? call.skip + m0 : nullptr;
        a.cot = call.cot ? call.cot + 2 * npix * m0 : nullptr;
        a.np = call.np;
        for (int k = 0; k < call.np; ++k) a.free_idx[k] = call.free_idx[k];
        a.jtj = call.jtj ? call.jtj + (size_t)m0 * call.np * call.np : nullptr;
        a.jtv = call.jtv ? call.jtv + (size_t)m0 * call.np : nullptr;
        a.chi2 = call.chi2 ? call.chi2 + m0 : nullptr;
        a.part = (double *)(base + L.part_off);
        a.arrived = (unsigned *)(base + L.arr_off);
        a.nxp = L.nxp;
        a.ezp = L.ezp;
        a.ra = L.ra;
        a.tiles_x = L.tiles_x;
        a.tiles = L.tiles;
        ts_taps(g.R, g.sig_xy, a);
        if (overlap && c >= 2 && (e = cudaStreamWaitEvent(st, aux->psf[b], 0)) != cudaSuccess)
            return cuda_fail(e, "split Jacobian: ordering the stages");
        gbk_status s = ts_launch_stage_r(0, tm, a, st);
        if (s) return s;
        if (overlap && ((e = cudaEventRecord(aux->line[b], st)) || (e = cudaStreamWaitEvent(sb, aux->line[b], 0))))
            return cuda_fail(e, "split Jacobian: ordering the stages");
        if ((s = ts_launch_stage_r(1, tm, a, sb))) return s;
        if (overlap && (e = cudaEventRecord(aux->psf[b], sb)) != cudaSuccess)
            return cuda_fail(e, "split Jacobian: ordering the stages");
    }
    if (overlap && (e = cudaStreamWaitEvent(st, aux->psf[(c - 1) & 1], 0)) != cudaSuccess)
        return cuda_fail(e, "split Jacobian: joining the stages");
    return GBK_OK;
}

// ---------------------------------------------------------------------------
// Ragged batches.
void tsplit_ragged_plan(const std::vector<Geom> &geo, TsRaggedPlan *p, const std::vector<char> *active)
{
    *p = TsRaggedPlan();
    const int n = (int)geo.size();
    p->n = n;
    if (n == 0) return;
    for (const Geom &g : geo) {
        if (g.model != GBK_MODEL_CUBE || g.u != 1 || g.R > kTsplitMaxR || g.ex > 1024 || ts_smem_a(g, 1) > 200 * 1024 ||
            ts_smem_b(g.R) > 200 * 1024)
            return;
    }
    // galaxies by PSF radius (the stages are compiled per radius) and PSF
    // width (a launch's taps travel in its parameters), index order within
    // those; a chunk never mixes them
    std::vector<int> ord(n);
    for (int m = 0; m < n; ++m) ord[m] = m;
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
        return geo[a].R != geo[b].R ? geo[a].R < geo[b].R : geo[a].sig_xy < geo[b].sig_xy;
    });
    p->tab_off.resize(n);
    p->ra.resize(n);
    p->tile_base.resize(n);
    p->pl_off.resize(n);
    const long long budget = (long long)(kTsL2Budget / sizeof(float));
    long long tab = 0, chunk_start = 0, cum = 0, largest = 0;
    int slots = 0;
    std::vector<int> chunk_of(n, 0);
    p->chunk_a.push_back(0);
    p->chunk_b.push_back(0);
    bool first = true;
    int prev_r = -1;
    float prev_sig = 0.f;
    for (int j = 0; j < n; ++j) {
        const int m = ord[j];
        if (active && !(*active)[m]) continue;  // no work, no planes, no part slots
        const Geom &g = geo[m];
        const int nxp = (g.nx + 3) & ~3;
        const long long planes = (long long)kTsPlanes * g.ey * nxp;
        if (!first && (g.R != prev_r || g.sig_xy != prev_sig || cum + planes - chunk_start > budget)) {
            // close the chunk before galaxy m
            p->chunk_a.push_back((int)p->work_a.size());
            p->chunk_b.push_back((int)p->work_b.size());
            p->chunk_r.push_back(prev_r);
            p->chunk_sig.push_back(prev_sig);
            chunk_start = cum;
        }
        first = false;
        prev_r = g.R;
        prev_sig = g.sig_xy;
        p->pl_off[m] = cum - chunk_start;
        chunk_of[m] = (int)p->chunk_r.size();
        largest = std::max(largest, planes);
        cum += planes;
        p->tab_off[m] = (int)tab;
        tab += (kTsTabZ + 3 * ts_ezp(g) + 3) & ~3;
        p->ra[m] = ts_rows_a(g);
        p->smem_a = std::max(p->smem_a, ts_smem_a(g, p->ra[m]));
        for (int b = 0; b * p->ra[m] < g.ey; ++b) p->work_a.push_back(make_int2(m, b));
        const int tiles = ((g.nx + kTsTX - 1) / kTsTX) * ((g.ny + kTsTY - 1) / kTsTY);
        p->tile_base[m] = slots;
        slots += tiles;
        for (int t = 0; t < tiles; ++t) p->work_b.push_back(make_int2(m, t));
    }
    if (!first) {
        p->chunk_a.push_back((int)p->work_a.size());
        p->chunk_b.push_back((int)p->work_b.size());
        p->chunk_r.push_back(prev_r);
        p->chunk_sig.push_back(prev_sig);
    }
    // A plane buffer holds any chunk: no chunk exceeds the budget unless one
    // galaxy does, nor the planes of all the active galaxies.  The bound
    // does not grow when galaxies leave the plan, so a plan over the running
    // galaxies fits the full plan's workspace.  Odd chunks use the second
    // buffer.
    const long long cap = (std::max(largest, std::min(budget, cum)) + 3) & ~3LL;  // 16-byte multiple
    p->nbuf = p->chunk_r.size() > 1 ? 2 : 1;
    if (p->nbuf == 2)
        for (int m = 0; m < n; ++m)
            if ((!active || (*active)[m]) && (chunk_of[m] & 1)) p->pl_off[m] += cap;
    size_t o = 0;
    auto take = [&](size_t bytes) { const size_t r = o; o += ts_al256(bytes); return r; };
    p->o_mcs = take(sizeof(ModelConst) * n);
    p->o_tab = take(sizeof(float) * (size_t)tab);
    p->o_pl = take(sizeof(float) * (size_t)cap * p->nbuf);
    p->o_part = take(sizeof(double) * (size_t)slots * kTsEnt);
    p->o_arr = take(sizeof(unsigned) * n);
    p->o_taboff = take(sizeof(int) * n);
    p->o_ra = take(sizeof(int) * n);
    p->o_tbase = take(sizeof(int) * n);
    p->o_ploff = take(sizeof(long long) * n);
    p->o_wa = take(sizeof(int2) * p->work_a.size());
    p->o_wb = take(sizeof(int2) * p->work_b.size());
    p->total = o;
    p->ok = true;
}

gbk_status tsplit_ragged_upload(const TsRaggedPlan &p, char *ws, cudaStream_t st)
{
    if (!p.ok) return fail(GBK_EUNSUPPORTED, "the split Jacobian does not serve this batch of geometries");
    cudaError_t e;
    if ((e = cudaMemcpyAsync(ws + p.o_taboff, p.tab_off.data(), sizeof(int) * p.n, cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(ws + p.o_ra, p.ra.data(), sizeof(int) * p.n, cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(ws + p.o_tbase, p.tile_base.data(), sizeof(int) * p.n, cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(ws + p.o_ploff, p.pl_off.data(), sizeof(long long) * p.n, cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(ws + p.o_wa, p.work_a.data(), sizeof(int2) * p.work_a.size(), cudaMemcpyHostToDevice,
                             st)) ||
        (e = cudaMemcpyAsync(ws + p.o_wb, p.work_b.data(), sizeof(int2) * p.work_b.size(), cudaMemcpyHostToDevice,
                             st)))
        return cuda_fail(e, "split Jacobian: uploading the ragged plan");
    return GBK_OK;
}

// Stage `stage` (0: line, 1: PSF) of chunk c (its galaxies share the PSF radius R).
template <int R>
static gbk_status ts_launch_ragged(const TsRaggedPlan &p, int c, int stage, TsArgs a, char *ws, cudaStream_t st)
{
    static KernelAttrMemo memo_a, memo_b;
    const size_t sb = ts_smem_b(R);
    gbk_status s;
    if ((s = ensure_kernel_attrs((const void *)tsplit_line_kernel<R, true>, p.smem_a, false, memo_a,
                                 "split Jacobian: setting the ragged line stage's shared memory")) ||
        (s = ensure_kernel_attrs((const void *)tsplit_psf_kernel<R, true>, sb, false, memo_b,
                                 "split Jacobian: setting the ragged PSF stage's shared memory")))
        return s;
    CUtensorMap none;
    std::memset(&none, 0, sizeof(none));
    const int2 *wa = (const int2 *)(ws + p.o_wa), *wb = (const int2 *)(ws + p.o_wb);
    const int na = p.chunk_a[c + 1] - p.chunk_a[c], nb = p.chunk_b[c + 1] - p.chunk_b[c];
    cudaError_t e;
    if (stage == 0 && na > 0) {
        a.work = wa + p.chunk_a[c];
        tsplit_line_kernel<R, true><<<(unsigned)na, kTsThreads, p.smem_a, st>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "split Jacobian: ragged line stage launch");
    }
    if (stage == 1 && nb > 0) {
        a.work = wb + p.chunk_b[c];
        tsplit_psf_kernel<R, true><<<(unsigned)nb, kTsThreads, sb, st>>>(none, a);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "split Jacobian: ragged PSF stage launch");
    }
    return GBK_OK;
}

gbk_status launch_tsplit_ragged(const TsRaggedPlan &p, const TsplitRaggedCall &call, char *ws, cudaStream_t st)
{
    if (!p.ok) return fail(GBK_EUNSUPPORTED, "the split Jacobian does not serve this batch of geometries");
    if (call.np < 1 || call.np > kTsNP) return fail(GBK_EUNSUPPORTED, "split Jacobian: free parameters among x0 .. sigma0");
    for (int k = 0; k < call.np; ++k)
        if (call.free_idx[k] < 0 || call.free_idx[k] >= kTsNP)
            return fail(GBK_EUNSUPPORTED, "split Jacobian: free parameters among x0 .. sigma0");
    if (p.n == 0) return GBK_OK;
    ModelConst *mcs = (ModelConst *)(ws + p.o_mcs);
    float *tab = (float *)(ws + p.o_tab);
    cudaError_t e = cudaMemsetAsync(ws + p.o_arr, 0, sizeof(unsigned) * p.n, st);
    if (e != cudaSuccess) return cuda_fail(e, "split Jacobian: clearing the arrival counters");
    tsplit_setup_ragged_kernel<<<(unsigned)p.n, 128, 0, st>>>(call.params, call.d_geo, (const int *)(ws + p.o_taboff),
                                                              call.skip, mcs, tab);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "split Jacobian: ragged set-up launch");
    TsArgs a = {};
    a.g = Geom();
    a.n_models = p.n;
    a.params = call.params;
    a.mcs = mcs;
    a.tab = tab;
    a.pl = (float *)(ws + p.o_pl);
    a.obs_list = call.obs_list;
    a.skip = call.skip;
    a.cot = nullptr;
    a.np = call.np;
    for (int k = 0; k < call.np; ++k) a.free_idx[k] = call.free_idx[k];
    a.jtj = call.jtj;
    a.jtv = call.jtv;
    a.chi2 = call.chi2;
    a.part = (double *)(ws + p.o_part);
    a.arrived = (unsigned *)(ws + p.o_arr);
    a.geo = call.d_geo;
    a.tab_off = (const int *)(ws + p.o_taboff);
    a.pl_off = (const long long *)(ws + p.o_ploff);
    a.ra_m = (const int *)(ws + p.o_ra);
    a.tile_base = (const int *)(ws + p.o_tbase);
    // chunk c's PSF stage on the auxiliary stream beside chunk c + 1's line
    // stage (plane buffer c % 2); chunk c + 2's line stage waits for it
    const int nch = (int)p.chunk_a.size() - 1;
    const bool overlap = p.nbuf == 2;
    SplitAux *aux = nullptr;
    if (overlap) {
        gbk_status s = split_aux(&aux);
        if (s) return s;
    }
    cudaStream_t sb = overlap ? aux->s : st;
    for (int c = 0; c < nch; ++c) {
        const int b = c & 1;
        if (p.chunk_r[c] > kTsplitMaxR)
            return fail(GBK_EUNSUPPORTED, "split Jacobian: PSF radius %d > %d", p.chunk_r[c], kTsplitMaxR);
        ts_taps(p.chunk_r[c], p.chunk_sig[c], a);
        if (overlap && c >= 2 && (e = cudaStreamWaitEvent(st, aux->psf[b], 0)) != cudaSuccess)
            return cuda_fail(e, "split Jacobian: ordering the stages");
        for (int stage = 0; stage < 2; ++stage) {
            cudaStream_t ss = stage == 0 ? st : sb;
            gbk_status s;
            switch (p.chunk_r[c]) {
            case 0: s = ts_launch_ragged<0>(p, c, stage, a, ws, ss); break;
            case 1: s = ts_launch_ragged<1>(p, c, stage, a, ws, ss); break;
            case 2: s = ts_launch_ragged<2>(p, c, stage, a, ws, ss); break;
            case 3: s = ts_launch_ragged<3>(p, c, stage, a, ws, ss); break;
            case 4: s = ts_launch_ragged<4>(p, c, stage, a, ws, ss); break;
            case 5: s = ts_launch_ragged<5>(p, c, stage, a, ws, ss); break;
            case 6: s = ts_launch_ragged<6>(p, c, stage, a, ws, ss); break;
            case 7: s = ts_launch_ragged<7>(p, c, stage, a, ws, ss); break;
            case 8: s = ts_launch_ragged<8>(p, c, stage, a, ws, ss); break;
            default: return fail(GBK_EUNSUPPORTED, "split Jacobian: PSF radius %d > %d", p.chunk_r[c], kTsplitMaxR);
            }
            if (s) return s;
            if (overlap && stage == 0 &&
                ((e = cudaEventRecord(aux->line[b], st)) || (e = cudaStreamWaitEvent(sb, aux->line[b], 0))))
                return cuda_fail(e, "split Jacobian: ordering the stages");
        }
        if (overlap && (e = cudaEventRecord(aux->psf[b], sb)) != cudaSuccess)
            return cuda_fail(e, "split Jacobian: ordering the stages");
    }
    if (overlap && nch > 0 && (e = cudaStreamWaitEvent(st, aux->psf[(nch - 1) & 1], 0)) != cudaSuccess)
        return cuda_fail(e, "split Jacobian: joining the stages");
    return GBK_OK;
}

}  // namespace gbk
