// k_split.cu -- the folded forward model (cube -> PSF x LSF convolution ->
// moments -> masked chi-squared, Sec. 2.2.2-2.2.6 of Bekiaris et al. 2015)
// in stages that meet in an L2-resident buffer, instead of one thread-block
// cluster per model (k_fused.cu).
//
// The arithmetic per extended spaxel is the fused evaluator's (fused_line.cuh:
// the sampled Gaussian line with the LSF convolution and the channel sums of
// the moments folded into channel weights).  The PSF passes differ in how
// they accumulate (below); the maps agree with k_fused.cu's to FP32 rounding.
//
//  set-up   (split_setup_kernel) per-model constants, the PSF taps and the
//           LSF band-edge tables, once per call, into the workspace.
//  stage A  (split_line_kernel<R>) one CTA per RA extended rows of a model:
//           every spaxel's moment triplet (q0, q1, q2, a) into shared memory
//           (four planes), then the PSF pass along x of those rows (four
//           outputs per thread from the sixteen inputs they share), written
//           as four coalesced planes [model][ey][nxp] to the buffer.  Each
//           row is sampled and filtered once: no halo is computed twice.
//  stage B  (split_psf_kernel<R>) one CTA per TY x TX tile of data spaxels:
//           the tile's TY + 2R rows of the four x-filtered planes into shared
//           memory by four TMA tile loads (cp.async.bulk.tensor, completion on
//           an mbarrier with a bounded wait: a load that does not complete
//           sets a status word and the tile is abandoned, no hang),
//           the PSF pass along y (four outputs per thread down a column),
//           the moments, residuals and the tile's part of chi2; the last CTA
//           of a model to finish (an arrival counter) adds the tile parts in
//           tile order, so chi2 is deterministic.
//
// Both passes accumulate an output's sums about its centre c (the line-of-
// sight velocity of the output spaxel, clamped into the band) from inputs
// (q0, q1, q2) about their own centres a, with D = a - c:
//   s0 += w q0,   s1 += w (q1 + a q0)  [about 0; s1 - c s0 once at the end],
//   s2 += w (q2 + D (2 q1 + D q0))     [exactly re-centred],
// six FP32 operations per tap.  The first moment about 0 costs about
// 300 km/s x 2^-24 relative of s0 in s1 (m1 within 1e-4 km/s); the second
// moment, which would cancel badly about 0, is re-centred on every tap.
//
// The models are processed in chunks whose buffer fits comfortably in L2
// (stage A of a chunk, then stage B), so it is written and read on chip.
#include <algorithm>
#include <mutex>

#include "fused_line.cuh"
#include "gbk_api_internal.h"
#include "k_split.h"
#include "tma_util.cuh"

namespace gbk {

constexpr int kSplitThreads = 256;
constexpr int kSplitMaxRA = 12;                      // most extended rows per stage-A CTA
constexpr int kSplitTX = 64, kSplitTY = 32;          // data spaxels per stage-B tile
constexpr size_t kSplitL2Budget = (size_t)48 << 20;  // buffer bytes per chunk (two buffers in flight)
constexpr int kSplitMaxEx = 1024;                    // widest extended row served
constexpr long kSplitWaitLimit = 1L << 18;           // tries: about one second (3.75 us per failed try_wait)

__device__ int g_split_status;  // 0 = fine; 1 = a tile's TMA load did not complete in time

__host__ __device__ constexpr int split_rowpitch_a(int ex) { return ((ex + 3) & ~3) + 4; }
__host__ __device__ inline int split_nxp(int nx) { return (nx + 3) & ~3; }

// Workspace tables: LSF variance, PSF taps, then the three edge tables.
constexpr int kTabTaps = 4;                          // float offset of the taps
constexpr int kTabEdge = kTabTaps + 2 * kSplitMaxR + 4;  // float offset of the edge tables
__host__ __device__ inline int split_tab_floats(const Geom &g) { return kTabEdge + 3 * edge_table_len(g); }

struct SplitArgs {
    Geom g;
    int n_models;            // models of this chunk
    const double *params;    // [n_models][GBK_NPAR]
    const ModelConst *mcs;   // [n_models] per-model constants
    const float *tab;        // split_tab_floats(g) floats
    float *pl;               // x-filtered planes, [n_models][4][ey][nxp]
    int pl_z0;               // first plane of this buffer in the PSF stage's tensor map
    gbk_obs obs;
    const gbk_obs *obs_list; // per galaxy (model m0 + i is galaxy (m0 + i) / mpg), or null: obs for all
    const int32_t *skip;     // per galaxy: non-zero = leave the galaxy's models alone (or null)
    int m0, mpg;             // first model of the chunk in the call, models per galaxy
    float *maps;             // [n_models][3][ny][nx] or null
    double *chi2;            // [n_models] or null
    float *resid;            // [n_models][2][ny][nx] or null
    double *part;            // [n_models][tiles] chi2 parts of the tiles
    unsigned *arrived;       // [n_models] tiles done (zero at the start, reset by the last)
    int nxp;                 // plane row pitch (floats)
    int ra;                  // extended rows per stage-A CTA
    int tiles_x, tiles;
};

// ---------------------------------------------------------------------------
// Set-up: per-model constants (one thread each) and, in block 0, the tables.
__global__ void split_setup_kernel(const double *params, int n, Geom g, ModelConst *mcs, float *tab)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) mcs[i] = model_const(params + (size_t)i * GBK_NPAR, g);
    if (blockIdx.x != 0) return;
    const int tid = threadIdx.x;
    if (tid == 0) tab[0] = lsf_var(g);
    if (tid <= 2 * g.R) {
        const float S = tap_sum(g.sig_xy, g.R);
        tab[kTabTaps + tid] = tap_raw(tid - g.R, g.sig_xy, g.R) / S;
    }
    const int etl = edge_table_len(g);
    float *e = tab + kTabEdge;
    edge_tables(g, e, e + etl, e + 2 * etl, tid, blockDim.x);
}

// ---------------------------------------------------------------------------
// Stage A: the moment triplets of RA extended rows, then their x pass.
template <int R>
__global__ void __launch_bounds__(kSplitThreads, 4) split_line_kernel(SplitArgs a)
{
    constexpr int W = 2 * R + 1;
    constexpr int NIN = 4 + 2 * R;        // inputs of four consecutive outputs
    constexpr int NC4 = (NIN + 3) / 4;    // ... as float4 groups
    extern __shared__ __align__(16) float sm[];
    __shared__ ModelConst mc;
    const Geom &g = a.g;
    const int tid = threadIdx.x, model = blockIdx.y;
    if (a.skip && a.skip[(a.m0 + model) / a.mpg] != 0) return;  // the whole CTA
    const int row0 = blockIdx.x * a.ra, nrows = min(a.ra, g.ey - row0);
    const int PA = split_rowpitch_a(g.ex);        // floats per plane row
    const int NPL = a.ra * PA;
    float *const Q0 = sm, *const Q1 = sm + NPL, *const Q2 = sm + 2 * NPL, *const QA = sm + 3 * NPL;
    const int etl = edge_table_len(g);
    float *const eG0 = sm + 4 * NPL, *const eA1 = eG0 + etl, *const eA2 = eA1 + etl;
    // constants and tables: copies, no arithmetic
    if (tid < (int)(sizeof(ModelConst) / 4))
        reinterpret_cast<float *>(&mc)[tid] = reinterpret_cast<const float *>(a.mcs + model)[tid];
    for (int i = tid; i < 3 * etl; i += kSplitThreads) eG0[i] = a.tab[kTabEdge + i];
    float w[W];
#pragma unroll
    for (int j = 0; j < W; ++j) w[j] = a.tab[kTabTaps + j];
    const float var_z = a.tab[0];
    __syncthreads();

    // phase 1: the line of every extended spaxel of the rows
    const LineCtx lc = line_ctx(g, mc, var_z);
    const int nsp = nrows * g.ex;
    int r = tid / g.ex, xe = tid - r * g.ex;
    const int dr = kSplitThreads / g.ex, dx = kSplitThreads - dr * g.ex;
    for (int idx = tid; idx < nsp; idx += kSplitThreads) {
        const float4 q = line_sums(g, mc, lc, eG0, eA1, eA2, (float)(xe - R), (float)(row0 + r - R));
        const int o = r * PA + xe;
        Q0[o] = q.x; Q1[o] = q.y; Q2[o] = q.z; QA[o] = q.w;
        xe += dx; r += dr;
        if (xe >= g.ex) { xe -= g.ex; ++r; }
    }
    __syncthreads();

    // phase 2: x pass; task (row, outputs 4 gx .. 4 gx + 3)
    const int ngx = (g.nx + 3) / 4;
    const size_t pstride = (size_t)g.ey * a.nxp;  // floats per plane
    float *const P0 = a.pl + (size_t)model * 4 * pstride + (size_t)row0 * a.nxp;
    for (int t = tid; t < nrows * ngx; t += kSplitThreads) {
        const int rr = t / ngx, gx = 4 * (t - rr * ngx);
        const int ro = rr * PA + gx;
        float s[4][3], cen[4];
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            cen[o] = QA[ro + o + R];
            s[o][0] = s[o][1] = s[o][2] = 0.f;
        }
        const float ref = cen[1];  // the task's reference velocity
#pragma unroll
        for (int c4 = 0; c4 < NC4; ++c4) {
            const float4 v0 = *reinterpret_cast<const float4 *>(Q0 + ro + 4 * c4);
            const float4 v1 = *reinterpret_cast<const float4 *>(Q1 + ro + 4 * c4);
            const float4 v2 = *reinterpret_cast<const float4 *>(Q2 + ro + 4 * c4);
            const float4 va = *reinterpret_cast<const float4 *>(QA + ro + 4 * c4);
            const float q0[4] = {v0.x, v0.y, v0.z, v0.w}, q1[4] = {v1.x, v1.y, v1.z, v1.w};
            const float q2[4] = {v2.x, v2.y, v2.z, v2.w}, qa[4] = {va.x, va.y, va.z, va.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int e = 4 * c4 + k;
                if (e >= NIN) break;
                float l1, l2;
                about_ref(q0[k], q1[k], q2[k], qa[k], ref, l1, l2);
#pragma unroll
                for (int o = 0; o < 4; ++o) {
                    const int j = e - o;
                    if (j >= 0 && j < W) {
                        s[o][0] = fmaf(w[j], q0[k], s[o][0]);
                        s[o][1] = fmaf(w[j], l1, s[o][1]);
                        s[o][2] = fmaf(w[j], l2, s[o][2]);
                    }
                }
            }
        }
#pragma unroll
        for (int o = 0; o < 4; ++o) shift_sums(cen[o] - ref, s[o][0], s[o][1], s[o][2]);
        float *const p = P0 + (size_t)rr * a.nxp + gx;
        *reinterpret_cast<float4 *>(p) = make_float4(s[0][0], s[1][0], s[2][0], s[3][0]);
        *reinterpret_cast<float4 *>(p + pstride) = make_float4(s[0][1], s[1][1], s[2][1], s[3][1]);
        *reinterpret_cast<float4 *>(p + 2 * pstride) = make_float4(s[0][2], s[1][2], s[2][2], s[3][2]);
        *reinterpret_cast<float4 *>(p + 3 * pstride) = make_float4(cen[0], cen[1], cen[2], cen[3]);
    }
}

// ---------------------------------------------------------------------------
// Stage B: y pass, moments, residuals and chi2 of one tile.
template <int R>
__global__ void __launch_bounds__(kSplitThreads, 4)
    split_psf_kernel(const __grid_constant__ CUtensorMap tmap, SplitArgs a)
{
    constexpr int W = 2 * R + 1;
    constexpr int NR = kSplitTY + 2 * R;  // rows of the tile's planes
    constexpr int NPL = NR * kSplitTX;    // floats per plane
    constexpr int NIN = 4 + 2 * R;
    extern __shared__ __align__(128) unsigned char sraw[];
    // TMA destinations 128-byte aligned (the allocation has 128 bytes to spare)
    float *const sp = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(sraw) + 127) & ~(uintptr_t)127);
    float *const S0 = sp, *const S1 = sp + NPL, *const S2 = sp + 2 * NPL, *const SA = sp + 3 * NPL;
    __shared__ ModelConst mc;
    __shared__ gbk_obs s_ob;
    __shared__ double red[kSplitThreads / 32];
    __shared__ bool s_last;
    __shared__ __align__(8) uint64_t bar;

    const Geom &g = a.g;
    const int tid = threadIdx.x, lane = tid & 31;
    const int model = blockIdx.y, tile = blockIdx.x;
    const int gal = (a.m0 + model) / a.mpg;
    if (a.skip && a.skip[gal] != 0) return;  // the whole CTA
    const int tx0 = (tile % a.tiles_x) * kSplitTX, ty0 = (tile / a.tiles_x) * kSplitTY;
    const int nxo = min(kSplitTX, g.nx - tx0), nyo = min(kSplitTY, g.ny - ty0);
    if (tid == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (tid == 0) {
        // the tile's rows of the four planes (beyond the buffer: zeros)
        tma_expect(&bar, (uint32_t)(4 * NPL * sizeof(float)));
#pragma unroll
        for (int pl = 0; pl < 4; ++pl) tma_load_3d(&tmap, sp + pl * NPL, &bar, tx0, ty0, a.pl_z0 + 4 * model + pl);
    }
    if (tid < (int)(sizeof(ModelConst) / 4))
        reinterpret_cast<float *>(&mc)[tid] = reinterpret_cast<const float *>(a.mcs + model)[tid];
    if (tid == 32) s_ob = a.obs_list ? a.obs_list[gal] : a.obs;
    float w[W];
#pragma unroll
    for (int j = 0; j < W; ++j) w[j] = a.tab[kTabTaps + j];
    // the same decision in every thread (and the barrier publishes mc, s_ob)
    const bool loaded = mbar_wait(&bar, 0, kSplitWaitLimit);
    if (__syncthreads_or(!loaded)) {
        if (tid == 0) {
            atomicExch(&g_split_status, 1);
            mbar_wait(&bar, 0, kSplitWaitLimit);  // a bounded chance for the copies in flight to land
        }
        return;
    }

    const ModelConst &c = mc;
    const size_t np = (size_t)g.nx * g.ny;
    const float thr = kInvalidFraction * c.i0;
    const float nanf_ = __int_as_float(0x7fc00000);
    const bool want_chi2 = (a.chi2 != nullptr), want_obs = want_chi2 || a.resid;
    KahanF acc;
    for (int t = tid; t < kSplitTX * (kSplitTY / 4); t += kSplitThreads) {
        const int x = t % kSplitTX, gy = 4 * (t / kSplitTX);
        if (x >= nxo || gy >= nyo) continue;
        // the observed values of the four outputs first: their latency
        // overlaps the y pass
        uint8_t mk[4] = {0, 0, 0, 0};
        float vo[4] = {0.f, 0.f, 0.f, 0.f}, so[4] = {0.f, 0.f, 0.f, 0.f};
        float wv[4] = {0.f, 0.f, 0.f, 0.f}, ws[4] = {0.f, 0.f, 0.f, 0.f};
        if (want_obs) {
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                if (gy + o < nyo) {
                    const size_t pix = (size_t)(ty0 + gy + o) * g.nx + (tx0 + x);
                    mk[o] = __ldg(s_ob.mask + pix);
                    vo[o] = __ldg(s_ob.v_obs + pix);
                    so[o] = __ldg(s_ob.s_obs + pix);
                    wv[o] = __ldg(s_ob.w_v + pix);
                    ws[o] = __ldg(s_ob.w_s + pix);
                }
            }
        }
        float s[4][3], cen[4];
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            cen[o] = SA[(gy + o + R) * kSplitTX + x];
            s[o][0] = s[o][1] = s[o][2] = 0.f;
        }
        const float ref = cen[1];  // the task's reference velocity
#pragma unroll
        for (int e = 0; e < NIN; ++e) {
            const int oi = (gy + e) * kSplitTX + x;
            const float q0 = S0[oi];
            float l1, l2;
            about_ref(q0, S1[oi], S2[oi], SA[oi], ref, l1, l2);
#pragma unroll
            for (int o = 0; o < 4; ++o) {
                const int j = e - o;
                if (j >= 0 && j < W) {
                    s[o][0] = fmaf(w[j], q0, s[o][0]);
                    s[o][1] = fmaf(w[j], l1, s[o][1]);
                    s[o][2] = fmaf(w[j], l2, s[o][2]);
                }
            }
        }
#pragma unroll
        for (int o = 0; o < 4; ++o) shift_sums(cen[o] - ref, s[o][0], s[o][1], s[o][2]);
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            const int yl = gy + o;
            if (yl >= nyo) break;
            const size_t pix = (size_t)(ty0 + yl) * g.nx + (tx0 + x);
            const float s0 = s[o][0], s1 = s[o][1], s2 = s[o][2];
            float m0, m1, m2;
            const bool valid = s0 > thr;
            if (!c.valid) {
                m0 = m1 = m2 = nanf_;
            } else if (valid) {
                const float inv = __frcp_rn(s0);
                const float mu = s1 * inv;
                const float var = fmaf(-mu, mu, s2 * inv);
                m0 = s0;
                m1 = cen[o] + mu;
                m2 = sqrtf(fmaxf(var, 0.f));
            } else {
                m0 = 0.f; m1 = c.vsys; m2 = 0.f;
            }
            if (a.maps) {
                float *mp = a.maps + 3 * (size_t)model * np;
                mp[pix] = m0; mp[np + pix] = m1; mp[2 * np + pix] = m2;
            }
            if (want_obs) {
                float rv = 0.f, rs = 0.f;
                if (mk[o] != 0 && (valid || !c.valid)) {
                    rv = wv[o] * (m1 - vo[o]);
                    rs = ws[o] * (m2 - so[o]);
                }
                acc.add(rv * rv);
                acc.add(rs * rs);
                if (a.resid) {
                    float *rp = a.resid + 2 * (size_t)model * np;
                    rp[pix] = rv; rp[np + pix] = rs;
                }
            }
        }
    }
    if (!want_chi2) return;
    // the tile's part, then the model's total from the last tile to finish
    // each warp's sum in FP32 (the compensated per-thread sums, a fixed
    // shuffle tree), the warps and tiles in FP64
    float v = acc.s - acc.c;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) red[tid >> 5] = (double)v;
    __syncthreads();
    if (tid == 0) {
        double sum = 0.0;
        for (int k = 0; k < kSplitThreads / 32; ++k) sum += red[k];
        a.part[(size_t)model * a.tiles + tile] = sum;
        __threadfence();
        const unsigned prev = atomicAdd(&a.arrived[model], 1u);
        s_last = (prev == (unsigned)a.tiles - 1);
    }
    __syncthreads();
    if (s_last && tid == 0) {
        __threadfence();
        const volatile double *p = a.part + (size_t)model * a.tiles;
        double sum = 0.0;
        for (int k = 0; k < a.tiles; ++k) sum += p[k];
        a.chi2[model] = c.valid ? sum : (double)nanf_;
        a.arrived[model] = 0u;  // ready for the next chunk or call
    }
}

// ---------------------------------------------------------------------------
// Host side.
SplitEncodeFn split_encode_fn()
{
    static SplitEncodeFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, []() {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (SplitEncodeFn)p;
    });
    return fn;
}

struct SplitLayout {
    int chunk, nbuf, nxp, tiles_x, tiles;
    size_t mc_off, tab_off, pl_off, pl_bytes, part_off, arr_off, total;  // pl_bytes: one buffer
};

static size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

static SplitLayout split_layout(const Geom &g, int n_models)
{
    SplitLayout L = {};
    L.nxp = split_nxp(g.nx);
    const size_t plb = (size_t)4 * g.ey * L.nxp * sizeof(float);
    size_t chunk = kSplitL2Budget / plb;
    if (chunk < 1) chunk = 1;
    if (chunk > (size_t)n_models) chunk = (size_t)n_models;
    const size_t nchunks = ((size_t)n_models + chunk - 1) / chunk;
    chunk = ((size_t)n_models + nchunks - 1) / nchunks;  // balanced chunks
    L.chunk = (int)chunk;
    L.nbuf = (size_t)n_models > chunk ? 2 : 1;  // chunk k + 1's line stage runs beside chunk k's PSF stage
    L.tiles_x = (g.nx + kSplitTX - 1) / kSplitTX;
    L.tiles = L.tiles_x * ((g.ny + kSplitTY - 1) / kSplitTY);
    L.mc_off = 0;
    L.tab_off = al256((size_t)n_models * sizeof(ModelConst));
    L.pl_off = L.tab_off + al256((size_t)split_tab_floats(g) * sizeof(float));
    L.pl_bytes = chunk * plb;  // a multiple of 16 bytes (nxp is a multiple of 4)
    L.part_off = L.pl_off + al256(L.nbuf * L.pl_bytes);
    L.arr_off = L.part_off + al256(chunk * L.tiles * sizeof(double));
    L.total = L.arr_off + al256(chunk * sizeof(unsigned));
    return L;
}

static size_t split_smem_a(const Geom &g, int ra)
{
    return (size_t)(4 * ra * split_rowpitch_a(g.ex) + 3 * edge_table_len(g)) * sizeof(float);
}

// Extended rows per stage-A CTA: the count (up to kSplitMaxRA, within a
// shared-memory target that keeps four CTAs per SM) with the least cost per
// row, counting whole rounds of the CTA's threads in the line sums (about
// 580 warp instructions a round) and in the x pass (about 330); the larger
// count on a tie.
static int split_rows_a(const Geom &g)
{
    const int ngx = (g.nx + 3) / 4;
    int best_ra = 1;
    double best = 1e30;
    for (int ra = 1; ra <= kSplitMaxRA; ++ra) {
        if (ra > 1 && split_smem_a(g, ra) > (size_t)56 * 1024) break;
        const int r1 = (ra * g.ex + kSplitThreads - 1) / kSplitThreads;
        const int r2 = (ra * ngx + kSplitThreads - 1) / kSplitThreads;
        const double cost = (580.0 * r1 + 330.0 * r2) / ra;
        if (cost <= best * (1.0 + 1e-9)) {
            best = cost;
            best_ra = ra;
        }
    }
    return best_ra;
}

static size_t split_smem_b(int R) { return 128 + (size_t)4 * (kSplitTY + 2 * R) * kSplitTX * sizeof(float); }

bool split_supported(const Geom &g)
{
    return g.model == GBK_MODEL_CUBE && g.u == 1 && g.R <= kSplitMaxR && g.ex <= kSplitMaxEx &&
           split_smem_a(g, 1) <= 200 * 1024;
}

size_t split_workspace_bytes(const Geom &g, int n_models)
{
    if (!split_supported(g) || n_models < 1) return 0;
    return split_layout(g, n_models).total;
}

gbk_status split_status_read(int *v)
{
    int zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(v, g_split_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_split_status, &zero, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "reading the split evaluator's status");
    return GBK_OK;
}

template <int R>
static gbk_status launch_stage(int stage, const CUtensorMap &tm, const SplitArgs &a, cudaStream_t st)
{
    static KernelAttrMemo memo_a, memo_b;
    const size_t sa = split_smem_a(a.g, a.ra), sb = split_smem_b(R);
    gbk_status s;
    if ((s = ensure_kernel_attrs((const void *)split_line_kernel<R>, sa, false, memo_a,
                                 "split evaluator: setting the line stage's shared memory")) ||
        (s = ensure_kernel_attrs((const void *)split_psf_kernel<R>, sb, false, memo_b,
                                 "split evaluator: setting the PSF stage's shared memory")))
        return s;
    cudaError_t e;
    if (stage == 0) {
        const unsigned blocks_a = (unsigned)((a.g.ey + a.ra - 1) / a.ra);
        split_line_kernel<R><<<dim3(blocks_a, (unsigned)a.n_models), kSplitThreads, sa, st>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "split evaluator: line stage launch");
    } else {
        split_psf_kernel<R><<<dim3((unsigned)a.tiles, (unsigned)a.n_models), kSplitThreads, sb, st>>>(tm, a);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "split evaluator: PSF stage launch");
    }
    return GBK_OK;
}

static gbk_status launch_stage_r(int stage, const CUtensorMap &tm, const SplitArgs &a, cudaStream_t st)
{
    switch (a.g.R) {
    case 0: return launch_stage<0>(stage, tm, a, st);
    case 1: return launch_stage<1>(stage, tm, a, st);
    case 2: return launch_stage<2>(stage, tm, a, st);
    case 3: return launch_stage<3>(stage, tm, a, st);
    case 4: return launch_stage<4>(stage, tm, a, st);
    case 5: return launch_stage<5>(stage, tm, a, st);
    case 6: return launch_stage<6>(stage, tm, a, st);
    case 7: return launch_stage<7>(stage, tm, a, st);
    case 8: return launch_stage<8>(stage, tm, a, st);
    default: return fail(GBK_EUNSUPPORTED, "split evaluator: PSF radius %d > %d", a.g.R, kSplitMaxR);
    }
}

gbk_status split_aux(SplitAux **out)
{
    constexpr int kMaxDev = 64;
    thread_local SplitAux aux[kMaxDev];
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "split evaluator: current device");
    if (dev < 0 || dev >= kMaxDev) return fail(GBK_EUNSUPPORTED, "split evaluator: device ordinal %d", dev);
    SplitAux &x = aux[dev];
    if (!x.s) {
        SplitAux y;
        if ((e = cudaStreamCreateWithFlags(&y.s, cudaStreamNonBlocking)) ||
            (e = cudaEventCreateWithFlags(&y.line[0], cudaEventDisableTiming)) ||
            (e = cudaEventCreateWithFlags(&y.line[1], cudaEventDisableTiming)) ||
            (e = cudaEventCreateWithFlags(&y.psf[0], cudaEventDisableTiming)) ||
            (e = cudaEventCreateWithFlags(&y.psf[1], cudaEventDisableTiming)) ||
            (e = cudaEventCreateWithFlags(&y.start, cudaEventDisableTiming)) ||
            (e = cudaEventCreateWithFlags(&y.obs, cudaEventDisableTiming)))
            return cuda_fail(e, "split evaluator: creating the PSF stages' stream");
        x = y;
    }
    *out = &x;
    return GBK_OK;
}

gbk_status launch_split(const Geom &g, int n, const double *params, const gbk_obs *obs, float *maps, double *chi2,
                        float *resid, void *ws, size_t ws_bytes, cudaStream_t st, SplitTimer *timer,
                        const SplitBatch *batch, cudaEvent_t obs_ready)
{
    if (batch && batch->mpg < 1) return fail(GBK_EINVAL, "split evaluator: models per galaxy must be >= 1");
    if ((chi2 || resid) && !obs && !(batch && batch->obs_list))
        return fail(GBK_EINVAL, "split evaluator: chi2 and residuals need observed maps");
    if (!split_supported(g)) return fail(GBK_EUNSUPPORTED, "the split evaluator does not serve this geometry");
    if (n == 0) return GBK_OK;
    const SplitLayout L = split_layout(g, n);
    const int ra = split_rows_a(g);
    if (!ws || ws_bytes < L.total)
        return fail(GBK_EWORKSPACE, "the split evaluator needs %zu bytes of workspace (got %zu)", L.total, ws_bytes);
    char *base = (char *)ws;
    ModelConst *mcs = (ModelConst *)(base + L.mc_off);
    float *tab = (float *)(base + L.tab_off);
    cudaError_t e = cudaSuccess;
    if (chi2) {
        e = cudaMemsetAsync(base + L.arr_off, 0, (size_t)L.chunk * sizeof(unsigned), st);
        if (e != cudaSuccess) return cuda_fail(e, "split evaluator: clearing the arrival counters");
    }
    // the buffers' planes as one 3-D tensor [nbuf * 4 * chunk][ey][nxp] for the PSF stage's tile loads
    CUtensorMap tm;
    if (!split_encode_fn()) return fail(GBK_EUNSUPPORTED, "cuTensorMapEncodeTiled is not available from the driver");
    {
        const cuuint64_t dims[3] = {(cuuint64_t)L.nxp, (cuuint64_t)g.ey, (cuuint64_t)4 * L.chunk * L.nbuf};
        const cuuint64_t strides[2] = {(cuuint64_t)L.nxp * sizeof(float), (cuuint64_t)L.nxp * g.ey * sizeof(float)};
        const cuuint32_t box[3] = {(cuuint32_t)kSplitTX, (cuuint32_t)(kSplitTY + 2 * g.R), 1};
        const cuuint32_t estr[3] = {1, 1, 1};
        CUresult r = split_encode_fn()(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base + L.pl_off, dims, strides, box,
                                       estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                       CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(GBK_ECUDA, "split evaluator: cuTensorMapEncodeTiled failed (%d)", (int)r);
    }
    if (timer && (e = timer->mark(st)) != cudaSuccess) return cuda_fail(e, "split evaluator: timing event");
    split_setup_kernel<<<(n + 127) / 128, 128, 0, st>>>(params, n, g, mcs, tab);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "split evaluator: set-up launch");
    if (timer && (e = timer->mark(st)) != cudaSuccess) return cuda_fail(e, "split evaluator: timing event");
    const size_t np = (size_t)g.nx * g.ny;
    // Two plane buffers: chunk c fills buffer c % 2, so chunk c + 1's line
    // stage (caller's stream) can run while chunk c's PSF stage (the
    // auxiliary stream) reads the other buffer; chunk c + 2's line stage
    // waits for chunk c's PSF stage.  Timed runs keep one stream.
    const bool overlap = !timer && L.nbuf == 2;
    SplitAux *aux = nullptr;
    if (overlap) {
        gbk_status s = split_aux(&aux);
        if (s) return s;
    }
    cudaStream_t sb = overlap ? aux->s : st;
    int c = 0;
    for (int m0 = 0; m0 < n; m0 += L.chunk, ++c) {
        const int b = c & (L.nbuf - 1);
        SplitArgs a = {};
        a.g = g;
        a.n_models = std::min(L.chunk, n - m0);
        a.params = params + (size_t)m0 * GBK_NPAR;
        a.mcs = mcs + m0;
        a.tab = tab;
        a.pl = (float *)(base + L.pl_off + (size_t)b * L.pl_bytes);
        a.pl_z0 = 4 * L.chunk * b;
        if (obs) a.obs = *obs;
        a.obs_list = batch ? batch->obs_list : nullptr;
        a.skip = batch ? batch->skip : nullptr;
        a.m0 = m0;
        a.mpg = batch ? batch->mpg : 1;
        a.maps = maps ? maps + 3 * np * m0 : nullptr;
        a.chi2 = chi2 ? chi2 + m0 : nullptr;
        a.resid = resid ? resid + 2 * np * m0 : nullptr;
        a.part = (double *)(base + L.part_off);
        a.arrived = (unsigned *)(base + L.arr_off);
        a.nxp = L.nxp;
        a.ra = ra;
        a.tiles_x = L.tiles_x;
        a.tiles = L.tiles;
        if (overlap && c >= 2 && (e = cudaStreamWaitEvent(st, aux->psf[b], 0)) != cudaSuccess)
            return cuda_fail(e, "split evaluator: ordering the stages");
        gbk_status s = launch_stage_r(0, tm, a, st);
        if (s) return s;
        if (timer && (e = timer->mark(st)) != cudaSuccess) return cuda_fail(e, "split evaluator: timing event");
        if (overlap && ((e = cudaEventRecord(aux->line[b], st)) || (e = cudaStreamWaitEvent(sb, aux->line[b], 0))))
            return cuda_fail(e, "split evaluator: ordering the stages");
        if (obs_ready && c == 0 && (e = cudaStreamWaitEvent(sb, obs_ready, 0)) != cudaSuccess)
            return cuda_fail(e, "split evaluator: waiting for the observed maps");
        if ((s = launch_stage_r(1, tm, a, sb))) return s;
        if (timer && (e = timer->mark(st)) != cudaSuccess) return cuda_fail(e, "split evaluator: timing event");
        if (overlap && (e = cudaEventRecord(aux->psf[b], sb)) != cudaSuccess)
            return cuda_fail(e, "split evaluator: ordering the stages");
    }
    if (overlap && (e = cudaStreamWaitEvent(st, aux->psf[(c - 1) & 1], 0)) != cudaSuccess)
        return cuda_fail(e, "split evaluator: joining the stages");
    return GBK_OK;
}

}  // namespace gbk

using namespace gbk;

extern "C" gbk_status gbk_split_stage_times(const gbk_geom *gin, int32_t n_models, const double *params,
                                            const gbk_obs *obs, double *chi2, void *workspace, size_t ws_bytes,
                                            float *stage_ms, int32_t *launches, void *stream)
{
    Geom g;
    gbk_status s = derive_geom(gin, &g);
    if (s) return s;
    if (n_models < 1) return fail(GBK_EINVAL, "n_models must be >= 1");
    if (!stage_ms) return fail(GBK_EINVAL, "stage_ms is NULL");
    if ((s = check_device_ptr(params, "params", 8)) || (s = check_device_ptr(chi2, "chi2", 8)) || (s = check_obs(obs)))
        return s;
    if (workspace && (s = check_device_ptr(workspace, "workspace", 256))) return s;
    cudaStream_t st = (cudaStream_t)stream;
    SplitTimer timer;
    s = launch_split(g, n_models, params, obs, nullptr, chi2, nullptr, workspace, ws_bytes, st, &timer);
    cudaError_t e = cudaSuccess;
    if (!s && timer.n > 0) e = cudaEventSynchronize(timer.ev[timer.n - 1]);
    if (!s && e == cudaSuccess) {
        // events: start, after set-up, then after each stage A and stage B launch
        stage_ms[0] = stage_ms[1] = stage_ms[2] = 0.f;
        for (int i = 1; i < timer.n && e == cudaSuccess; ++i) {
            float ms = 0.f;
            e = cudaEventElapsedTime(&ms, timer.ev[i - 1], timer.ev[i]);
            stage_ms[i == 1 ? 0 : ((i % 2 == 0) ? 1 : 2)] += ms;
        }
        if (launches) *launches = timer.n - 1;
    }
    timer.release();
    if (s) return s;
    if (e != cudaSuccess) return cuda_fail(e, "split stage times");
    return ok();
}
