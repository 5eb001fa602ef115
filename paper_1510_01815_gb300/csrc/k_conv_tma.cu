// k_conv_tma.cu -- the staged separable PSF x LSF convolution (Eq. 9,
// Sec. 2.2.3), built for HBM bandwidth.
//
// One CTA owns a 32 x 32 tile of output spaxels of one model and walks every
// extended channel once:
//   - TMA (cp.async.bulk.tensor, mbarrier completion) loads the tile's input
//     slab of each channel, (32 + 2R) rows x (32 + 2R, rounded to 4) columns,
//     two channels ahead, into a double buffer, so the cube is read from HBM
//     exactly once and the load overlaps the arithmetic;
//   - the x pass gives each thread four adjacent outputs from one float4-
//     loaded row segment; the y pass gives each thread four outputs of one
//     column;
//   - the z pass keeps, per owned spaxel, the 2 Rz + 1 partial output
//     channels the current input channel contributes to in registers (a
//     shifting window, template-sized), and writes a channel as soon as its
//     window is complete -- coalesced rows of 32 floats.
// Waits on the mbarriers are bounded: a CTA that gives up records a status in
// g_conv_status and stops (the host reports it as GBK_ECUDA via
// gbk_device_status()).
#include <cuda.h>

#include "gbk_api_internal.h"
#include "gbk_internal.cuh"
#include "k_staged.h"
#include "tma_util.cuh"

namespace gbk {

constexpr int kCT = 32;            // output tile edge
constexpr int kCThreads = 256;     // 8 warps
constexpr long kWaitLimit = 1L << 18;  // tries: about one second (3.75 us per failed try_wait)

__device__ int g_conv_status;      // 0 = fine; 1 = a TMA wait timed out

struct ConvTmaArgs {
    Geom g;
    int n_models;
    int tiles_x, tiles_y;
    int box_w;                     // TMA box width, >= 32 + 2R, multiple of 4
    float *fine;                   // [n][nzf][nyf][nxf]
    size_t f_model_stride;
};

template <int W>
__global__ void __launch_bounds__(kCThreads, (W <= 15 ? 2 : 1)) conv3d_tma_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                 ConvTmaArgs a)
{
    const Geom &g = a.g;
    const int R = g.R, Rz = g.Rz;
    const int SY = kCT + 2 * R, BW = a.box_w;
    const int tiles = a.tiles_x * a.tiles_y;
    const int model = blockIdx.x / tiles;
    const int t = blockIdx.x - model * tiles;
    const int ty0 = (t / a.tiles_x) * kCT, tx0 = (t % a.tiles_x) * kCT;
    const int tid = threadIdx.x;

    // A tensor copy's shared-memory destination must be 128-byte aligned: the
    // base is rounded up by hand (the launch adds 128 bytes for that) and each
    // slab is padded to a multiple of 32 floats.
    extern __shared__ __align__(128) float csm_raw[];
    float *csm = csm_raw + (((128u - (smem_u32(csm_raw) & 127u)) & 127u) >> 2);
    const int SS = (SY * BW + 31) & ~31;
    float *slab0 = csm;                        // [SY][BW]
    float *slab1 = slab0 + SS;
    float *X = slab1 + SS;                     // [SY][32] after the x pass
    float *wxy = X + SY * kCT;                 // 2R+1 taps (padded)
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ float s_wz[W];
    __shared__ int s_abort;

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    // taps (each thread that writes one computes the normalisation itself)
    for (int j = tid; j <= 2 * R; j += kCThreads) {
        float s = 0.f;
        for (int q = -R; q <= R; ++q) s += (R == 0) ? 1.f : gauss_tap(q, g.sig_xy);
        wxy[j] = ((R == 0) ? 1.f : gauss_tap(j - R, g.sig_xy)) / s;
    }
    if (tid < W) {
        float s = 0.f;
        for (int q = -Rz; q <= Rz; ++q) s += (Rz == 0) ? 1.f : gauss_tap(q, g.sig_z);
        s_wz[tid] = ((Rz == 0) ? 1.f : gauss_tap(tid - Rz, g.sig_z)) / s;
    }
    __syncthreads();

    const uint32_t bytes = (uint32_t)(SY * BW * sizeof(float));
    const int zbase = model * g.ez;
    if (tid == 0) {
        tma_load_slab(&tmap, slab0, &bar[0], tx0, ty0, zbase, bytes);
        if (g.ez > 1) tma_load_slab(&tmap, slab1, &bar[1], tx0, ty0, zbase + 1, bytes);
    }
    float wz[W];
#pragma unroll
    for (int q = 0; q < W; ++q) wz[q] = s_wz[q];

    // y-pass / z-pass ownership: column c, rows 4 gq .. 4 gq + 3
    const int c = tid & 31, gq = tid >> 5;
    float acc[4][W];
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < W; ++q) acc[p][q] = 0.f;
    float *F = a.fine + (size_t)model * a.f_model_stride;
    const size_t fplane = (size_t)g.nyf * g.nxf;
    const int ox = tx0 + c;
    const int nitems = SY * (kCT / 4);  // x pass: (row, 4-column group)

    for (int e = 0; e < g.ez; ++e) {
        float *slab = (e & 1) ? slab1 : slab0;
        if (!mbar_wait(&bar[e & 1], (uint32_t)((e >> 1) & 1), kWaitLimit)) {
            if (atomicExch(&s_abort, 1) == 0) atomicExch(&g_conv_status, 1);
        }
        __syncthreads();
        if (s_abort) {
            // give the other buffer's copy, if one is in flight, a bounded
            // chance to land before the CTA leaves
            if (tid == 0 && e + 1 < g.ez) mbar_wait(&bar[(e + 1) & 1], (uint32_t)(((e + 1) >> 1) & 1), kWaitLimit);
            return;  // every thread sees the same flag after the barrier
        }
        // x pass: X[r][4 m .. 4 m + 3] from slab[r][4 m .. 4 m + 3 + 2R]
        for (int it = tid; it < nitems; it += kCThreads) {
            int r = it >> 3, m = it & 7;
            const float *row = slab + r * BW + 4 * m;
            float o0 = 0.f, o1 = 0.f, o2 = 0.f, o3 = 0.f;
            float v0 = row[0], v1 = row[1], v2 = row[2];
            for (int j = 0; j <= 2 * R; ++j) {
                float v3 = row[j + 3];
                float w = wxy[j];
                o0 = fmaf(w, v0, o0);
                o1 = fmaf(w, v1, o1);
                o2 = fmaf(w, v2, o2);
                o3 = fmaf(w, v3, o3);
                v0 = v1; v1 = v2; v2 = v3;
            }
            *reinterpret_cast<float4 *>(X + r * kCT + 4 * m) = make_float4(o0, o1, o2, o3);
        }
        __syncthreads();
        // the slab is consumed: refill it with channel e + 2
        if (tid == 0 && e + 2 < g.ez) tma_load_slab(&tmap, slab, &bar[e & 1], tx0, ty0, zbase + e + 2, bytes);
        // y pass: rows 4 gq .. 4 gq + 3 of column c
        float y0 = 0.f, y1 = 0.f, y2 = 0.f, y3 = 0.f;
        {
            const float *col = X + (4 * gq) * kCT + c;
            float v0 = col[0], v1 = col[kCT], v2 = col[2 * kCT];
            for (int j = 0; j <= 2 * R; ++j) {
                float v3 = col[(j + 3) * kCT];
                float w = wxy[j];
                y0 = fmaf(w, v0, y0);
                y1 = fmaf(w, v1, y1);
                y2 = fmaf(w, v2, y2);
                y3 = fmaf(w, v3, y3);
                v0 = v1; v1 = v2; v2 = v3;
            }
        }
        // z pass: slot q holds output channel e - 2 Rz + q, weight wz[q]
        float yv[4] = {y0, y1, y2, y3};
#pragma unroll
        for (int p = 0; p < 4; ++p) {
#pragma unroll
            for (int q = 0; q < W; ++q) acc[p][q] = fmaf(wz[q], yv[p], acc[p][q]);
        }
        int k = e - 2 * Rz;
        if (k >= 0 && ox < g.nxf) {
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                int oy = ty0 + 4 * gq + p;
                if (oy < g.nyf) F[(size_t)k * fplane + (size_t)oy * g.nxf + ox] = acc[p][0];
            }
        }
#pragma unroll
        for (int p = 0; p < 4; ++p) {
#pragma unroll
            for (int q = 0; q + 1 < W; ++q) acc[p][q] = acc[p][q + 1];
            acc[p][W - 1] = 0.f;
        }
        // X is rewritten by the next x pass
        __syncthreads();
    }
}

// ----------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

size_t conv_tma_smem_bytes(const Geom &g)
{
    int SY = kCT + 2 * g.R, BW = (kCT + 2 * g.R + 3) & ~3;
    int SS = (SY * BW + 31) & ~31;
    return 128 + sizeof(float) * (size_t)(2 * SS + SY * kCT + ((2 * g.R + 1 + 3) & ~3));
}

bool conv_tma_supported(const Geom &g)
{
    int W = 2 * g.Rz + 1;
    return W <= 23 && (kCT + 2 * g.R) <= 256 && conv_tma_smem_bytes(g) <= 200 * 1024 && encode_fn() != nullptr;
}

template <int W>
static gbk_status launch_w(const CUtensorMap &tm, const ConvTmaArgs &a, size_t smem, int blocks, cudaStream_t st)
{
    static KernelAttrMemo memo;
    gbk_status s = ensure_kernel_attrs((const void *)conv3d_tma_kernel<W>, smem, false, memo,
                                       "TMA convolution: setting dynamic shared memory");
    if (s) return s;
    conv3d_tma_kernel<W><<<blocks, kCThreads, smem, st>>>(tm, a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "TMA convolution launch");
    return GBK_OK;
}

gbk_status launch_conv_tma(const StagedArgs &sa, cudaStream_t st)
{
    const Geom &g = sa.g;
    EncodeTiledFn enc = encode_fn();
    if (!enc) return fail(GBK_EUNSUPPORTED, "cuTensorMapEncodeTiled is not available from the driver");
    ConvTmaArgs a = {};
    a.g = g;
    a.n_models = sa.n_models;
    a.tiles_x = (g.nxf + kCT - 1) / kCT;
    a.tiles_y = (g.nyf + kCT - 1) / kCT;
    a.box_w = (kCT + 2 * g.R + 3) & ~3;
    a.fine = sa.fine;
    a.f_model_stride = sa.f_model_stride;
    CUtensorMap tm;
    cuuint64_t dims[3] = {(cuuint64_t)sa.e_pitch, (cuuint64_t)g.ey, (cuuint64_t)g.ez * (cuuint64_t)sa.n_models};
    cuuint64_t strides[2] = {(cuuint64_t)sa.e_pitch * sizeof(float), (cuuint64_t)sa.e_pitch * g.ey * sizeof(float)};
    cuuint32_t box[3] = {(cuuint32_t)a.box_w, (cuuint32_t)(kCT + 2 * g.R), 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void *)sa.ext, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(GBK_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    size_t smem = conv_tma_smem_bytes(g);
    int blocks = a.tiles_x * a.tiles_y * sa.n_models;
    switch (2 * g.Rz + 1) {
    case 1: return launch_w<1>(tm, a, smem, blocks, st);
    case 3: return launch_w<3>(tm, a, smem, blocks, st);
    case 5: return launch_w<5>(tm, a, smem, blocks, st);
    case 7: return launch_w<7>(tm, a, smem, blocks, st);
    case 9: return launch_w<9>(tm, a, smem, blocks, st);
    case 11: return launch_w<11>(tm, a, smem, blocks, st);
    case 13: return launch_w<13>(tm, a, smem, blocks, st);
    case 15: return launch_w<15>(tm, a, smem, blocks, st);
    case 17: return launch_w<17>(tm, a, smem, blocks, st);
    case 19: return launch_w<19>(tm, a, smem, blocks, st);
    case 21: return launch_w<21>(tm, a, smem, blocks, st);
    case 23: return launch_w<23>(tm, a, smem, blocks, st);
    default: return fail(GBK_EUNSUPPORTED, "LSF window %d not served by the TMA convolution", 2 * g.Rz + 1);
    }
}

gbk_status conv_status_read(int *v)
{
    int zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(v, g_conv_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_conv_status, &zero, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "reading the convolution status");
    return GBK_OK;
}

}  // namespace gbk
