// k_conv_fir.cu -- the staged separable PSF x LSF convolution (Eq. 9,
// Sec. 2.2.3) with the LSF pass as a register FIR filter along z, for PSF
// and LSF radii up to 8 (one template instance per pair of radii, so every
// tap loop is fully unrolled).
//
// One CTA of 256 threads owns a 64 x 16 tile of output spaxels of one model
// and streams the extended channels once:
//   - TMA loads each channel's (64 + 2R) x (16 + 2R) input slab into a ring
//     of kFStages buffers, kFStages - 1 channels ahead (bounded mbarrier
//     waits by one thread, status word instead of a hang);
//   - pass 1 (PSF along y) on column PAIRS of the slab: one 8-byte load and
//     one packed FMA per tap for two outputs, four rows per task; the rows
//     go to a double buffer as row pairs, even columns in one half of a row
//     and odd columns in the other, so that the 8-byte accesses of both
//     passes are consecutive across a warp;
//   - pass 2 (PSF along x) on ROW pairs of that buffer: every thread owns
//     two adjacent columns and two rows of the tile for the whole channel
//     walk (2 R + 2 loads for four outputs);
//   - pass 3 (LSF along z) never touches shared memory: each thread keeps
//     the 2 Rz partial sums of the output channels its incoming x-y-filtered
//     values still feed (a transposed FIR: the value of extended channel e
//     finishes output channel e - 2 Rz and starts channel e), one packed FMA
//     per tap, and writes each finished channel coalesced.
// The taps travel in the kernel parameters (host-computed, normalised), so
// the FMAs read them from the constant bank instead of registers.  One
// block barrier per channel, between pass 1 and pass 2; the double buffer
// lets pass 1 of the next channel overlap pass 2 of this one.  The separable
// passes are exact in real arithmetic in any order; here y, x, z.
#include <cmath>
#include <cstring>

#include <cuda.h>

#include "gbk_api_internal.h"
#include "gbk_internal.cuh"
#include "k_split.h"
#include "k_staged.h"
#include "tma_util.cuh"

namespace gbk {

constexpr int kFTX = 64, kFTY = 16;     // output tile
constexpr int kFThreads = 256;
constexpr int kFRmax = 8, kFRzMax = 8;  // largest PSF and LSF radii served
constexpr int kFStages = 6;             // slabs in flight
constexpr long kFWaitLimit = 1L << 18;  // tries: about one second

__device__ int g_conv_fir_status;  // 0 fine; 1 a TMA wait timed out

struct ConvFirArgs {
    Geom g;
    int tiles_x, tiles_y;
    float *fine;
    size_t f_model_stride;
    f32x2 w2[2 * kFRmax + 1];    // PSF taps (w, w), normalised
    f32x2 wz2[2 * kFRzMax + 1];  // LSF taps (w, w), normalised
};

template <int R>
struct FirDims {
    static constexpr int SY = kFTY + 2 * R;          // slab rows
    static constexpr int C1W = kFTX + 2 * R;         // pass-1 columns (even)
    static constexpr int C1P = C1W / 2;              // ... as pairs
    static constexpr int BW = (C1W + 3) & ~3;        // slab row pitch: the box width, 16-byte rows
    static constexpr int SS = (SY * BW + 31) & ~31;  // floats per slab (128-byte multiple)
    static constexpr int OH = C1P + 1;               // odd columns' offset in a buffer row pair (pairs)
    static constexpr int P1 = 2 * C1P + 2;           // pair pitch of a buffer row pair
    static constexpr int Y1F = (kFTY / 2) * P1 * 2;  // floats per pass-1 buffer
    static constexpr int T1 = (kFTY / 4) * C1P;      // pass-1 tasks (4 rows x a column pair)
};

__host__ __device__ constexpr size_t conv_fir_smem(int R)
{
    return 128 + sizeof(float) * ((size_t)kFStages * (((kFTY + 2 * R) * ((kFTX + 2 * R + 3) & ~3) + 31) & ~31) +
                                  (size_t)2 * (kFTY / 2) * (2 * ((kFTX + 2 * R) / 2) + 2) * 2);
}

__device__ __forceinline__ f32x2 fld2(const float *p) { return *reinterpret_cast<const f32x2 *>(p); }

// Three CTAs per SM (80 registers) where the FIR state allows it.
__host__ __device__ constexpr int conv_fir_min_blocks(int RZ) { return RZ >= 8 ? 2 : 3; }

template <int R, int RZ>
__global__ void __launch_bounds__(kFThreads, conv_fir_min_blocks(RZ))
    conv3d_fir_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ ConvFirArgs a)
{
    using D = FirDims<R>;
    constexpr int NPZ = (RZ > 0) ? 2 * RZ : 1;
    const Geom &g = a.g;
    const int tiles = a.tiles_x * a.tiles_y;
    const int model = blockIdx.x / tiles;
    const int tt = blockIdx.x - model * tiles;
    const int ty0 = (tt / a.tiles_x) * kFTY, tx0 = (tt % a.tiles_x) * kFTX;
    const int tid = threadIdx.x;

    extern __shared__ __align__(128) float fsm_raw[];
    // 128-byte aligned tensor-copy destinations (the launch adds 128 bytes)
    float *const fsm = fsm_raw + (((128u - (smem_u32(fsm_raw) & 127u)) & 127u) >> 2);
    float *const slabs = fsm;                    // [kFStages][SS]
    float *const Y1 = slabs + kFStages * D::SS;  // [2][rows / 2][P1][2]
    __shared__ __align__(8) uint64_t bar[kFStages];

    const uint32_t bytes = (uint32_t)(D::SY * D::BW * sizeof(float));
    const int zbase = model * g.ez;
    bool ok = true;
    if (tid == 0) {
#pragma unroll
        for (int s = 0; s < kFStages; ++s) mbar_init(&bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int s = 0; s < kFStages && s < g.ez; ++s)
            tma_load_slab(&tmap, slabs + s * D::SS, &bar[s], tx0, ty0, zbase + s, bytes);
        ok = mbar_wait(&bar[0], 0u, kFWaitLimit);
    }

    // passes 2 and 3: columns 2 c, 2 c + 1 and rows 2 p, 2 p + 1 of the tile
    const int c = tid & 31, p = tid >> 5;
    const int ox = tx0 + 2 * c, oy = ty0 + 2 * p;
    const bool row0 = oy < g.nyf, row1 = oy + 1 < g.nyf, col0 = ox < g.nxf, col1 = ox + 1 < g.nxf;
    const bool vec = ((g.nxf & 1) == 0) && col1;  // an aligned 8-byte store per row
    const size_t fplane = (size_t)g.nyf * g.nxf;
    float *Fk = a.fine + (size_t)model * a.f_model_stride + (size_t)oy * g.nxf + ox;  // output channel 0
    const f32x2 Z = pk2(0.f, 0.f);
    // P0[d] / P1[d]: partial sums of output channel e - 2 Rz + 1 + d of the two
    // columns after channel e
    f32x2 P0[NPZ], P1[NPZ];
#pragma unroll
    for (int d = 0; d < NPZ; ++d) P0[d] = P1[d] = Z;
    if (__syncthreads_or(!ok)) {  // slab 0 did not arrive: leave (the same decision in every thread)
        if (tid == 0) {
            atomicExch(&g_conv_fir_status, 1);
            // a bounded chance for the copies in flight to land before the CTA leaves
            for (int q = 0; q < g.ez && q < kFStages; ++q) mbar_wait(&bar[q], 0u, q == 0 ? kFWaitLimit : 1L << 12);
        }
        return;
    }

    for (int e = 0; e < g.ez; ++e) {
        const int s = e % kFStages;
        const float *const slab = slabs + s * D::SS;
        float *const Yb = Y1 + (e & 1) * D::Y1F;
        // ---- pass 1: y on column pairs, rows 4 rb .. 4 rb + 3 (slab e has arrived) ----
        for (int t = tid; t < D::T1; t += kFThreads) {
            const int rb = t / D::C1P, cq = t - rb * D::C1P;
            const float *src = slab + (4 * rb) * D::BW + 2 * cq;
            f32x2 A0 = Z, A1 = Z, A2 = Z, A3 = Z;
#pragma unroll
            for (int i = 0; i < 4 + 2 * R; ++i) {
                const f32x2 x = fld2(src + i * D::BW);
                if (i <= 2 * R) A0 = fma2(a.w2[i], x, A0);
                if (i >= 1 && i - 1 <= 2 * R) A1 = fma2(a.w2[i >= 1 ? i - 1 : 0], x, A1);
                if (i >= 2 && i - 2 <= 2 * R) A2 = fma2(a.w2[i >= 2 ? i - 2 : 0], x, A2);
                if (i >= 3 && i - 3 <= 2 * R) A3 = fma2(a.w2[i >= 3 ? i - 3 : 0], x, A3);
            }
            float a0x, a0y, a1x, a1y, a2x, a2y, a3x, a3y;
            upk2(A0, a0x, a0y);
            upk2(A1, a1x, a1y);
            upk2(A2, a2x, a2y);
            upk2(A3, a3x, a3y);
            // rows (4 rb, 4 rb + 1) -> row pair 2 rb, (4 rb + 2, 4 rb + 3) -> 2 rb + 1;
            // column 2 cq -> even half, 2 cq + 1 -> odd half
            f32x2 *d0 = reinterpret_cast<f32x2 *>(Yb) + (2 * rb) * D::P1 + cq;
            f32x2 *d1 = d0 + D::P1;
            d0[0] = pk2(a0x, a1x);
            d0[D::OH] = pk2(a0y, a1y);
            d1[0] = pk2(a2x, a3x);
            d1[D::OH] = pk2(a2y, a3y);
        }
        // one thread waits for the next slab; the barrier passes the outcome
        // (and, through the barrier, the slab's contents) to every thread
        if (tid == 0 && e + 1 < g.ez)
            ok = mbar_wait(&bar[(e + 1) % kFStages], (uint32_t)(((e + 1) / kFStages) & 1), kFWaitLimit);
        if (__syncthreads_or(!ok)) {
            if (tid == 0) {
                atomicExch(&g_conv_fir_status, 1);
                // a bounded chance for the copies in flight to land before the CTA leaves
                for (int q = e + 1; q < g.ez && q < e + kFStages; ++q)
                    mbar_wait(&bar[q % kFStages], (uint32_t)((q / kFStages) & 1),
                              q == e + 1 ? kFWaitLimit : 1L << 12);
            }
            return;
        }
        // slab e is consumed: refill it with channel e + kFStages
        if (tid == 0 && e + kFStages < g.ez)
            tma_load_slab(&tmap, slabs + s * D::SS, &bar[s], tx0, ty0, zbase + e + kFStages, bytes);
        // ---- pass 2: x for columns 2 c and 2 c + 1 of row pair p ----
        // inputs: even columns 2 c + 2 m and odd columns 2 c + 2 m + 1, m <= R
        const f32x2 *yr = reinterpret_cast<const f32x2 *>(Yb) + p * D::P1 + c;
        f32x2 v0 = Z, v1 = Z;
#pragma unroll
        for (int m = 0; m <= R; ++m) {
            const f32x2 ev = yr[m], od = yr[D::OH + m];
            v0 = fma2(a.w2[2 * m], ev, v0);                  // column 2 c + 2 m, tap 2 m
            if (m >= 1) v1 = fma2(a.w2[2 * m - 1], ev, v1);  // column 2 c + 2 m, tap 2 m - 1
            if (m < R) v0 = fma2(a.w2[2 * m + 1], od, v0);   // column 2 c + 2 m + 1, tap 2 m + 1
            v1 = fma2(a.w2[2 * m], od, v1);                  // column 2 c + 2 m + 1, tap 2 m
        }
        // ---- pass 3: z, transposed FIR: channel e finishes output e - 2 Rz ----
        f32x2 o0, o1;
        if constexpr (RZ == 0) {
            o0 = mul2(a.wz2[0], v0);
            o1 = mul2(a.wz2[0], v1);
        } else {
            o0 = fma2(a.wz2[2 * RZ], v0, P0[0]);
            o1 = fma2(a.wz2[2 * RZ], v1, P1[0]);
#pragma unroll
            for (int d = 1; d < 2 * RZ; ++d) {
                P0[d - 1] = fma2(a.wz2[2 * RZ - d], v0, P0[d]);
                P1[d - 1] = fma2(a.wz2[2 * RZ - d], v1, P1[d]);
            }
            P0[2 * RZ - 1] = mul2(a.wz2[0], v0);
            P1[2 * RZ - 1] = mul2(a.wz2[0], v1);
        }
        if (e >= 2 * RZ) {
            float a0, b0, a1, b1;  // (row 2 p, row 2 p + 1) of columns 2 c and 2 c + 1
            upk2(o0, a0, b0);
            upk2(o1, a1, b1);
            if (vec) {
                if (row0) *reinterpret_cast<float2 *>(Fk) = make_float2(a0, a1);
                if (row1) *reinterpret_cast<float2 *>(Fk + g.nxf) = make_float2(b0, b1);
            } else {
                if (row0 && col0) Fk[0] = a0;
                if (row0 && col1) Fk[1] = a1;
                if (row1 && col0) Fk[g.nxf] = b0;
                if (row1 && col1) Fk[g.nxf + 1] = b1;
            }
            Fk += fplane;
        }
    }
}

// ----------------------------------------------------------------------------
bool conv_fir_supported(const Geom &g)
{
    return g.R <= kFRmax && g.Rz <= kFRzMax && conv_fir_smem(g.R) <= 200 * 1024;
}

template <int R, int RZ>
static gbk_status launch_fir_rr(const CUtensorMap &tm, const ConvFirArgs &a, int blocks, cudaStream_t st)
{
    static KernelAttrMemo memo;
    const size_t smem = conv_fir_smem(R);
    gbk_status s = ensure_kernel_attrs((const void *)conv3d_fir_kernel<R, RZ>, smem, false, memo,
                                       "FIR convolution: setting dynamic shared memory");
    if (s) return s;
    conv3d_fir_kernel<R, RZ><<<blocks, kFThreads, smem, st>>>(tm, a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "FIR convolution launch");
    return GBK_OK;
}

template <int R>
static gbk_status launch_fir_r(const CUtensorMap &tm, const ConvFirArgs &a, int blocks, cudaStream_t st)
{
    switch (a.g.Rz) {
    case 0: return launch_fir_rr<R, 0>(tm, a, blocks, st);
    case 1: return launch_fir_rr<R, 1>(tm, a, blocks, st);
    case 2: return launch_fir_rr<R, 2>(tm, a, blocks, st);
    case 3: return launch_fir_rr<R, 3>(tm, a, blocks, st);
    case 4: return launch_fir_rr<R, 4>(tm, a, blocks, st);
    case 5: return launch_fir_rr<R, 5>(tm, a, blocks, st);
    case 6: return launch_fir_rr<R, 6>(tm, a, blocks, st);
    case 7: return launch_fir_rr<R, 7>(tm, a, blocks, st);
    case 8: return launch_fir_rr<R, 8>(tm, a, blocks, st);
    default: return fail(GBK_EUNSUPPORTED, "LSF radius %d not served by the FIR convolution", a.g.Rz);
    }
}

gbk_status launch_conv_fir(const StagedArgs &sa, cudaStream_t st)
{
    const Geom &g = sa.g;
    if (!conv_fir_supported(g)) return fail(GBK_EUNSUPPORTED, "the FIR convolution does not serve this geometry");
    if (!split_encode_fn()) return fail(GBK_EUNSUPPORTED, "cuTensorMapEncodeTiled is not available from the driver");
    ConvFirArgs a = {};
    a.g = g;
    // normalised Gaussian taps exp(-j^2 / (2 sigma^2)) / sum, as (w, w) pairs
    auto taps = [](int RR, float sigma, f32x2 *out) {
        double w[2 * kFRmax + 1], sum = 0.0;
        for (int j = -RR; j <= RR; ++j) {
            const double t = (RR == 0) ? 0.0 : (double)j / (double)sigma;
            w[j + RR] = std::exp(-0.5 * t * t);
            sum += w[j + RR];
        }
        for (int j = 0; j <= 2 * RR; ++j) {
            const float f = (float)(w[j] / sum);
            uint32_t b;
            std::memcpy(&b, &f, 4);
            out[j] = ((f32x2)b << 32) | (f32x2)b;
        }
    };
    taps(g.R, g.sig_xy, a.w2);
    taps(g.Rz, g.sig_z, a.wz2);
    a.tiles_x = (g.nxf + kFTX - 1) / kFTX;
    a.tiles_y = (g.nyf + kFTY - 1) / kFTY;
    a.fine = sa.fine;
    a.f_model_stride = sa.f_model_stride;
    // the extended cubes as one 3-D tensor [n * ez][ey][e_pitch]; box = one channel's slab
    CUtensorMap tm;
    const cuuint64_t dims[3] = {(cuuint64_t)sa.e_pitch, (cuuint64_t)g.ey, (cuuint64_t)g.ez * (cuuint64_t)sa.n_models};
    const cuuint64_t strides[2] = {(cuuint64_t)sa.e_pitch * sizeof(float),
                                   (cuuint64_t)sa.e_pitch * g.ey * sizeof(float)};
    const cuuint32_t box[3] = {(cuuint32_t)((kFTX + 2 * g.R + 3) & ~3), (cuuint32_t)(kFTY + 2 * g.R), 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = split_encode_fn()(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void *)sa.ext, dims, strides, box, estr,
                                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                   CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(GBK_ECUDA, "FIR convolution: cuTensorMapEncodeTiled failed (%d)", (int)r);
    const int blocks = a.tiles_x * a.tiles_y * sa.n_models;
    switch (g.R) {
    case 0: return launch_fir_r<0>(tm, a, blocks, st);
    case 1: return launch_fir_r<1>(tm, a, blocks, st);
    case 2: return launch_fir_r<2>(tm, a, blocks, st);
    case 3: return launch_fir_r<3>(tm, a, blocks, st);
    case 4: return launch_fir_r<4>(tm, a, blocks, st);
    case 5: return launch_fir_r<5>(tm, a, blocks, st);
    case 6: return launch_fir_r<6>(tm, a, blocks, st);
    case 7: return launch_fir_r<7>(tm, a, blocks, st);
    case 8: return launch_fir_r<8>(tm, a, blocks, st);
    default: return fail(GBK_EUNSUPPORTED, "PSF radius %d not served by the FIR convolution", g.R);
    }
}

gbk_status conv_fir_status_read(int *v)
{
    int zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(v, g_conv_fir_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_conv_fir_status, &zero, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "reading the FIR convolution status");
    return GBK_OK;
}

}  // namespace gbk
