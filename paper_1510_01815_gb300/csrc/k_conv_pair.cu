// k_conv_pair.cu -- the staged separable PSF x LSF convolution (Eq. 9,
// Sec. 2.2.3) on packed FP32 pairs (f32x2), for PSF radii R <= 8 (one
// template instance per R, so every tap loop is fully unrolled).
//
// One CTA of 256 threads owns a 32 x 32 tile of output spaxels of one model
// and walks the extended channels:
//   - TMA loads each channel's (32 + 2R) x (32 + 2R) input slab two channels
//     ahead into a double buffer (bounded mbarrier waits);
//   - pass 1 (PSF along y) runs first, on column PAIRS of the slab: a pair of
//     adjacent columns is one naturally aligned 8-byte load, so every tap is
//     one packed FMA for two outputs; each thread computes 4 rows and writes
//     them to a buffer whose rows are interleaved in pairs;
//   - pass 2 (PSF along x) then reads ROW pairs from that buffer, again one
//     8-byte load and one packed FMA per tap for two outputs, and writes
//     into a ring of the last W + 4 x-pass results (W = 2 Rz + 1);
//   - pass 3 (LSF along z) runs every fourth channel, while pass 2 of the
//     channel fills the next slot: each thread computes FOUR consecutive
//     output channels of its column pairs from the 4 + W - 1 ring entries
//     they need (register blocking along z: 4 + W - 1 shared loads for 4
//     outputs instead of 4 W), so each channel needs two block barriers;
//     finished rows of 32 floats are written coalesced.  Pass 3 is
//     compiled for each window width W, and the ring has a multiple of four
//     slots, so every aligned group of four ring entries is contiguous: one
//     slot base per four loads and no runtime bounds in its loops.
// The separable passes are exact in real arithmetic in any order; here y
// comes before x.
#include <cuda.h>

#include "gbk_api_internal.h"
#include "gbk_internal.cuh"
#include "k_staged.h"
#include "tma_util.cuh"

namespace gbk {

constexpr int kPT = 32;            // output tile edge
constexpr int kPThreads = 256;
constexpr int kPRmax = 8;          // largest PSF radius served
constexpr int kXP = kPT + 1;       // pair pitch of a ring row (conflict-free pass-2 stores)
constexpr int kZT = 4;             // output channels per pass-3 group
constexpr int kWmax = 2 * 8 + 1;   // widest LSF window served (Rz <= 8)
constexpr long kPWaitLimit = 1L << 18;  // tries: about one second (3.75 us per failed try_wait)

__device__ int g_conv_pair_status;  // 0 fine; 1 a TMA wait timed out

struct ConvPairArgs {
    Geom g;
    int tiles_x, tiles_y;
    int box_w;
    float *fine;
    size_t f_model_stride;
};

__device__ __forceinline__ f32x2 ld2(const float *p) { return *reinterpret_cast<const f32x2 *>(p); }

// Four outputs of one separable pass: A_m = sum_j w[j] * P[j + m], m < 4,
// with the 4 + 2R inputs P loaded from src + i * stride.
template <int R>
__device__ __forceinline__ void pass4(const float *src, int stride, const f32x2 *w2, f32x2 &A0, f32x2 &A1,
                                      f32x2 &A2, f32x2 &A3)
{
    f32x2 P[4 + 2 * R];
#pragma unroll
    for (int i = 0; i < 4 + 2 * R; ++i) P[i] = ld2(src + i * stride);
    const f32x2 Z = pk2(0.f, 0.f);
    A0 = A1 = A2 = A3 = Z;
#pragma unroll
    for (int j = 0; j <= 2 * R; ++j) {
        const f32x2 w = w2[j];
        A0 = fma2(w, P[j], A0);
        A1 = fma2(w, P[j + 1], A1);
        A2 = fma2(w, P[j + 2], A2);
        A3 = fma2(w, P[j + 3], A3);
    }
}

// Ring slots: at least W + kZT (the window of a pass-3 group plus the slot
// pass 2 fills meanwhile), rounded up to a multiple of kZT.
__host__ __device__ inline int conv_ring_slots(int Rz) { return (2 * Rz + 1 + kZT + kZT - 1) / kZT * kZT; }

// Pass 3 for output channels k0 .. k0 + kZT - 1 (k0 a multiple of kZT, ring
// slot s0 = k0 % NR): the thread's column c at row pairs rp and rp + 8.
// Entries 4q .. 4q + 3 of the window sit in slots (s0 + 4q) % NR + 0..3:
// s0 and NR are multiples of four, so such a group never wraps.
template <int W>
__device__ __forceinline__ void conv_pass3(const float *Xr, const f32x2 *wz2, int s0, int NR, int c, int rp, int k0,
                                           float *F, size_t fplane, int ox, int oy0, const Geom &g)
{
    constexpr int NI = kZT + W - 1;         // ring entries read
    constexpr int NQ = (NI + 3) / 4;        // groups of four entries
    constexpr int SLOT = 16 * kXP * 2;      // floats per ring slot
    int qb[NQ];                             // first float of each group's slot
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        int sl = s0 + 4 * q;                // < 2 NR: 4 q <= NI - 1 < NR
        if (sl >= NR) sl -= NR;
        qb[q] = sl * SLOT;
    }
    const f32x2 Z = pk2(0.f, 0.f);
#pragma unroll 1
    for (int half = 0; half < 2; ++half) {
        const int prow = rp + 8 * half;  // row pair of this thread's column
        const float *col = Xr + (size_t)(prow * kXP + c) * 2;
        f32x2 xin[NI];
#pragma unroll
        for (int i = 0; i < NI; ++i) xin[i] = ld2(col + qb[i >> 2] + (i & 3) * SLOT);
        f32x2 B[kZT];
#pragma unroll
        for (int t = 0; t < kZT; ++t) B[t] = Z;
#pragma unroll
        for (int j = 0; j < W; ++j) {
            const f32x2 wq = wz2[j];
#pragma unroll
            for (int t = 0; t < kZT; ++t) B[t] = fma2(wq, xin[t + j], B[t]);
        }
        const int oy = oy0 + 16 * half;
        if (ox < g.nxf) {
            const bool y0 = oy < g.nyf, y1 = oy + 1 < g.nyf;
            float *Fk = F + (size_t)k0 * fplane + (size_t)oy * g.nxf + ox;
#pragma unroll
            for (int t = 0; t < kZT; ++t, Fk += fplane) {
                if (k0 + t < g.nzf) {
                    float v0, v1;
                    upk2(B[t], v0, v1);
                    if (y0) Fk[0] = v0;
                    if (y1) Fk[g.nxf] = v1;
                }
            }
        }
    }
}

template <int R>
__global__ void __launch_bounds__(kPThreads, 2)
    conv3d_pair_kernel(const __grid_constant__ CUtensorMap tmap, ConvPairArgs a)
{
    const Geom &g = a.g;
    const int W = 2 * g.Rz + 1, NR = conv_ring_slots(g.Rz);  // ring of NR x-pass results
    const int SY = kPT + 2 * R, BW = a.box_w, C1W = kPT + 2 * R, C1P = C1W / 2;
    // Pair-row pitches of the two buffers (in pairs), chosen odd / 33 so that a
    // warp's 8-byte accesses spread over all 32 banks.
    const int P1 = C1W + 1;
    const int tiles = a.tiles_x * a.tiles_y;
    const int model = blockIdx.x / tiles;
    const int tt = blockIdx.x - model * tiles;
    const int ty0 = (tt / a.tiles_x) * kPT, tx0 = (tt % a.tiles_x) * kPT;
    const int tid = threadIdx.x;

    extern __shared__ __align__(128) float psm_raw[];
    // 128-byte aligned tensor-copy destinations (the launch adds 128 bytes)
    float *psm = psm_raw + (((128u - (smem_u32(psm_raw) & 127u)) & 127u) >> 2);
    const int SS = (SY * BW + 31) & ~31;
    float *slab0 = psm, *slab1 = psm + SS;
    float *Y1 = slab1 + SS;                                              // [16 row pairs][P1][2]
    float *Xr = Y1 + 32 * P1;                                            // [NR][16 row pairs][kXP][2]
    f32x2 *w2 = reinterpret_cast<f32x2 *>(Xr + (size_t)NR * 32 * kXP);  // PSF taps, duplicated
    f32x2 *wz2 = w2 + (2 * R + 1);                                       // LSF taps, duplicated
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int s_abort;

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    for (int j = tid; j <= 2 * R; j += kPThreads) {
        float s = 0.f;
        for (int q = -R; q <= R; ++q) s += (R == 0) ? 1.f : gauss_tap(q, g.sig_xy);
        const float w = ((R == 0) ? 1.f : gauss_tap(j - R, g.sig_xy)) / s;
        w2[j] = pk2(w, w);
    }
    for (int q = tid; q < W; q += kPThreads) {
        const int Rz = g.Rz;
        float s = 0.f;
        for (int i = -Rz; i <= Rz; ++i) s += (Rz == 0) ? 1.f : gauss_tap(i, g.sig_z);
        const float w = ((Rz == 0) ? 1.f : gauss_tap(q - Rz, g.sig_z)) / s;
        wz2[q] = pk2(w, w);
    }
    __syncthreads();

    const uint32_t bytes = (uint32_t)(SY * BW * sizeof(float));
    const int zbase = model * g.ez;
    if (tid == 0) {
        tma_load_slab(&tmap, slab0, &bar[0], tx0, ty0, zbase, bytes);
        if (g.ez > 1) tma_load_slab(&tmap, slab1, &bar[1], tx0, ty0, zbase + 1, bytes);
    }
    // pass-3 ownership: column c, row pairs rp and rp + 8 (rows 2 rp, 2 rp + 1,
    // 2 rp + 16, 2 rp + 17)
    const int c = tid & 31, rp = tid >> 5;
    float *F = a.fine + (size_t)model * a.f_model_stride;
    const size_t fplane = (size_t)g.nyf * g.nxf;
    const int ox = tx0 + c;
    const int oy0 = ty0 + 2 * rp;

    // Step e runs passes 1 and 2 of channel e (e < ez) into ring slot e % NR
    // and, when k0 = e - (kZT + W - 1) is a multiple of kZT, pass 3 of output
    // channels k0 .. k0 + kZT - 1, whose inputs k0 .. e - 1 sit in the other
    // kZT + W - 1 slots.
    for (int e = 0; e < g.ez + kZT; ++e) {
        if (e < g.ez) {
            float *slab = (e & 1) ? slab1 : slab0;
            if (!mbar_wait(&bar[e & 1], (uint32_t)((e >> 1) & 1), kPWaitLimit)) {
                if (atomicExch(&s_abort, 1) == 0) atomicExch(&g_conv_pair_status, 1);
            }
            __syncthreads();
            if (s_abort) {
                // give the other buffer's copy, if one is in flight, a bounded
                // chance to land before the CTA leaves
                if (tid == 0 && e + 1 < g.ez)
                    mbar_wait(&bar[(e + 1) & 1], (uint32_t)(((e + 1) >> 1) & 1), kPWaitLimit);
                return;
            }
            // ---- pass 1: y, on column pairs; 4 rows per item ----
            if (tid < 8 * C1P) {
                const int rb = tid / C1P, cp = tid - rb * C1P;
                f32x2 A0, A1, A2, A3;
                pass4<R>(slab + (4 * rb) * BW + 2 * cp, BW, w2, A0, A1, A2, A3);
                float a0x, a0y, a1x, a1y, a2x, a2y, a3x, a3y;
                upk2(A0, a0x, a0y);
                upk2(A1, a1x, a1y);
                upk2(A2, a2x, a2y);
                upk2(A3, a3x, a3y);
                // rows (4 rb, 4 rb + 1) -> row pair 2 rb; (4 rb + 2, 4 rb + 3) -> 2 rb + 1
                // (8-byte stores: with P1 odd, an odd row pair starts at 2 mod 4 floats)
                f32x2 *d0 = reinterpret_cast<f32x2 *>(Y1 + ((2 * rb) * P1 + 2 * cp) * 2);
                f32x2 *d1 = reinterpret_cast<f32x2 *>(Y1 + ((2 * rb + 1) * P1 + 2 * cp) * 2);
                d0[0] = pk2(a0x, a1x);
                d0[1] = pk2(a0y, a1y);
                d1[0] = pk2(a2x, a3x);
                d1[1] = pk2(a2y, a3y);
            }
        }
        __syncthreads();
        if (e < g.ez) {
            // the slab is consumed: refill it with channel e + 2
            if (tid == 0 && e + 2 < g.ez)
                tma_load_slab(&tmap, (e & 1) ? slab1 : slab0, &bar[e & 1], tx0, ty0, zbase + e + 2, bytes);
            // ---- pass 2: x, on row pairs; 4 columns per item, into ring slot e % NR ----
            // (the 16 lanes of a half-warp take 16 row pairs of one column block:
            // with pitches of P1 = 32 + 2R + 1 and 33 pairs their 8-byte loads and
            // stores fall on distinct bank pairs)
            if (tid < 16 * 8) {
                const int p2 = tid & 15, cb = tid >> 4;
                f32x2 A0, A1, A2, A3;
                pass4<R>(Y1 + (p2 * P1 + 4 * cb) * 2, 2, w2, A0, A1, A2, A3);
                f32x2 *dst = reinterpret_cast<f32x2 *>(Xr + ((size_t)(e % NR) * 16 * kXP + p2 * kXP + 4 * cb) * 2);
                dst[0] = A0;
                dst[1] = A1;
                dst[2] = A2;
                dst[3] = A3;
            }
        }
        // ---- pass 3: z for output channels k0 .. k0 + kZT - 1 ----
        const int k0 = e - (kZT + W - 1);
        if (k0 >= 0 && k0 % kZT == 0 && k0 < g.nzf) {
            const int s0 = k0 % NR;
            switch (g.Rz) {  // the same case in every thread
            case 0: conv_pass3<1>(Xr, wz2, s0, NR, c, rp, k0, F, fplane, ox, oy0, g); break;
            case 1: conv_pass3<3>(Xr, wz2, s0, NR, c, rp, k0, F, fplane, ox, oy0, g); break;
            case 2: conv_pass3<5>(Xr, wz2, s0, NR, c, rp, k0, F, fplane, ox, oy0, g); break;
            case 3: conv_pass3<7>(Xr, wz2, s0, NR, c, rp, k0, F, fplane, ox, oy0, g); break;
            case 4: conv_pass3<9>(Xr, wz2, s0, NR, c, rp, k0, F, fplane, ox, oy0, g); break;
            case 5: conv_pass3<11>(Xr, wz2, s0, NR, c, rp, k0, F, fplane, ox, oy0, g); break;
            case 6: conv_pass3<13>(Xr, wz2, s0, NR, c, rp, k0, F, fplane, ox, oy0, g); break;
            case 7: conv_pass3<15>(Xr, wz2, s0, NR, c, rp, k0, F, fplane, ox, oy0, g); break;
            default: conv_pass3<17>(Xr, wz2, s0, NR, c, rp, k0, F, fplane, ox, oy0, g); break;
            }
        }
    }
}

// ----------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFnP)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFnP encode_fn_p()
{
    static EncodeTiledFnP fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFnP)p;
    }
    return fn;
}

static size_t conv_pair_smem_bytes(const Geom &g)
{
    const int SY = kPT + 2 * g.R, BW = (kPT + 2 * g.R + 3) & ~3, C1W = kPT + 2 * g.R;
    const int SS = (SY * BW + 31) & ~31, NR = conv_ring_slots(g.Rz);
    return 128 + sizeof(float) * ((size_t)2 * SS + 32 * (C1W + 1) + (size_t)NR * 32 * kXP) +
           sizeof(f32x2) * (2 * g.R + 1 + 2 * g.Rz + 1);
}

bool conv_pair_supported(const Geom &g)
{
    return g.R <= kPRmax && 2 * g.Rz + 1 <= kWmax && conv_pair_smem_bytes(g) <= 200 * 1024 &&
           encode_fn_p() != nullptr;
}

template <int R>
static gbk_status launch_pr(const CUtensorMap &tm, const ConvPairArgs &a, size_t smem, int blocks, cudaStream_t st)
{
    static KernelAttrMemo memo;
    gbk_status s = ensure_kernel_attrs((const void *)conv3d_pair_kernel<R>, smem, false, memo,
                                       "pair convolution: setting dynamic shared memory");
    if (s) return s;
    conv3d_pair_kernel<R><<<blocks, kPThreads, smem, st>>>(tm, a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "pair convolution launch");
    return GBK_OK;
}

gbk_status launch_conv_pair(const StagedArgs &sa, cudaStream_t st)
{
    const Geom &g = sa.g;
    EncodeTiledFnP enc = encode_fn_p();
    if (!enc) return fail(GBK_EUNSUPPORTED, "cuTensorMapEncodeTiled is not available from the driver");
    ConvPairArgs a = {};
    a.g = g;
    a.tiles_x = (g.nxf + kPT - 1) / kPT;
    a.tiles_y = (g.nyf + kPT - 1) / kPT;
    a.box_w = (kPT + 2 * g.R + 3) & ~3;
    a.fine = sa.fine;
    a.f_model_stride = sa.f_model_stride;
    CUtensorMap tm;
    cuuint64_t dims[3] = {(cuuint64_t)sa.e_pitch, (cuuint64_t)g.ey, (cuuint64_t)g.ez * (cuuint64_t)sa.n_models};
    cuuint64_t strides[2] = {(cuuint64_t)sa.e_pitch * sizeof(float), (cuuint64_t)sa.e_pitch * g.ey * sizeof(float)};
    cuuint32_t box[3] = {(cuuint32_t)a.box_w, (cuuint32_t)(kPT + 2 * g.R), 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, (void *)sa.ext, dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(GBK_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    const size_t smem = conv_pair_smem_bytes(g);
    const int blocks = a.tiles_x * a.tiles_y * sa.n_models;
    switch (g.R) {
    case 0: return launch_pr<0>(tm, a, smem, blocks, st);
    case 1: return launch_pr<1>(tm, a, smem, blocks, st);
    case 2: return launch_pr<2>(tm, a, smem, blocks, st);
    case 3: return launch_pr<3>(tm, a, smem, blocks, st);
    case 4: return launch_pr<4>(tm, a, smem, blocks, st);
    case 5: return launch_pr<5>(tm, a, smem, blocks, st);
    case 6: return launch_pr<6>(tm, a, smem, blocks, st);
    case 7: return launch_pr<7>(tm, a, smem, blocks, st);
    case 8: return launch_pr<8>(tm, a, smem, blocks, st);
    default: return fail(GBK_EUNSUPPORTED, "PSF radius %d not served by the pair convolution", g.R);
    }
}

gbk_status conv_pair_status_read(int *v)
{
    int zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(v, g_conv_pair_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_conv_pair_status, &zero, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "reading the pair convolution status");
    return GBK_OK;
}

}  // namespace gbk
