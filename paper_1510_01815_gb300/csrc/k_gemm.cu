// k_gemm.cu -- BF16 tensor-core GEMM on the 5th-generation tensor cores
// (tcgen05), the dense building block of the CNN that seeds the fits.
//
//   D[m][n] = alpha * sum_k A[m][k] * B[n][k]  (+ bias[n]) (ReLU) (* [mask[m][n] > 0])
//
// A [M][K] and B [N][K] are BF16, row-major (both "K-major"); D is written as
// BF16 and/or FP32 with leading dimension ldo.  The output is cut into
// 128 x BN tiles (BN = 16..256, a multiple of 16; 256 when N allows), and a
// persistent grid of one CTA per SM (at most) walks them in a grouped order;
// each CTA of 192 threads is warp-specialised:
//   - warp 0 lane 0 streams 64-wide K slabs of A and B with TMA
//     (cp.async.bulk.tensor.2d, 128-byte swizzle) into a 4-stage ring shared
//     by all of the CTA's tiles, completion counted on "full" mbarriers;
//   - warp 1 lane 0 issues tcgen05.mma (kind::f16, BF16 in, FP32 accumulate,
//     M = 128, N = BN, K = 16 per instruction, four per slab) into one of two
//     accumulators in tensor memory, releases each slab with tcgen05.commit
//     onto its "empty" mbarrier and, after a tile's last slab, commits onto
//     that accumulator's "full" mbarrier;
//   - warps 2-5 read the accumulator's 128 TMEM lanes (each warp its quarter)
//     with tcgen05.ld, apply the epilogue, store, and hand the accumulator
//     back on its "empty" mbarrier -- so a tile's epilogue overlaps the next
//     tile's loads and MMAs.
// Every wait is bounded: a thread that gives up records a status in
// g_gemm_status and raises a CTA-wide abort flag that every other wait
// checks, the roles leave their loops, and the CTA still frees its tensor
// memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

#include "gbk_api_internal.h"
#include "k_gemm.h"

namespace gbk {

constexpr int kGBM = 128, kGBK = 64, kGStages = 4, kGThreads = 192, kGGroup = 16;
// Bounded waits: 2^18 try_wait attempts, about one second (a try that finds
// its phase incomplete suspends about 3.75 us on GB300, as gbk_wait_selfcheck
// measures); a TMA load or an MMA stage completes in microseconds.
constexpr long kGWaitLimit = 1L << 18;

__device__ int g_gemm_status;  // 0 fine; 1 a pipeline wait timed out

__device__ __forceinline__ uint32_t g_smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void g_mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(g_smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ bool g_mbar_wait(uint64_t *bar, uint32_t phase)
{
    for (long it = 0; it < kGWaitLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(g_smem_u32(bar)), "r"(phase)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Bounded wait that gives up early once another role of the CTA has raised
// `abort`; on its own timeout it raises it and records the status.
__device__ __forceinline__ bool g_mbar_wait_abortable(uint64_t *bar, uint32_t phase, volatile int *abort)
{
    for (long it = 0; it < kGWaitLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(g_smem_u32(bar)), "r"(phase)
            : "memory");
        if (done) return true;
        if (*abort) return false;
    }
    *abort = 1;
    atomicExch(&g_gemm_status, 1);
    return false;
}

// One unit of work: an output tile (and, with split-K, a K range).
struct GTile {
    int m0, n0, z, kt0, KT;
};

__device__ __forceinline__ GTile gemm_unit(const GemmArgs &a, int u, int tiles_m, int tiles_n, int KT_all)
{
    GTile t;
    const int tiles = tiles_m * tiles_n;
    t.z = u / tiles;
    const int tt = u - t.z * tiles;
    // grouped order: groups of kGGroup M-tiles with the N-tiles fastest
    // inside a group, so the tiles in flight at one time share their A and
    // B strips in L2
    const int per_group = kGGroup * tiles_n;
    const int grp = tt / per_group, in_grp = tt - grp * per_group;
    const int gm = min(kGGroup, tiles_m - grp * kGGroup);
    const int tm = grp * kGGroup + in_grp % gm, tn = in_grp / gm;
    t.m0 = tm * kGBM;
    t.n0 = tn * a.bn;
    t.kt0 = a.kt_split > 0 ? t.z * a.kt_split : 0;
    t.KT = a.kt_split > 0 ? min(a.kt_split, KT_all - t.kt0) : KT_all;
    return t;
}

__device__ __forceinline__ void g_tma_2d(const CUtensorMap *tmap, void *dst, uint64_t *bar, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(g_smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(g_smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor of a K-major BF16 tile stored as TMA
// writes it with 128-byte swizzling: rows of 64 elements (128 B), atoms of
// 8 rows (1024 B) stacked along M/N.  Fields: start address >> 4 (bits 0-13),
// leading-dimension offset >> 4 (16-29; not used by swizzled K-major
// layouts, set to 1), stride-dimension offset >> 4 (32-45: 1024 B between
// 8-row atoms), descriptor version 1 (46-47), swizzle mode 2 = 128 B (61-63).
__device__ __forceinline__ uint64_t smem_desc_k128(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator (bits 4-5 = 1), A and
// B BF16 (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0),
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ __forceinline__ uint32_t idesc_bf16_f32(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// Epilogue of 16 accumulator columns of row m (columns nb .. nb + 15).
__device__ __forceinline__ void gemm_epilogue16(const GemmArgs &a, float *out_f32, int m, int nb, const uint32_t *r,
                                                bool vec_bf, bool vec_f)
{
    float v[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const int n = nb + j;
        float x = a.alpha * __uint_as_float(r[j]);
        if (n < a.N) {
            if (a.bias) x += a.bias[n];
            if (a.relu) x = fmaxf(x, 0.f);
            if (a.mask && !(__bfloat162float(a.mask[(size_t)m * a.ldm + n]) > 0.f)) x = 0.f;
        }
        v[j] = x;
    }
    const size_t o = (size_t)m * a.ldo + nb;
    const bool full_chunk = nb + 16 <= a.N;
    if (out_f32) {
        if (full_chunk && vec_f) {
            float4 *q = reinterpret_cast<float4 *>(out_f32 + o);
#pragma unroll
            for (int j = 0; j < 4; ++j) q[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
        } else {
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if (nb + j < a.N) out_f32[o + j] = v[j];
        }
    }
    if (a.out_t) {
        if (a.t_mode == 1) {
            const int q = 1 << a.t_log2;
            const size_t rowb = (size_t)(m & (q - 1)) * a.N, col = (size_t)(m >> a.t_log2);
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if (nb + j < a.N) a.out_t[(rowb + nb + j) * a.ldt + col] = __float2bfloat16_rn(v[j]);
        } else {
            const int c = 1 << a.t_log2;
            const size_t colb = (size_t)m * (a.N >> a.t_log2);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int n = nb + j;
                if (n < a.N) a.out_t[(size_t)(n & (c - 1)) * a.ldt + colb + (n >> a.t_log2)] = __float2bfloat16_rn(v[j]);
            }
        }
    }
    if (a.out_bf16) {
        if (full_chunk && vec_bf) {
            uint32_t w[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
                w[j] = *reinterpret_cast<uint32_t *>(&h);
            }
            uint4 *q = reinterpret_cast<uint4 *>(a.out_bf16 + o);
            q[0] = make_uint4(w[0], w[1], w[2], w[3]);
            q[1] = make_uint4(w[4], w[5], w[6], w[7]);
        } else {
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if (nb + j < a.N) a.out_bf16[o + j] = __float2bfloat16_rn(v[j]);
        }
    }
}

__global__ void __launch_bounds__(kGThreads, 1)
    gemm_bf16_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, GemmArgs a,
                     int units)
{
    const int BN = a.bn;
    const int tiles_m = (a.M + kGBM - 1) / kGBM, tiles_n = (a.N + BN - 1) / BN;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int KT_all = (a.K + kGBK - 1) / kGBK;
    const uint32_t bytesA = kGBM * kGBK * 2, bytesB = (uint32_t)BN * kGBK * 2;

    extern __shared__ __align__(1024) unsigned char gsm_raw[];
    // 128-byte swizzled tiles must start on 1024-byte boundaries
    unsigned char *gsm = gsm_raw + ((1024u - (g_smem_u32(gsm_raw) & 1023u)) & 1023u);
    unsigned char *sA = gsm;                      // [stages][128][64] bf16
    unsigned char *sB = gsm + kGStages * bytesA;  // [stages][BN][64] bf16
    __shared__ __align__(8) uint64_t full[kGStages], empty[kGStages], acc_full[2], acc_empty[2];
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    volatile int *abort = &s_abort;

    // two accumulators of nbuf columns each
    const uint32_t nbuf = BN <= 32 ? 32u : (BN <= 64 ? 64u : (BN <= 128 ? 128u : 256u)), ncols = 2 * nbuf;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(g_smem_u32(&s_tmem)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 32) {
        for (int s = 0; s < kGStages; ++s) {
            g_mbar_init(&full[s], 1);
            g_mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            g_mbar_init(&acc_full[b], 1);   // one tcgen05.commit per tile
            g_mbar_init(&acc_empty[b], 4);  // one arrival per epilogue warp
        }
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;

    if (warp == 0) {
        if (lane == 0) {
            // producer: one ring of slabs across all of the CTA's tiles
            uint32_t slab = 0;
            bool go = true;
            for (int u = blockIdx.x; u < units && go; u += gridDim.x) {
                const GTile t = gemm_unit(a, u, tiles_m, tiles_n, KT_all);
                for (int kt = 0; kt < t.KT; ++kt, ++slab) {
                    const int s = (int)(slab % kGStages);
                    const uint32_t ph = (slab / kGStages) & 1u;
                    if (slab >= (uint32_t)kGStages && !g_mbar_wait_abortable(&empty[s], ph ^ 1u, abort)) {
                        go = false;
                        break;
                    }
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(g_smem_u32(&full[s])),
                                 "r"(bytesA + bytesB)
                                 : "memory");
                    g_tma_2d(&tmA, sA + (size_t)s * bytesA, &full[s], (t.kt0 + kt) * kGBK, t.m0);
                    g_tma_2d(&tmB, sB + (size_t)s * bytesB, &full[s], (t.kt0 + kt) * kGBK, t.n0);
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer: tile i accumulates into buffer i % 2
            const uint32_t idesc = idesc_bf16_f32(kGBM, BN);
            uint32_t slab = 0;
            bool go = true;
            int i = 0;
            for (int u = blockIdx.x; u < units && go; u += gridDim.x, ++i) {
                const GTile t = gemm_unit(a, u, tiles_m, tiles_n, KT_all);
                const int buf = i & 1;
                const uint32_t use = (uint32_t)(i >> 1);
                // the epilogue must have read this buffer's previous tile
                if (use > 0 && !g_mbar_wait_abortable(&acc_empty[buf], (use - 1) & 1u, abort)) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t dtm = tmem + (uint32_t)buf * nbuf;
                for (int kt = 0; kt < t.KT; ++kt, ++slab) {
                    const int s = (int)(slab % kGStages);
                    const uint32_t ph = (slab / kGStages) & 1u;
                    if (!g_mbar_wait_abortable(&full[s], ph, abort)) {
                        go = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint64_t da = smem_desc_k128(g_smem_u32(sA + (size_t)s * bytesA));
                    const uint64_t db = smem_desc_k128(g_smem_u32(sB + (size_t)s * bytesB));
#pragma unroll
                    for (int kk = 0; kk < kGBK / 16; ++kk) {
                        // advance 16 elements (32 B) along K inside the swizzle atom
                        const uint32_t acc = (kt > 0 || kk > 0) ? 1u : 0u;
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtm),
                            "l"(da + (uint64_t)(2 * kk)), "l"(db + (uint64_t)(2 * kk)), "r"(idesc), "r"(acc)
                            : "memory");
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     g_smem_u32(&empty[s]))
                                 : "memory");
                }
                if (!go) break;
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 g_smem_u32(&acc_full[buf]))
                             : "memory");
            }
        }
    } else {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (tile rows)
        const int q = warp & 3;
        float *const out_f32_base = a.out_f32;
        // 16-byte vector stores need 16-byte aligned rows and base pointers
        const bool vec_bf = a.out_bf16 && (a.ldo % 8) == 0 && ((uintptr_t)a.out_bf16 % 16) == 0;
        const bool vec_f = a.out_f32 && (a.ldo % 4) == 0 && ((uintptr_t)a.out_f32 % 16) == 0 && (a.split_stride % 4) == 0;
        int i = 0;
        for (int u = blockIdx.x; u < units; u += gridDim.x, ++i) {
            const GTile t = gemm_unit(a, u, tiles_m, tiles_n, KT_all);
            const int buf = i & 1;
            const uint32_t use = (uint32_t)(i >> 1);
            // the loads below are warp-collective: one decision per warp
            const bool have = __all_sync(0xffffffffu, g_mbar_wait_abortable(&acc_full[buf], use & 1u, abort));
            if (!have) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int m = t.m0 + q * 32 + lane;
            float *const out_f32 = out_f32_base ? out_f32_base + (size_t)t.z * a.split_stride : nullptr;
            for (int c0 = 0; c0 < BN; c0 += 16) {
                uint32_t r[16];
                const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)buf * nbuf + (uint32_t)c0;
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                    "%13, %14, %15}, [%16];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                      "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                      "=r"(r[15])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (m < a.M) gemm_epilogue16(a, out_f32, m, t.n0 + c0, r, vec_bf, vec_f);
            }
            // hand the buffer back to the MMA issuer
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0)
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(g_smem_u32(&acc_empty[buf])) : "memory");
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
    }
}

// ----------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFnG)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFnG g_encode()
{
    static EncodeTiledFnG fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFnG)p;
    }
    return fn;
}

// K-major BF16 operand [rows][K] with leading dimension ld, box 64 x box_rows.
static gbk_status encode_kmajor(CUtensorMap *tm, const void *ptr, int rows, int K, int ld, int box_rows)
{
    EncodeTiledFnG enc = g_encode();
    if (!enc) return fail(GBK_EUNSUPPORTED, "cuTensorMapEncodeTiled is not available from the driver");
    cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)kGBK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(GBK_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return GBK_OK;
}

size_t gemm_smem_bytes(int bn) { return 1024 + (size_t)kGStages * (kGBM * kGBK * 2 + (size_t)bn * kGBK * 2); }

gbk_status launch_gemm_bf16(const void *A, int lda, const void *B, int ldb, const GemmArgs &args, cudaStream_t st)
{
    GemmArgs a = args;
    if (a.M < 1 || a.N < 1 || a.K < 1) return fail(GBK_EINVAL, "GEMM sizes must be >= 1");
    if (lda < a.K || ldb < a.K || (lda % 8) || (ldb % 8))
        return fail(GBK_EINVAL, "lda and ldb must be >= K and multiples of 8 (16-byte rows)");
    if (((uintptr_t)A % 16) || ((uintptr_t)B % 16)) return fail(GBK_EINVAL, "A and B must be 16-byte aligned");
    if (a.ldo < a.N) return fail(GBK_EINVAL, "ldo must be >= N");
    if (!a.out_bf16 && !a.out_f32) return fail(GBK_EINVAL, "no output");
    a.bn = a.N >= 256 ? 256 : (a.N >= 128 ? 128 : ((a.N + 15) / 16) * 16);
    CUtensorMap ta, tb;
    gbk_status s = encode_kmajor(&ta, A, a.M, a.K, lda, kGBM);
    if (s) return s;
    if ((s = encode_kmajor(&tb, B, a.N, a.K, ldb, a.bn))) return s;
    size_t smem = gemm_smem_bytes(a.bn);
    static KernelAttrMemo memo;
    if ((s = ensure_kernel_attrs((const void *)gemm_bf16_kernel, smem, false, memo,
                                 "GEMM: setting dynamic shared memory")))
        return s;
    int splits = 1;
    if (a.kt_split > 0) {
        if (!a.out_f32 || a.out_bf16 || a.out_t) return fail(GBK_EINVAL, "split-K writes FP32 slices only");
        int KT = (a.K + kGBK - 1) / kGBK;
        splits = (KT + a.kt_split - 1) / a.kt_split;
        if (splits > 65535) return fail(GBK_EINVAL, "too many K splits");
    }
    if (a.out_t) {
        if (a.t_mode != 1 && a.t_mode != 2) return fail(GBK_EINVAL, "unknown transposed-output mode");
        if (a.t_log2 < 0 || a.t_log2 > 16) return fail(GBK_EINVAL, "transposed-output factor out of range");
        if (a.t_mode == 1 && (a.M & ((1 << a.t_log2) - 1))) return fail(GBK_EINVAL, "M must be a multiple of q");
        if (a.t_mode == 2 && (a.N & ((1 << a.t_log2) - 1))) return fail(GBK_EINVAL, "N must be a multiple of c");
    }
    const long units = (long)((a.M + kGBM - 1) / kGBM) * ((a.N + a.bn - 1) / a.bn) * splits;
    if (units > 0x7fffffffL) return fail(GBK_EINVAL, "GEMM too large");
    // persistent grid: at most one CTA per SM, each walking units
    // blockIdx.x, blockIdx.x + gridDim.x, ...
    static int sm_count[64] = {0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "GEMM: current device");
    if (dev < 0 || dev >= 64) return fail(GBK_EUNSUPPORTED, "GEMM: device index %d", dev);
    if (sm_count[dev] == 0) {
        int n = 0;
        if ((e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
            return cuda_fail(e, "GEMM: SM count");
        sm_count[dev] = n > 0 ? n : 1;
    }
    const int grid = (int)std::min<long>(units, sm_count[dev]);
    gemm_bf16_kernel<<<grid, kGThreads, smem, st>>>(ta, tb, a, (int)units);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "GEMM launch");
    return GBK_OK;
}

// Sum of the split-K slices: a block takes 32 consecutive outputs (one per
// lane: coalesced loads) and its 8 warps the slices z = w, w + 8, ... in
// increasing order; the 8 partial sums are added in a fixed tree, so the
// result does not depend on timing.
constexpr int kRedWarps = 8;

__global__ void __launch_bounds__(32 * kRedWarps) splitk_reduce_kernel(const float *part, int splits, size_t stride,
                                                                     int M, int N, int ldo, float *out)
{
    __shared__ float red[kRedWarps][32];
    const size_t total = (size_t)M * N;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (size_t base = (size_t)blockIdx.x * 32; base < total; base += (size_t)gridDim.x * 32) {
        const size_t i = base + lane;
        const bool ok = i < total;
        const size_t m = ok ? i / N : 0, o = ok ? m * ldo + (i - m * N) : 0;
        float s = 0.f;
        if (ok)
            for (int z = w; z < splits; z += kRedWarps) s += part[(size_t)z * stride + o];
        red[w][lane] = s;
        __syncthreads();
        if (w == 0 && ok)
            out[o] = ((red[0][lane] + red[1][lane]) + (red[2][lane] + red[3][lane])) +
                     ((red[4][lane] + red[5][lane]) + (red[6][lane] + red[7][lane]));
        __syncthreads();
    }
}

gbk_status launch_splitk_reduce(const float *part, int splits, size_t stride, int M, int N, int ldo, float *out,
                                cudaStream_t st)
{
    size_t total = (size_t)M * N;
    int blocks = (int)std::min<size_t>((total + 31) / 32, 152 * 16);
    splitk_reduce_kernel<<<blocks, 32 * kRedWarps, 0, st>>>(part, splits, stride, M, N, ldo, out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "split-K reduction launch");
    return GBK_OK;
}

gbk_status gemm_status_read(int *v)
{
    int zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(v, g_gemm_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_gemm_status, &zero, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "reading the GEMM status");
    return GBK_OK;
}

}  // namespace gbk

using namespace gbk;

extern "C" gbk_status gbk_gemm_bf16(int32_t M, int32_t N, int32_t K, const void *A, int32_t lda, const void *B,
                                    int32_t ldb, const float *bias, int32_t relu, const void *mask, int32_t ldm,
                                    float alpha, void *out_bf16, float *out_f32, int32_t ldo, void *stream)
{
    gbk_status s;
    if ((s = check_device_ptr(A, "A", 16)) || (s = check_device_ptr(B, "B", 16))) return s;
    if (bias && (s = check_device_ptr(bias, "bias", 4))) return s;
    if (mask && (s = check_device_ptr(mask, "mask", 2))) return s;
    if (out_bf16 && (s = check_device_ptr(out_bf16, "out_bf16", 2))) return s;
    if (out_f32 && (s = check_device_ptr(out_f32, "out_f32", 4))) return s;
    if (mask && ldm < N) return fail(GBK_EINVAL, "ldm must be >= N");
    GemmArgs a = {};
    a.M = M;
    a.N = N;
    a.K = K;
    a.alpha = alpha;
    a.bias = bias;
    a.relu = relu;
    a.mask = (const __nv_bfloat16 *)mask;
    a.ldm = ldm;
    a.out_bf16 = (__nv_bfloat16 *)out_bf16;
    a.out_f32 = out_f32;
    a.ldo = ldo;
    if ((s = launch_gemm_bf16(A, lda, B, ldb, a, (cudaStream_t)stream))) return s;
    return ok();
}
