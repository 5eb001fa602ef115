// k_gemm.h -- BF16 tensor-core GEMM (tcgen05) used by the CNN seed.
#pragma once

#include <cuda_bf16.h>

#include "gbk_internal.cuh"

namespace gbk {

// D[m][n] = alpha * sum_k A[m][k] B[n][k] (+ bias[n]) (ReLU) (* [mask[m][n] > 0]);
// A [M][lda], B [N][ldb] BF16 row-major; D BF16 and/or FP32 [M][ldo].
struct GemmArgs {
    int M, N, K;
    int bn;                       // output tile width (set by the launcher)
    float alpha;
    const float *bias;            // [N] or null
    int relu;
    const __nv_bfloat16 *mask;    // [M][ldm] or null
    int ldm;
    __nv_bfloat16 *out_bf16;      // or null
    float *out_f32;               // or null
    int ldo;
    // Optional transposed BF16 copy of D seen through a row-major reshape:
    //  t_mode 1: D [M][N] viewed as [M/q][q N]   -> out_t[((m % q) N + n) ldt + m / q]
    //  t_mode 2: D [M][N] viewed as [M N/c][c]   -> out_t[(n % c) ldt + m (N/c) + n / c]
    // (q = 2^t_log2, c = 2^t_log2; q = 1 or c = N is the plain transpose).
    __nv_bfloat16 *out_t;
    int ldt, t_mode, t_log2;
    // Split-K: unit z of a tile sums K tiles [z kt_split, (z+1) kt_split) into
    // the FP32 slice out_f32 + z * split_stride (0: no split).
    int kt_split;
    size_t split_stride;
};

gbk_status launch_gemm_bf16(const void *A, int lda, const void *B, int ldb, const GemmArgs &args, cudaStream_t st);
gbk_status gemm_status_read(int *v);
// Fixed-order sum of split-K slices: out[m][n] = sum_z part[z][m][n] (FP32, ld ldo).
gbk_status launch_splitk_reduce(const float *part, int splits, size_t stride, int M, int N, int ldo, float *out,
                                cudaStream_t st);

}  // namespace gbk
