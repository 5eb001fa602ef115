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
};

gbk_status launch_gemm_bf16(const void *A, int lda, const void *B, int ldb, const GemmArgs &args, cudaStream_t st);
gbk_status gemm_status_read(int *v);

}  // namespace gbk
