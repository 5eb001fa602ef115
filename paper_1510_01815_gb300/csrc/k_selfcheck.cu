// k_selfcheck.cu -- gbk_wait_selfcheck: the bounded mbarrier wait that the
// TMA-fed convolution and the tensor-core GEMM use, run on a barrier that
// nothing completes (or that one arrival completes), so that the timeout
// path -- give up after a bounded number of tries, record it in the device
// status word, return -- can be exercised without a fault, a trap or a hang.
#include "gbk_api_internal.h"
#include "tma_util.cuh"

namespace gbk {

__device__ int g_selfcheck_status;              // 0 fine; 1 the self-check's wait ran out
__device__ unsigned long long g_selfcheck_ns;   // duration of the last self-check wait

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__global__ void wait_selfcheck_kernel(long limit, int complete)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (complete) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bar)) : "memory");
    const uint64_t t0 = global_ns();
    const bool done = mbar_wait(&bar, 0, limit);
    g_selfcheck_ns = (unsigned long long)(global_ns() - t0);
    if (!done) atomicExch(&g_selfcheck_status, 1);
}

gbk_status selfcheck_status_read(int *v)
{
    int zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(v, g_selfcheck_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_selfcheck_status, &zero, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e, "reading the self-check status");
    return GBK_OK;
}

}  // namespace gbk

using namespace gbk;

extern "C" gbk_status gbk_wait_selfcheck(int64_t limit, int32_t complete, int64_t *elapsed_ns, void *stream)
{
    if (limit < 1 || limit > (1LL << 24)) return fail(GBK_EINVAL, "limit must be in 1..2^24");
    if (complete != 0 && complete != 1) return fail(GBK_EINVAL, "complete must be 0 or 1");
    cudaStream_t st = (cudaStream_t)stream;
    wait_selfcheck_kernel<<<1, 32, 0, st>>>((long)limit, complete);
    cudaError_t e = cudaGetLastError();
    unsigned long long ns = 0;
    if (e == cudaSuccess) e = cudaMemcpyFromSymbolAsync(&ns, g_selfcheck_ns, sizeof(ns), 0, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "self-check wait");
    if (elapsed_ns) *elapsed_ns = (int64_t)ns;
    return ok();
}
