// noalloc.cu -- gbk_chi2_noalloc: the staged chi-squared path with its
// scratch in a fixed array that the library carries itself.
//
// Some callers cannot allocate device memory at the point where they need a
// chi-squared: a host application whose device memory is owned and fully
// pre-planned by another framework (no allocator is exposed to plug-ins), a
// real-time or embedded caller that forbids allocation after start-up, or a
// caller that must not touch the allocator while other work is queued.  This
// entry point lets them run the staged path (model cube -> separable
// convolution -> moments -> chi-squared) without providing a workspace: the
// scratch is a file-scope __device__ array of kNoAllocScratchBytes that every
// GPU loading this library holds until the process exits.
//
// The array's name is a host-side stand-in in host code, not a device
// address, so its device address is looked up once per device with
// cudaGetSymbolAddress (with that device current) and cached.  The first call
// on a device does that look-up, so make the first call before any stream
// capture; a first call made while its stream is capturing is refused with
// GBK_EUNSUPPORTED before the look-up.  A device reset (cudaDeviceReset, or
// a primary context torn down and made again) reloads the module, and the
// cached address is then stale: such a caller must not use this entry point
// after the reset.  Every call shares the one array: calls that overlap on
// the GPU (on different streams, or from different host threads) race on it
// and must be serialised by the caller.  No byte of the array needs to start at zero:
// the kernels of the staged path write every value (including row padding)
// before any kernel of the same call reads it.  The entry point calls no
// cudaMalloc, cudaFree or allocating library routine.
#include <mutex>

#include "gbk_api_internal.h"

namespace gbk {

constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;  // 32 MiB
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

static std::mutex g_noalloc_mu;
static void *g_noalloc_ptr[kNoAllocMaxDevices];

// Device address of the scratch array on the current device.  The look-up is
// not made while `stream` is capturing (it would end the capture).
static gbk_status noalloc_scratch(void **out, cudaStream_t stream)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(GBK_EUNSUPPORTED, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        e = cudaStreamIsCapturing(stream, &cap);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamIsCapturing");
        if (cap != cudaStreamCaptureStatusNone)
            return fail(GBK_EUNSUPPORTED, "gbk_chi2_noalloc: the first call on device %d must not be captured "
                        "(it looks up the built-in scratch's address); call it once before capturing", dev);
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the built-in scratch");
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return GBK_OK;
}

}  // namespace gbk

using namespace gbk;

extern "C" gbk_status gbk_chi2_noalloc(const gbk_geom *g, int32_t n_models, const double *params,
                                       const gbk_obs *obs, double *chi2, float *resid, void *stream)
{
    size_t need = gbk_workspace_bytes(g, n_models, GBK_PATH_STAGED);
    if (n_models == 0 && need == 0 && gbk_last_error()[0] == '\0') return ok();
    if (need == 0 && gbk_last_error()[0] != '\0') return GBK_EINVAL;  // message already set
    if (need > kNoAllocScratchBytes)
        return fail(GBK_EWORKSPACE,
                    "%d models of this geometry need %zu bytes of scratch; the built-in scratch holds %zu "
                    "(split the batch, or use gbk_chi2 with a workspace)",
                    n_models, need, kNoAllocScratchBytes);
    void *ws = nullptr;
    gbk_status s = noalloc_scratch(&ws, (cudaStream_t)stream);
    if (s) return s;
    return gbk_chi2(g, n_models, params, obs, chi2, resid, GBK_PATH_STAGED, ws, kNoAllocScratchBytes, stream);
}
