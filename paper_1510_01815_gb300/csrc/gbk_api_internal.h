// gbk_api_internal.h -- host-side helpers shared by the C ABI translation units.
#pragma once

#include "gbk_internal.cuh"

namespace gbk {

gbk_status fail(gbk_status code, const char *fmt, ...);
gbk_status ok();
gbk_status cuda_fail(cudaError_t e, const char *what);
gbk_status derive_geom(const gbk_geom *in, Geom *g);
gbk_status check_device_ptr(const void *p, const char *name, size_t align);
gbk_status check_obs(const gbk_obs *obs);
// reads and clears the wait self-check's status (k_selfcheck.cu)
gbk_status selfcheck_status_read(int *v);

// Kernel attributes apply per device, so what a launcher has already set is
// remembered per device ordinal.  KernelAttrMemo holds, for one kernel, the
// largest dynamic shared-memory limit set so far and whether its non-portable
// cluster sizes are enabled.
constexpr int kMaxDevices = 64;
struct KernelAttrMemo {
    size_t smem[kMaxDevices] = {};
    bool cluster16[kMaxDevices] = {};
};
// Raises `kernel`'s dynamic shared-memory limit on the current device to at
// least `smem` (a no-op when it already is); with `cluster16` also allows
// clusters of up to 16 CTAs.  Thread-safe.
gbk_status ensure_kernel_attrs(const void *kernel, size_t smem, bool cluster16, KernelAttrMemo &memo,
                               const char *what);

}  // namespace gbk
