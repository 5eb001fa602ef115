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

}  // namespace gbk
