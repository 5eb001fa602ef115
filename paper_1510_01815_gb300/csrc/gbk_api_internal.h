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

}  // namespace gbk
