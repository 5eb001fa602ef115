// gbk_api.cu -- C ABI entry points of libgbk.so: argument validation, path
// selection, workspace layout and kernel launches.  All model arithmetic is in
// the kernels (k_fused.cu, k_staged.cu).
#include <mutex>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <string>

#include "gbk_api_internal.h"
#include "k_fused.h"
#include "k_split.h"
#include "k_tsplit.h"
#include "k_gemm.h"
#include "k_staged.h"

namespace gbk {

static thread_local std::string t_last_error;

gbk_status fail(gbk_status code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    t_last_error = buf;
    return code;
}

gbk_status ok()
{
    t_last_error.clear();
    return GBK_OK;
}

gbk_status ensure_kernel_attrs(const void *kernel, size_t smem, bool cluster16, KernelAttrMemo &memo,
                               const char *what)
{
    static std::mutex mu;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(GBK_EUNSUPPORTED, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(mu);
    if (smem > memo.smem[dev]) {
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_fail(e, what);
        memo.smem[dev] = smem;
    }
    if (cluster16 && !memo.cluster16[dev]) {
        e = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return cuda_fail(e, what);
        memo.cluster16[dev] = true;
    }
    return GBK_OK;
}

gbk_status cuda_fail(cudaError_t e, const char *what)
{
    return fail(GBK_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

static bool finite_nonneg(double v) { return std::isfinite(v) && v >= 0.0; }

gbk_status derive_geom(const gbk_geom *in, Geom *g)
{
    if (!in) return fail(GBK_EINVAL, "geometry pointer is NULL");
    if (in->nx < 1 || in->ny < 1 || in->nz < 1)
        return fail(GBK_EINVAL, "cube size must be >= 1 (got %d x %d x %d)", in->nx, in->ny, in->nz);
    if (in->upsample < 1 || in->upsample > 16) return fail(GBK_EINVAL, "upsample must be in 1..16");
    if (!(std::isfinite(in->dv) && in->dv > 0.0)) return fail(GBK_EINVAL, "dv must be finite and > 0");
    if (!std::isfinite(in->vc)) return fail(GBK_EINVAL, "vc must be finite");
    if (!finite_nonneg(in->psf_fwhm)) return fail(GBK_EINVAL, "psf_fwhm must be finite and >= 0");
    if (!finite_nonneg(in->lsf_fwhm)) return fail(GBK_EINVAL, "lsf_fwhm must be finite and >= 0");
    if (in->lsf_mode != 0 && in->lsf_mode != 1) return fail(GBK_EINVAL, "lsf_mode must be 0 or 1");
    if (in->model < GBK_MODEL_CUBE || in->model > GBK_MODEL_VFIELD_EPINAT)
        return fail(GBK_EINVAL, "unknown model %d", in->model);
    if (in->model != GBK_MODEL_CUBE && in->upsample != 1)
        return fail(GBK_EINVAL, "velocity-field models need upsample == 1");
    if (!(std::isfinite(in->halo_sigmas) && in->halo_sigmas > 0.0 && in->halo_sigmas <= 16.0))
        return fail(GBK_EINVAL, "halo_sigmas must be in (0, 16]");
    const int u = in->upsample;
    double sxy = (double)u * in->psf_fwhm / kFwhmPerSigma;
    int R = sxy > 0.0 ? (int)std::ceil(in->halo_sigmas * sxy) : 0;
    double sz = 0.0;
    int Rz = 0;
    if (in->lsf_mode == 0) {
        sz = (double)u * (in->lsf_fwhm / kFwhmPerSigma) / in->dv;
        Rz = sz > 0.0 ? (int)std::ceil(in->halo_sigmas * sz) : 0;
    }
    if (R > kMaxRadius || Rz > kMaxRadius)
        return fail(GBK_EUNSUPPORTED, "kernel radius %d/%d exceeds the supported %d", R, Rz, kMaxRadius);
    g->nx = in->nx; g->ny = in->ny; g->nz = in->nz; g->u = u;
    g->R = R; g->Rz = Rz;
    g->nxf = u * in->nx; g->nyf = u * in->ny; g->nzf = u * in->nz;
    g->ex = g->nxf + 2 * R; g->ey = g->nyf + 2 * R; g->ez = g->nzf + 2 * Rz;
    long long ext_elems = (long long)g->ex * g->ey * g->ez;
    if (ext_elems > (1LL << 31) - 1 || (long long)g->nxf * g->nyf > (1LL << 28))
        return fail(GBK_EUNSUPPORTED, "cube too large for one model (%lld extended voxels)", ext_elems);
    g->dv = (float)in->dv;
    g->vc = (float)in->vc;
    g->sig_xy = (float)sxy;
    g->sig_z = (float)sz;
    g->sig_lsf_kms = (float)(in->lsf_fwhm / kFwhmPerSigma);
    g->lsf_mode = in->lsf_mode;
    g->model = in->model;
    return GBK_OK;
}

// Checks that p is usable by a kernel on the current device.
gbk_status check_device_ptr(const void *p, const char *name, size_t align)
{
    if (!p) return fail(GBK_EINVAL, "%s is NULL", name);
    if (((uintptr_t)p) % align != 0) return fail(GBK_EINVAL, "%s is not %zu-byte aligned", name, align);
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(GBK_EINVAL, "%s is not a CUDA pointer (%s)", name, cudaGetErrorString(e));
    }
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
        return fail(GBK_EINVAL, "%s must be device or managed memory", name);
    int dev = 0;
    cudaGetDevice(&dev);
    if (at.type == cudaMemoryTypeDevice && at.device != dev)
        return fail(GBK_EINVAL, "%s lives on device %d, current device is %d", name, at.device, dev);
    return GBK_OK;
}

gbk_status check_obs(const gbk_obs *obs)
{
    if (!obs) return fail(GBK_EINVAL, "obs is NULL");
    gbk_status s;
    if ((s = check_device_ptr(obs->v_obs, "obs.v_obs", 4))) return s;
    if ((s = check_device_ptr(obs->s_obs, "obs.s_obs", 4))) return s;
    if ((s = check_device_ptr(obs->w_v, "obs.w_v", 4))) return s;
    if ((s = check_device_ptr(obs->w_s, "obs.w_s", 4))) return s;
    if ((s = check_device_ptr(obs->mask, "obs.mask", 1))) return s;
    return GBK_OK;
}

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Staged workspace: [ext][fine (u > 1)][data (if not caller's)][partials].
struct StagedLayout {
    int e_pitch;
    size_t e_stride, f_stride, d_stride;
    size_t off_ext, off_fine, off_data, off_part, total;
    int bpm;
};

StagedLayout staged_layout(const Geom &g, int n, bool own_data, bool want_partials)
{
    StagedLayout L;
    L.e_pitch = (g.ex + 3) & ~3;
    L.e_stride = (size_t)g.ez * g.ey * L.e_pitch;
    L.f_stride = (size_t)g.nzf * g.nyf * g.nxf;
    L.d_stride = (size_t)g.nz * g.ny * g.nx;
    L.bpm = (g.nx * g.ny + 255) / 256;
    size_t off = 0;
    L.off_ext = off; off += align256(sizeof(float) * L.e_stride * n);
    L.off_fine = off; if (g.u > 1) off += align256(sizeof(float) * L.f_stride * n);
    L.off_data = off; if (own_data) off += align256(sizeof(float) * L.d_stride * n);
    L.off_part = off; if (want_partials) off += align256(sizeof(double) * L.bpm * n);
    L.total = off;
    return L;
}

}  // namespace gbk

using namespace gbk;

extern "C" {

const char *gbk_last_error(void) { return t_last_error.c_str(); }

const char *gbk_version(void) { return "gbk 0.1 (sm_103a)"; }

gbk_status gbk_device_status(int32_t *status)
{
    if (!status) return fail(GBK_EINVAL, "status is NULL");
    int c = 0, c2 = 0, g = 0, w = 0, sp = 0, ts = 0;
    gbk_status s;
    if ((s = conv_status_read(&c)) || (s = conv_fir_status_read(&c2)) || (s = gemm_status_read(&g)) ||
        (s = selfcheck_status_read(&w)) || (s = split_status_read(&sp)) || (s = tsplit_status_read(&ts)))
        return s;
    *status = ((c || c2) ? 1 : 0) | (g ? 2 : 0) | (w ? 4 : 0) | ((sp || ts) ? 8 : 0);
    return ok();
}

size_t gbk_workspace_bytes(const gbk_geom *gin, int32_t n_models, uint32_t flags)
{
    ok();
    Geom g;
    if (derive_geom(gin, &g) != GBK_OK) return 0;
    if (n_models < 0) { fail(GBK_EINVAL, "n_models must be >= 0"); return 0; }
    if (flags > GBK_PATH_SPLIT) { fail(GBK_EINVAL, "unknown flags 0x%x", flags); return 0; }
    FusedConfig fc;
    bool fused_ok = fused_config(g, &fc);
    if (g.model != GBK_MODEL_CUBE) return 0;
    if (flags == GBK_PATH_SPLIT || (flags == GBK_PATH_AUTO && split_supported(g)))
        return split_workspace_bytes(g, n_models);
    if (flags == GBK_PATH_FUSED || (flags == GBK_PATH_AUTO && fused_ok)) return 0;
    return staged_layout(g, n_models, true, true).total;
}

// The split path serves the request: its geometry, and a workspace that
// holds its triplets.
static bool split_fits(const Geom &g, int32_t n, const void *ws, size_t ws_bytes)
{
    return ws && split_supported(g) && ws_bytes >= split_workspace_bytes(g, n);
}

static gbk_status run_staged(const Geom &g, int32_t n, const double *params, float *cubes, float *maps,
                             const gbk_obs *obs, double *chi2, float *resid, void *ws, size_t ws_bytes,
                             cudaStream_t st, cudaEvent_t *ev = nullptr)
{
    if (g.model != GBK_MODEL_CUBE)
        return fail(GBK_EUNSUPPORTED, "velocity-field models have no cube (the staged path does not apply)");
    bool own_data = (cubes == nullptr);
    StagedLayout L = staged_layout(g, n, own_data, chi2 != nullptr);
    if (L.total > 0) {
        if (!ws) return fail(GBK_EWORKSPACE, "the staged path needs %zu bytes of workspace", L.total);
        if (ws_bytes < L.total)
            return fail(GBK_EWORKSPACE, "workspace of %zu bytes is smaller than the %zu needed", ws_bytes, L.total);
        gbk_status s = check_device_ptr(ws, "workspace", 256);
        if (s) return s;
    }
    char *base = (char *)ws;
    StagedArgs a = {};
    a.g = g;
    a.n_models = n;
    a.params = params;
    a.ext = (float *)(base + L.off_ext);
    a.e_pitch = L.e_pitch;
    a.e_model_stride = L.e_stride;
    a.data = own_data ? (float *)(base + L.off_data) : cubes;
    a.d_model_stride = L.d_stride;
    if (g.u > 1) {
        a.fine = (float *)(base + L.off_fine);
        a.f_model_stride = L.f_stride;
    } else {
        a.fine = a.data;
        a.f_model_stride = L.d_stride;
    }
    a.maps = maps;
    a.chi2 = chi2;
    a.resid = resid;
    a.partials = chi2 ? (double *)(base + L.off_part) : nullptr;
    if (obs) a.obs = *obs;
    bool want_moments = (maps || chi2 || resid);
    gbk_status s = launch_staged(a, want_moments, st, ev);
    if (s) return s;
    return ok();
}

static gbk_status run_fused(const Geom &g, int32_t n, const double *params, float *maps, const gbk_obs *obs,
                            double *chi2, float *resid, cudaStream_t st)
{
    FusedArgs a = {};
    FusedConfig fc;
    if (!fused_config(g, &fc))
        return fail(GBK_EUNSUPPORTED, "the fused path cannot serve this geometry (upsample %d, %d x %d)", g.u,
                    g.nx, g.ny);
    a.cs = fc.cs;
    a.band = fc.band;
    a.threads = fc.threads;
    a.persistent = fc.persistent;
    a.g = g;
    a.n_models = n;
    a.params = params;
    if (obs) a.obs = *obs;
    a.maps = maps;
    a.chi2 = chi2;
    a.resid = resid;
    if (n == 0) return ok();
    gbk_status s = launch_fused(a, st);
    if (s) return s;
    return ok();
}

gbk_status gbk_eval_cubes(const gbk_geom *gin, int32_t n_models, const double *params, float *cubes,
                          float *maps, void *workspace, size_t ws_bytes, void *stream)
{
    Geom g;
    gbk_status s = derive_geom(gin, &g);
    if (s) return s;
    if (n_models < 0) return fail(GBK_EINVAL, "n_models must be >= 0");
    if (n_models == 0) return ok();
    if ((s = check_device_ptr(params, "params", 8))) return s;
    if (cubes && (s = check_device_ptr(cubes, "cubes", 16))) return s;
    if (maps && (s = check_device_ptr(maps, "maps", 4))) return s;
    if (!cubes && !maps) return ok();
    cudaStream_t st = (cudaStream_t)stream;
    FusedConfig fc;
    if (!cubes && split_fits(g, n_models, workspace, ws_bytes)) {
        if ((s = check_device_ptr(workspace, "workspace", 256))) return s;
        if ((s = launch_split(g, n_models, params, nullptr, maps, nullptr, nullptr, workspace, ws_bytes, st)))
            return s;
        return ok();
    }
    if (cubes || !fused_config(g, &fc))
        return run_staged(g, n_models, params, cubes, maps, nullptr, nullptr, nullptr, workspace, ws_bytes, st);
    return run_fused(g, n_models, params, maps, nullptr, nullptr, nullptr, st);
}

gbk_status gbk_chi2(const gbk_geom *gin, int32_t n_models, const double *params, const gbk_obs *obs,
                    double *chi2, float *resid, uint32_t flags, void *workspace, size_t ws_bytes, void *stream)
{
    Geom g;
    gbk_status s = derive_geom(gin, &g);
    if (s) return s;
    if (n_models < 0) return fail(GBK_EINVAL, "n_models must be >= 0");
    if (flags > GBK_PATH_SPLIT) return fail(GBK_EINVAL, "unknown flags 0x%x", flags);
    if (n_models == 0) return ok();
    if ((s = check_device_ptr(params, "params", 8))) return s;
    if ((s = check_device_ptr(chi2, "chi2", 8))) return s;
    if (resid && (s = check_device_ptr(resid, "resid", 4))) return s;
    if ((s = check_obs(obs))) return s;
    cudaStream_t st = (cudaStream_t)stream;
    FusedConfig fc;
    bool fused_ok = fused_config(g, &fc);
    if (flags == GBK_PATH_SPLIT || (flags == GBK_PATH_AUTO && split_fits(g, n_models, workspace, ws_bytes))) {
        if (workspace && (s = check_device_ptr(workspace, "workspace", 256))) return s;
        if ((s = launch_split(g, n_models, params, obs, nullptr, chi2, resid, workspace, ws_bytes, st))) return s;
        return ok();
    }
    if (flags == GBK_PATH_STAGED || (flags == GBK_PATH_AUTO && !fused_ok))
        return run_staged(g, n_models, params, nullptr, nullptr, obs, chi2, resid, workspace, ws_bytes, st);
    return run_fused(g, n_models, params, nullptr, obs, chi2, resid, st);
}

// Workspace of gbk_chi2_host: the device copies of the parameters, the
// chi2 values and the observed maps, then the split evaluator's region.
struct HostCallLayout {
    size_t params, chi2, maps, mask, split, total;
};

static HostCallLayout host_call_layout(const Geom &g, int n)
{
    HostCallLayout L;
    const size_t np = (size_t)g.nx * g.ny;
    size_t o = 0;
    L.params = o; o += align256(sizeof(double) * GBK_NPAR * n);
    L.chi2 = o; o += align256(sizeof(double) * n);
    L.maps = o; o += align256(sizeof(float) * 4 * np);
    L.mask = o; o += align256(np);
    L.split = o; o += split_workspace_bytes(g, n);
    L.total = o;
    return L;
}

size_t gbk_chi2_host_workspace_bytes(const gbk_geom *gin, int32_t n_models)
{
    ok();
    Geom g;
    if (derive_geom(gin, &g) != GBK_OK) return 0;
    if (n_models < 1) { fail(GBK_EINVAL, "n_models must be >= 1"); return 0; }
    if (!split_supported(g)) { fail(GBK_EUNSUPPORTED, "the split evaluator does not serve this geometry"); return 0; }
    return host_call_layout(g, n_models).total;
}

gbk_status gbk_chi2_host(const gbk_geom *gin, int32_t n_models, const double *params, const gbk_obs *obs,
                         double *chi2, void *workspace, size_t ws_bytes, void *stream)
{
    Geom g;
    gbk_status s = derive_geom(gin, &g);
    if (s) return s;
    if (n_models < 0) return fail(GBK_EINVAL, "n_models must be >= 0");
    if (n_models == 0) return ok();
    if (!params || !chi2 || !obs) return fail(GBK_EINVAL, "params, obs and chi2 must not be NULL");
    if (!obs->v_obs || !obs->s_obs || !obs->w_v || !obs->w_s || !obs->mask)
        return fail(GBK_EINVAL, "every observed map must be given");
    if (!split_supported(g)) return fail(GBK_EUNSUPPORTED, "the split evaluator does not serve this geometry");
    const HostCallLayout L = host_call_layout(g, n_models);
    if (!workspace || ws_bytes < L.total)
        return fail(GBK_EWORKSPACE, "gbk_chi2_host needs %zu bytes of workspace (got %zu)", L.total, ws_bytes);
    if ((s = check_device_ptr(workspace, "workspace", 256))) return s;
    SplitAux *aux = nullptr;
    if ((s = split_aux(&aux))) return s;
    cudaStream_t st = (cudaStream_t)stream;
    char *ws = (char *)workspace;
    const size_t np = (size_t)g.nx * g.ny, mb = sizeof(float) * np;
    double *d_params = (double *)(ws + L.params), *d_chi2 = (double *)(ws + L.chi2);
    float *d_maps = (float *)(ws + L.maps);
    uint8_t *d_mask = (uint8_t *)(ws + L.mask);
    const gbk_obs d_obs = {d_maps, d_maps + np, d_maps + 2 * np, d_maps + 3 * np, d_mask};
    // The parameters go on the caller's stream (the line stage needs them);
    // the maps on the PSF stages' stream, after everything the caller's
    // stream holds (an earlier call's PSF stage may still read this
    // workspace), so that their copy overlaps the line stage.
    cudaError_t e;
    if ((e = cudaMemcpyAsync(d_params, params, sizeof(double) * GBK_NPAR * n_models, cudaMemcpyDefault, st)) ||
        (e = cudaEventRecord(aux->start, st)) || (e = cudaStreamWaitEvent(aux->s, aux->start, 0)) ||
        (e = cudaMemcpyAsync((void *)d_obs.v_obs, obs->v_obs, mb, cudaMemcpyDefault, aux->s)) ||
        (e = cudaMemcpyAsync((void *)d_obs.s_obs, obs->s_obs, mb, cudaMemcpyDefault, aux->s)) ||
        (e = cudaMemcpyAsync((void *)d_obs.w_v, obs->w_v, mb, cudaMemcpyDefault, aux->s)) ||
        (e = cudaMemcpyAsync((void *)d_obs.w_s, obs->w_s, mb, cudaMemcpyDefault, aux->s)) ||
        (e = cudaMemcpyAsync((void *)d_obs.mask, obs->mask, np, cudaMemcpyDefault, aux->s)) ||
        (e = cudaEventRecord(aux->obs, aux->s)))
        return cuda_fail(e, "gbk_chi2_host: copies to the device");
    if ((s = launch_split(g, n_models, d_params, &d_obs, nullptr, d_chi2, nullptr, ws + L.split, L.total - L.split, st,
                          nullptr, nullptr, aux->obs)))
        return s;
    // the last PSF stage is joined to st (or ran on it after the maps'
    // event), so the maps' stream holds nothing past this point
    if ((e = cudaMemcpyAsync(chi2, d_chi2, sizeof(double) * n_models, cudaMemcpyDefault, st)))
        return cuda_fail(e, "gbk_chi2_host: chi2 to the host");
    return ok();
}

gbk_status gbk_chi2_stage_times(const gbk_geom *gin, int32_t n_models, const double *params, const gbk_obs *obs,
                                double *chi2, void *workspace, size_t ws_bytes, float *stage_ms, void *stream)
{
    Geom g;
    gbk_status s = derive_geom(gin, &g);
    if (s) return s;
    if (n_models < 1) return fail(GBK_EINVAL, "n_models must be >= 1");
    if (!stage_ms) return fail(GBK_EINVAL, "stage_ms is NULL");
    if ((s = check_device_ptr(params, "params", 8)) || (s = check_device_ptr(chi2, "chi2", 8)) || (s = check_obs(obs)))
        return s;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t ev[5] = {};
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < 5 && e == cudaSuccess; ++i) e = cudaEventCreate(&ev[i]);
    if (e == cudaSuccess) {
        s = run_staged(g, n_models, params, nullptr, nullptr, obs, chi2, nullptr, workspace, ws_bytes, st, ev);
        if (!s) e = cudaEventSynchronize(ev[4]);
        for (int i = 0; i < 4 && !s && e == cudaSuccess; ++i) e = cudaEventElapsedTime(&stage_ms[i], ev[i], ev[i + 1]);
    }
    for (int i = 0; i < 5; ++i)
        if (ev[i]) cudaEventDestroy(ev[i]);
    if (s) return s;
    if (e != cudaSuccess) return cuda_fail(e, "stage timing");
    return ok();
}

gbk_status gbk_chi2_from_maps(int32_t nx, int32_t ny, int32_t n_models, const float *maps, const gbk_obs *obs,
                              double *chi2, float *resid, void *stream)
{
    if (nx < 1 || ny < 1) return fail(GBK_EINVAL, "map size must be >= 1");
    if (n_models < 0) return fail(GBK_EINVAL, "n_models must be >= 0");
    if (n_models == 0) return ok();
    gbk_status s;
    if ((s = check_device_ptr(maps, "maps", 4))) return s;
    if ((s = check_device_ptr(chi2, "chi2", 8))) return s;
    if (resid && (s = check_device_ptr(resid, "resid", 4))) return s;
    if ((s = check_obs(obs))) return s;
    cudaError_t e = launch_chi2_maps(nx, ny, n_models, maps, *obs, chi2, resid, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "chi2_from_maps launch");
    return ok();
}

}  // extern "C"
