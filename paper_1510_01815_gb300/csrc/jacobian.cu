// jacobian.cu -- gbk_jacobian: host side of the analytic Jacobian kernel.
#include "gbk_api_internal.h"
#include "k_tangent.h"
#include "k_tsplit.h"

using namespace gbk;

extern "C" gbk_status gbk_jacobian(const gbk_geom *gin, int32_t n_models, const double *params,
                                   const gbk_obs *obs, uint32_t free_mask, const float *cot, double *jtj,
                                   double *jtv, double *chi2, float *jac, void *stream)
{
    Geom g;
    gbk_status s = derive_geom(gin, &g);
    if (s) return s;
    if (n_models < 0) return fail(GBK_EINVAL, "n_models must be >= 0");
    if (free_mask == 0 || (free_mask >> GBK_NPAR)) return fail(GBK_EINVAL, "free_mask must select 1..10 parameters");
    if (g.u != 1) return fail(GBK_EUNSUPPORTED, "the Jacobian kernel needs upsample == 1");
    TangentArgs a = {};
    a.jac = jac;
    a.np = 0;
    for (int k = 0; k < GBK_NPAR; ++k)
        if (free_mask & (1u << k)) a.free_idx[a.np++] = k;
    // velocity fields: one CTA per model, no shared-memory records
    if (g.model == GBK_MODEL_CUBE && !tangent_config(g, &a.cs, &a.band, &a.direct, tangent_narrow(a)))
        return fail(GBK_EUNSUPPORTED, "geometry %d x %d too large for the Jacobian kernel", g.nx, g.ny);
    if (n_models == 0) return ok();
    if ((s = check_device_ptr(params, "params", 8))) return s;
    if ((s = check_obs(obs))) return s;
    if (cot && (s = check_device_ptr(cot, "cot", 4))) return s;
    if (jtj && (s = check_device_ptr(jtj, "jtj", 8))) return s;
    if (jtv && (s = check_device_ptr(jtv, "jtv", 8))) return s;
    if (chi2 && (s = check_device_ptr(chi2, "chi2", 8))) return s;
    if (jac && (s = check_device_ptr(jac, "jac", 4))) return s;
    a.g = g;
    a.n_models = n_models;
    a.params = params;
    a.obs = *obs;
    a.cot = cot;
    a.jtj = jtj;
    a.jtv = jtv;
    a.chi2 = chi2;
    a.jac = jac;
    if ((s = launch_tangent(a, (cudaStream_t)stream))) return s;
    return ok();
}

extern "C" size_t gbk_jacobian_workspace_bytes(const gbk_geom *gin, int32_t n_models, uint32_t free_mask)
{
    ok();
    Geom g;
    if (derive_geom(gin, &g)) return 0;
    if (n_models < 0) { fail(GBK_EINVAL, "n_models must be >= 0"); return 0; }
    int np = 0, idx[GBK_NPAR];
    for (int k = 0; k < GBK_NPAR; ++k)
        if (free_mask & (1u << k)) idx[np++] = k;
    if (!tsplit_supported(g, np, idx)) {
        fail(GBK_EUNSUPPORTED, "the split Jacobian serves the cube model at u = 1, PSF radius <= %d, with free "
             "parameters among x0 .. sigma0", kTsplitMaxR);
        return 0;
    }
    return n_models ? tsplit_workspace_bytes(g, n_models) : 0;
}

extern "C" gbk_status gbk_jacobian_ws(const gbk_geom *gin, int32_t n_models, const double *params,
                                      const gbk_obs *obs, uint32_t free_mask, const float *cot, double *jtj,
                                      double *jtv, double *chi2, void *workspace, size_t ws_bytes, void *stream)
{
    Geom g;
    gbk_status s = derive_geom(gin, &g);
    if (s) return s;
    if (n_models < 0) return fail(GBK_EINVAL, "n_models must be >= 0");
    if (free_mask == 0 || (free_mask >> GBK_NPAR)) return fail(GBK_EINVAL, "free_mask must select 1..10 parameters");
    TsplitCall c = {};
    for (int k = 0; k < GBK_NPAR; ++k)
        if (free_mask & (1u << k)) c.free_idx[c.np++] = k;
    if (!tsplit_supported(g, c.np, c.free_idx))
        return fail(GBK_EUNSUPPORTED, "the split Jacobian serves the cube model at u = 1, PSF radius <= %d, with free "
                    "parameters among x0 .. sigma0", kTsplitMaxR);
    if (n_models == 0) return ok();
    if ((s = check_device_ptr(params, "params", 8))) return s;
    if ((s = check_obs(obs))) return s;
    if (cot && (s = check_device_ptr(cot, "cot", 4))) return s;
    if (jtj && (s = check_device_ptr(jtj, "jtj", 8))) return s;
    if (jtv && (s = check_device_ptr(jtv, "jtv", 8))) return s;
    if (chi2 && (s = check_device_ptr(chi2, "chi2", 8))) return s;
    if (workspace && (s = check_device_ptr(workspace, "workspace", 256))) return s;
    c.g = g;
    c.n_models = n_models;
    c.params = params;
    c.obs = *obs;
    c.cot = cot;
    c.jtj = jtj;
    c.jtv = jtv;
    c.chi2 = chi2;
    if ((s = launch_tsplit(c, workspace, ws_bytes, (cudaStream_t)stream))) return s;
    return ok();
}
