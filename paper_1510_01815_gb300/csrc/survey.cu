// survey.cu -- ragged survey batches (galaxies of different cube size,
// channel width and LSF in one batch), the setting of the survey-scale
// fitting Bekiaris et al. 2015 motivate in Sec. 1 and Sec. 5.
//
// The plan groups the galaxies by the smallest thread-block cluster whose
// per-CTA shared memory still lets two CTAs share an SM (small cubes need one
// CTA, the largest several), orders each group costliest first so that the
// hardware block scheduler, which hands out one cluster per model, ends with
// the cheap models, and issues one ragged fused launch per group.  The
// geometry table, the packed pixel offsets and the order live at the start of
// the caller's workspace.
#include <algorithm>
#include <cstring>
#include <numeric>

#include "gbk_api_internal.h"
#include "k_fused.h"
#include "k_tangent.h"
#include "survey.h"

namespace gbk {

static size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

// Shared memory per CTA that lets two CTAs of 512 threads share an SM.
constexpr size_t kSurveySmemCap = 228 * 1024 / 2 - 3 * 1024;

gbk_status survey_plan(const gbk_geom *geoms, int n_gal, SurveyPlan *sp)
{
    if (!geoms) return fail(GBK_EINVAL, "geoms is NULL");
    if (n_gal < 0) return fail(GBK_EINVAL, "n_gal must be >= 0");
    sp->n_gal = n_gal;
    sp->geo.resize(n_gal);
    sp->pix_off.assign(n_gal + 1, 0);
    std::vector<int> cs_of(n_gal), thr_of(n_gal);
    for (int i = 0; i < n_gal; ++i) {
        gbk_status s = derive_geom(&geoms[i], &sp->geo[i]);
        if (s) return fail(s, "galaxy %d: %s", i, gbk_last_error());
        const Geom &g = sp->geo[i];
        if (g.u != 1) return fail(GBK_EUNSUPPORTED, "galaxy %d: survey batches need upsample == 1", i);
        if (g.model != GBK_MODEL_CUBE)
            return fail(GBK_EUNSUPPORTED, "galaxy %d: survey batches serve the intensity-cube model", i);
        sp->pix_off[i + 1] = sp->pix_off[i] + (int64_t)g.nx * g.ny;
        int pick = 0;
        for (int pass = 0; pass < 2 && !pick; ++pass) {
            size_t cap = pass == 0 ? kSurveySmemCap : (size_t)kFusedMaxSmem;
            for (int cs = 1; cs <= kFusedMaxCluster && cs <= g.ey; ++cs) {
                size_t need;
                if (fused_config_ragged(&g, 1, cs, 512, &need) && need <= cap) {
                    pick = cs;
                    break;
                }
            }
        }
        if (!pick) return fail(GBK_EUNSUPPORTED, "galaxy %d (%d x %d x %d) is too large for the fused path", i, g.nx, g.ny, g.nz);
        cs_of[i] = pick;
        // small bands leave most of a 512-thread block idle
        int band = (g.ey + pick - 1) / pick;
        thr_of[i] = (long)band * g.ex >= 1536 ? 512 : 256;
    }
    // groups: larger clusters first, then costliest first; ties by index
    sp->order.resize(n_gal);
    std::iota(sp->order.begin(), sp->order.end(), 0);
    auto cost = [&](int i) { const Geom &g = sp->geo[i]; return (long long)g.ex * g.ey * g.ez; };
    std::stable_sort(sp->order.begin(), sp->order.end(), [&](int a, int b) {
        if (cs_of[a] != cs_of[b]) return cs_of[a] > cs_of[b];
        if (thr_of[a] != thr_of[b]) return thr_of[a] > thr_of[b];
        return cost(a) > cost(b);
    });
    sp->classes.clear();
    for (int k = 0; k < n_gal;) {
        int i0 = sp->order[k], e = k;
        while (e < n_gal && cs_of[sp->order[e]] == cs_of[i0] && thr_of[sp->order[e]] == thr_of[i0]) ++e;
        SurveyClass c;
        c.cs = cs_of[i0];
        c.threads = thr_of[i0];
        c.beg = k;
        c.end = e;
        std::vector<Geom> members;
        for (int j = k; j < e; ++j) members.push_back(sp->geo[sp->order[j]]);
        if (!fused_config_ragged(members.data(), (int)members.size(), c.cs, c.threads, &c.smem))
            return fail(GBK_EUNSUPPORTED, "survey class with %d-CTA clusters does not fit", c.cs);
        sp->classes.push_back(c);
        k = e;
    }
    // classes of the analytic Jacobian kernel: smallest cluster whose CTAs fit
    std::vector<int> tcs(n_gal);
    sp->tangent_ok = true;
    for (int i = 0; i < n_gal; ++i) {
        tcs[i] = tangent_cluster_for(sp->geo[i]);
        if (tcs[i] == 0) sp->tangent_ok = false;
    }
    sp->torder.resize(n_gal);
    std::iota(sp->torder.begin(), sp->torder.end(), 0);
    std::stable_sort(sp->torder.begin(), sp->torder.end(), [&](int a, int b) {
        if (tcs[a] != tcs[b]) return tcs[a] > tcs[b];
        return cost(a) > cost(b);
    });
    sp->tclasses.clear();
    for (int k = 0; k < n_gal && sp->tangent_ok;) {
        int i0 = sp->torder[k], e = k;
        while (e < n_gal && tcs[sp->torder[e]] == tcs[i0]) ++e;
        SurveyClass c;
        c.cs = tcs[i0];
        c.threads = kTangentThreads;
        c.beg = k;
        c.end = e;
        c.smem = 0;
        for (int j = k; j < e; ++j) {
            const Geom &g = sp->geo[sp->torder[j]];
            c.smem = std::max(c.smem, tangent_smem_bytes_host(g, (g.ey + c.cs - 1) / c.cs, kTangentThreads));
        }
        sp->tclasses.push_back(c);
        k = e;
    }
    sp->table_bytes = n_gal == 0 ? 0
                                 : al256(sizeof(Geom) * n_gal) + al256(sizeof(int64_t) * (n_gal + 1)) +
                                       2 * al256(sizeof(int32_t) * n_gal);
    return GBK_OK;
}

gbk_status survey_upload(SurveyPlan *sp, char *ws, cudaStream_t st)
{
    const int n = sp->n_gal;
    size_t o_geo = 0, o_pix = al256(sizeof(Geom) * n), o_ord = o_pix + al256(sizeof(int64_t) * (n + 1));
    size_t o_tord = o_ord + al256(sizeof(int32_t) * n);
    std::vector<char> h(sp->table_bytes, 0);
    std::memcpy(h.data() + o_geo, sp->geo.data(), sizeof(Geom) * n);
    std::memcpy(h.data() + o_pix, sp->pix_off.data(), sizeof(int64_t) * (n + 1));
    std::memcpy(h.data() + o_ord, sp->order.data(), sizeof(int32_t) * n);
    std::memcpy(h.data() + o_tord, sp->torder.data(), sizeof(int32_t) * n);
    // From pageable memory the copy returns once the source has been staged,
    // so h may be released afterwards.
    cudaError_t e = cudaMemcpyAsync(ws, h.data(), h.size(), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "survey: uploading the geometry tables");
    sp->d_geo = (Geom *)(ws + o_geo);
    sp->d_pix_off = (int64_t *)(ws + o_pix);
    sp->d_order = (int32_t *)(ws + o_ord);
    sp->d_torder = (int32_t *)(ws + o_tord);
    return GBK_OK;
}

gbk_status survey_tangent(const SurveyPlan &sp, const TangentArgs &proto, cudaStream_t st)
{
    if (!sp.tangent_ok) return fail(GBK_EUNSUPPORTED, "a galaxy of the batch is too large for the Jacobian kernel");
    for (const SurveyClass &c : sp.tclasses) {
        TangentArgs a = proto;
        a.g = sp.geo[sp.torder[c.beg]];
        a.n_models = c.end - c.beg;
        a.models_per_gal = 1;
        a.jac = nullptr;
        a.cot = nullptr;
        a.cs = c.cs;
        a.band = 0;
        a.geoms = sp.d_geo;
        a.order = sp.d_torder + c.beg;
        a.smem = c.smem;
        gbk_status s = launch_tangent(a, st);
        if (s) return s;
    }
    return GBK_OK;
}

gbk_status survey_eval(const SurveyPlan &sp, int mpg, const double *params, const gbk_obs *obs_list,
                       const int32_t *skip, float *maps, double *chi2, float *resid, cudaStream_t st)
{
    for (const SurveyClass &c : sp.classes) {
        FusedArgs a = {};
        a.g = sp.geo[sp.order[c.beg]];
        a.n_models = (c.end - c.beg) * mpg;
        a.params = params;
        a.obs_list = obs_list;
        a.models_per_gal = mpg;
        a.skip = skip;
        a.maps = maps;
        a.chi2 = chi2;
        a.resid = resid;
        a.cs = c.cs;
        a.band = 0;
        a.threads = c.threads;
        a.persistent = 0;
        a.geoms = sp.d_geo;
        a.pix_off = sp.d_pix_off;
        a.order = sp.d_order + c.beg;
        a.smem = c.smem;
        gbk_status s = launch_fused(a, st);
        if (s) return s;
    }
    return GBK_OK;
}

// Batched LM over a plan (lm.cu).
gbk_status lm_survey(SurveyPlan &sp, const gbk_geom *geoms, const gbk_obs *obs, const double *lo, const double *hi,
                     double *params, const gbk_lm_opts *o, double *chi2_out, int32_t *iters_out, int32_t *status_out,
                     char *ws, size_t ws_bytes, cudaStream_t st);
size_t lm_survey_workspace(const SurveyPlan &sp, const gbk_geom *geoms, const gbk_lm_opts *o);

}  // namespace gbk

using namespace gbk;

extern "C" {

size_t gbk_survey_workspace_bytes(const gbk_geom *geoms, int32_t n_gal, const gbk_lm_opts *opts)
{
    ok();
    SurveyPlan sp;
    if (survey_plan(geoms, n_gal, &sp)) return 0;
    if (!opts) return sp.table_bytes;
    size_t lm = lm_survey_workspace(sp, geoms, opts);
    if (lm == 0) return 0;
    return sp.table_bytes + lm;
}

gbk_status gbk_survey_eval(const gbk_geom *geoms, int32_t n_gal, const double *params, const gbk_obs *obs,
                           float *maps, double *chi2, float *resid, void *workspace, size_t ws_bytes, void *stream)
{
    SurveyPlan sp;
    gbk_status s = survey_plan(geoms, n_gal, &sp);
    if (s) return s;
    if (n_gal == 0) return ok();
    if ((s = check_device_ptr(params, "params", 8))) return s;
    if (maps && (s = check_device_ptr(maps, "maps", 4))) return s;
    if (chi2 && (s = check_device_ptr(chi2, "chi2", 8))) return s;
    if (resid && (s = check_device_ptr(resid, "resid", 4))) return s;
    if ((chi2 || resid) && (s = check_device_ptr(obs, "obs", 8))) return s;
    if (!maps && !chi2 && !resid) return ok();
    if (!workspace || ws_bytes < sp.table_bytes)
        return fail(GBK_EWORKSPACE, "gbk_survey_eval needs %zu bytes of workspace (got %zu)", sp.table_bytes, ws_bytes);
    if ((s = check_device_ptr(workspace, "workspace", 256))) return s;
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = survey_upload(&sp, (char *)workspace, st))) return s;
    if ((s = survey_eval(sp, 1, params, (chi2 || resid) ? obs : nullptr, nullptr, maps, chi2, resid, st))) return s;
    return ok();
}

gbk_status gbk_survey_fit_lm(const gbk_geom *geoms, int32_t n_gal, const gbk_obs *obs, const double *lo,
                             const double *hi, double *params, const gbk_lm_opts *opts, double *chi2_out,
                             int32_t *iters_out, int32_t *status_out, void *workspace, size_t ws_bytes, void *stream)
{
    SurveyPlan sp;
    gbk_status s = survey_plan(geoms, n_gal, &sp);
    if (s) return s;
    if (!opts) return fail(GBK_EINVAL, "opts is NULL");
    size_t lm = lm_survey_workspace(sp, geoms, opts);
    if (lm == 0) return fail(GBK_EINVAL, "%s", gbk_last_error());
    if (n_gal == 0) return ok();
    if ((s = check_device_ptr(obs, "obs", 8)) || (s = check_device_ptr(lo, "lo", 8)) ||
        (s = check_device_ptr(hi, "hi", 8)) || (s = check_device_ptr(params, "params", 8)) ||
        (s = check_device_ptr(chi2_out, "chi2_out", 8)) || (s = check_device_ptr(iters_out, "iters_out", 4)) ||
        (s = check_device_ptr(status_out, "status_out", 4)))
        return s;
    if (!workspace || ws_bytes < sp.table_bytes + lm)
        return fail(GBK_EWORKSPACE, "gbk_survey_fit_lm needs %zu bytes of workspace (got %zu)", sp.table_bytes + lm,
                    ws_bytes);
    if ((s = check_device_ptr(workspace, "workspace", 256))) return s;
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = survey_upload(&sp, (char *)workspace, st))) return s;
    return lm_survey(sp, geoms, obs, lo, hi, params, opts, chi2_out, iters_out, status_out,
                     (char *)workspace + sp.table_bytes, ws_bytes - sp.table_bytes, st);
}

}  // extern "C"
