// survey.cu -- ragged survey batches (galaxies of different cube size,
// channel width and LSF in one batch), the setting of the survey-scale
// fitting Bekiaris et al. 2015 motivate in Sec. 1 and Sec. 5.
//
// Two ways to serve a survey with the fused evaluator:
//  * one persistent launch: a resident wave of thread-block clusters of one
//    size (the smallest that fits every galaxy two CTAs to an SM) takes the
//    models, costliest galaxy first, from a work counter as each cluster
//    becomes free;
//  * one launch per class: the galaxies grouped by the smallest cluster that
//    fits each of them, one cluster per model, each group costliest first.
// A per-survey autotuner (gbk_survey_autotune) times both shapes and caches
// the winner for the survey's geometry list.  The geometry table, the packed
// pixel offsets, the orders and the work counter live at the start of the
// caller's workspace.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>

#include "gbk_api_internal.h"
#include "k_fused.h"
#include "k_tangent.h"
#include "k_tsplit.h"
#include "survey.h"

namespace gbk {

static size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

// Shared memory per CTA that lets two CTAs of 512 threads share an SM.
constexpr size_t kSurveySmemCap = 228 * 1024 / 2 - 3 * 1024;

// One persistent launch unless a survey tuning says otherwise.
constexpr int kSurveyDefaultOne = 1;

static std::mutex g_stune_mu;
static std::map<uint64_t, SurveyTuning> g_stune;

// Key of a survey's launch shapes: FNV-1a over the sizes that set them.
static uint64_t survey_key(const std::vector<Geom> &geo)
{
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](int v) {
        for (int k = 0; k < 4; ++k) {
            h ^= (uint64_t)((v >> (8 * k)) & 0xff);
            h *= 1099511628211ull;
        }
    };
    mix((int)geo.size());
    for (const Geom &g : geo) {
        mix(g.nx);
        mix(g.ny);
        mix(g.nz);
        mix(g.R);
        mix(g.Rz);
        mix(g.lsf_mode);
    }
    return h;
}

// Galaxies a single CTA serves with two CTAs per SM (the solo share of a
// persistent launch).
static bool solo_fits(const Geom &g, int threads)
{
    size_t need;
    return fused_config_ragged(&g, 1, 1, threads, &need) && need <= kSurveySmemCap;
}

// Smallest cluster size for the cluster share of one launch (the galaxies
// that are not solo): two CTAs per SM if possible, else one; 1 when every
// galaxy is solo.  0 if none fits.
static int one_launch_cs(const std::vector<Geom> &geo, int threads, size_t *smem)
{
    std::vector<Geom> big;
    for (const Geom &g : geo)
        if (!solo_fits(g, threads)) big.push_back(g);
    if (big.empty()) return fused_config_ragged(geo.data(), (int)geo.size(), 1, threads, smem) ? 1 : 0;
    for (int pass = 0; pass < 2; ++pass) {
        const size_t cap = pass == 0 ? kSurveySmemCap : (size_t)kFusedMaxSmem;
        for (int cs = 1; cs <= kFusedMaxCluster; ++cs) {
            size_t need;
            if (fused_config_ragged(big.data(), (int)big.size(), cs, threads, &need) && need <= cap) {
                *smem = need;
                return cs;
            }
        }
    }
    return 0;
}

gbk_status survey_plan(const gbk_geom *geoms, int n_gal, SurveyPlan *sp, const SurveyTuning *force)
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
    auto cost = [&](int i) { const Geom &g = sp->geo[i]; return (long long)g.ex * g.ey * g.ez; };
    SurveyTuning tu = {kSurveyDefaultOne, 0, 512};
    if (force) {
        tu = *force;
    } else if (n_gal > 0) {
        std::lock_guard<std::mutex> lk(g_stune_mu);
        auto it = g_stune.find(survey_key(sp->geo));
        if (it != g_stune.end()) tu = it->second;
    }
    sp->order.resize(n_gal);
    std::iota(sp->order.begin(), sp->order.end(), 0);
    sp->classes.clear();
    if (tu.one && n_gal > 0) {
        // one persistent launch: the galaxies that need a cluster first, then
        // the ones a single CTA serves; each share costliest first
        SurveyClass c;
        c.threads = tu.threads;
        std::vector<char> solo(n_gal);
        std::vector<Geom> big;
        for (int i = 0; i < n_gal; ++i) {
            solo[i] = solo_fits(sp->geo[i], c.threads);
            if (!solo[i]) big.push_back(sp->geo[i]);
        }
        if (tu.cs > 0) {
            c.cs = tu.cs;
            if (big.empty()) big = sp->geo;  // every galaxy is served by the clusters
            if (!fused_config_ragged(big.data(), (int)big.size(), c.cs, c.threads, &c.smem))
                return fail(GBK_EINVAL, "survey tuning: %d-CTA clusters of %d threads do not fit every galaxy", c.cs,
                            c.threads);
        } else if (!(c.cs = one_launch_cs(sp->geo, c.threads, &c.smem))) {
            return fail(GBK_EUNSUPPORTED, "no cluster size fits every galaxy of the survey");
        }
        // solo galaxies only where a cluster share exists (with none, the
        // clusters serve everything)
        const bool split = (int)big.size() < n_gal && !big.empty() && c.cs > 1;
        c.n_solo = 0;
        if (split) {
            for (int i = 0; i < n_gal; ++i) {
                if (!solo[i]) continue;
                size_t need;
                fused_config_ragged(&sp->geo[i], 1, 1, c.threads, &need);
                c.smem = std::max(c.smem, need);
                ++c.n_solo;
            }
        } else {
            std::fill(solo.begin(), solo.end(), 0);
            if (!fused_config_ragged(sp->geo.data(), n_gal, c.cs, c.threads, &c.smem))
                return fail(GBK_EINVAL, "survey tuning: %d-CTA clusters of %d threads do not fit every galaxy", c.cs,
                            c.threads);
        }
        c.beg = 0;
        c.end = n_gal;
        c.persistent = 1;
        std::stable_sort(sp->order.begin(), sp->order.end(), [&](int a, int b) {
            if (solo[a] != solo[b]) return solo[a] < solo[b];
            return cost(a) > cost(b);
        });
        sp->classes.push_back(c);
        tu.cs = c.cs;
    }
    // groups: larger clusters first, then costliest first; ties by index
    if (!tu.one)
        std::stable_sort(sp->order.begin(), sp->order.end(), [&](int a, int b) {
            if (cs_of[a] != cs_of[b]) return cs_of[a] > cs_of[b];
            if (thr_of[a] != thr_of[b]) return thr_of[a] > thr_of[b];
            return cost(a) > cost(b);
        });
    sp->tuning = tu;
    for (int k = 0; k < n_gal && !tu.one;) {
        int i0 = sp->order[k], e = k;
        while (e < n_gal && cs_of[sp->order[e]] == cs_of[i0] && thr_of[sp->order[e]] == thr_of[i0]) ++e;
        SurveyClass c;
        c.cs = cs_of[i0];
        c.threads = thr_of[i0];
        c.beg = k;
        c.end = e;
        c.persistent = 0;
        c.n_solo = 0;
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
        // galaxies whose halo rows do not fit the CTA (direct shape) are
        // fitted faster with finite differences of the fused evaluator
        if (tcs[i] == 0 || tangent_key_direct(tcs[i])) sp->tangent_ok = false;
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
        c.cs = tangent_key_cs(tcs[i0]);
        c.direct = tangent_key_direct(tcs[i0]);
        c.threads = kTangentThreads;
        c.beg = k;
        c.end = e;
        c.smem = 0;
        c.persistent = 0;
        c.n_solo = 0;
        for (int j = k; j < e; ++j) {
            const Geom &g = sp->geo[sp->torder[j]];
            c.smem = std::max(c.smem,
                              tangent_smem_bytes_host(g, (g.ey + c.cs - 1) / c.cs, kTangentThreads, c.direct, true));
        }
        sp->tclasses.push_back(c);
        k = e;
    }
    sp->table_bytes = n_gal == 0 ? 0
                                 : al256(sizeof(Geom) * n_gal) + al256(sizeof(int64_t) * (n_gal + 1)) +
                                       2 * al256(sizeof(int32_t) * n_gal) + al256(2 * sizeof(int));
    return GBK_OK;
}

// Host image of the device tables: geometry, pixel offsets, the two
// orders; the work counters that follow are reset on the device.
static void build_host_tables(SurveyPlan *sp)
{
    const int n = sp->n_gal;
    size_t o_geo = 0, o_pix = al256(sizeof(Geom) * n), o_ord = o_pix + al256(sizeof(int64_t) * (n + 1));
    size_t o_tord = o_ord + al256(sizeof(int32_t) * n);
    std::vector<char> &h = sp->h_tables;
    h.assign(sp->table_bytes, 0);
    if (n == 0) return;
    std::memcpy(h.data() + o_geo, sp->geo.data(), sizeof(Geom) * n);
    std::memcpy(h.data() + o_pix, sp->pix_off.data(), sizeof(int64_t) * (n + 1));
    std::memcpy(h.data() + o_ord, sp->order.data(), sizeof(int32_t) * n);
    std::memcpy(h.data() + o_tord, sp->torder.data(), sizeof(int32_t) * n);
}

// Recent plans, newest first, with the generation of the survey tunings
// they were made under.
struct CachedPlan {
    std::vector<unsigned char> key;  // the caller's gbk_geom array, byte for byte
    uint64_t gen;
    SurveyPlan plan;
};
static std::mutex g_plan_mu;
static std::vector<CachedPlan> g_plans;
static uint64_t g_tune_gen = 0;  // bumped whenever a survey tuning changes (under g_stune_mu)
constexpr size_t kPlanCache = 4;

gbk_status survey_plan_cached(const gbk_geom *geoms, int n_gal, SurveyPlan *sp)
{
    if (!geoms || n_gal <= 0) return survey_plan(geoms, n_gal, sp);
    const size_t nb = sizeof(gbk_geom) * (size_t)n_gal;
    uint64_t gen;
    {
        std::lock_guard<std::mutex> lk(g_stune_mu);
        gen = g_tune_gen;
    }
    {
        std::lock_guard<std::mutex> lk(g_plan_mu);
        for (size_t i = 0; i < g_plans.size(); ++i) {
            const CachedPlan &c = g_plans[i];
            if (c.gen == gen && c.key.size() == nb && std::memcmp(c.key.data(), geoms, nb) == 0) {
                *sp = c.plan;
                return GBK_OK;
            }
        }
    }
    gbk_status s = survey_plan(geoms, n_gal, sp);
    if (s) return s;
    build_host_tables(sp);
    CachedPlan c;
    c.key.assign((const unsigned char *)geoms, (const unsigned char *)geoms + nb);
    c.gen = gen;
    c.plan = *sp;
    std::lock_guard<std::mutex> lk(g_plan_mu);
    g_plans.insert(g_plans.begin(), std::move(c));
    if (g_plans.size() > kPlanCache) g_plans.pop_back();
    return GBK_OK;
}

gbk_status survey_upload(SurveyPlan *sp, char *ws, cudaStream_t st)
{
    const int n = sp->n_gal;
    size_t o_geo = 0, o_pix = al256(sizeof(Geom) * n), o_ord = o_pix + al256(sizeof(int64_t) * (n + 1));
    size_t o_tord = o_ord + al256(sizeof(int32_t) * n), o_work = o_tord + al256(sizeof(int32_t) * n);
    if (sp->h_tables.size() != sp->table_bytes) build_host_tables(sp);
    // From pageable memory the copy returns once the source has been staged,
    // so the host image may be released afterwards.
    cudaError_t e = cudaMemcpyAsync(ws, sp->h_tables.data(), sp->h_tables.size(), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "survey: uploading the geometry tables");
    sp->d_geo = (Geom *)(ws + o_geo);
    sp->d_pix_off = (int64_t *)(ws + o_pix);
    sp->d_order = (int32_t *)(ws + o_ord);
    sp->d_torder = (int32_t *)(ws + o_tord);
    sp->d_work = (int *)(ws + o_work);
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
        a.direct = c.direct;
        a.geoms = sp.d_geo;
        a.order = sp.d_torder + c.beg;
        a.smem = c.smem;
        gbk_status s = launch_tangent(a, st);
        if (s) return s;
    }
    return GBK_OK;
}

void survey_live(const SurveyPlan &sp, const std::vector<char> &active, SurveyLive *live,
                 std::vector<int32_t> *order)
{
    live->classes.clear();
    live->rep.clear();
    order->clear();
    for (const SurveyClass &c : sp.classes) {
        SurveyClass k = c;
        k.beg = (int)order->size();
        int solo = 0;
        for (int i = c.beg; i < c.end; ++i) {
            const int gal = sp.order[i];
            if (!active[gal]) continue;
            order->push_back(gal);
            if (i >= c.end - c.n_solo) ++solo;
        }
        k.end = (int)order->size();
        k.n_solo = solo;
        if (k.end > k.beg) {
            live->classes.push_back(k);
            live->rep.push_back(sp.order[c.beg]);
        }
    }
}

gbk_status survey_eval(const SurveyPlan &sp, int mpg, const double *params, const gbk_obs *obs_list,
                       const int32_t *skip, float *maps, double *chi2, float *resid, cudaStream_t st,
                       const SurveyLive *live)
{
    const std::vector<SurveyClass> &classes = live ? live->classes : sp.classes;
    const int32_t *d_order = live ? live->d_order : sp.d_order;
    for (size_t ci = 0; ci < classes.size(); ++ci) {
        const SurveyClass &c = classes[ci];
        FusedArgs a = {};
        a.g = sp.geo[live ? live->rep[ci] : sp.order[c.beg]];
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
        a.persistent = c.persistent;
        a.geoms = sp.d_geo;
        a.pix_off = sp.d_pix_off;
        a.order = d_order + c.beg;
        a.smem = c.smem;
        if (c.persistent) {
            cudaError_t e = cudaMemsetAsync(sp.d_work, 0, 2 * sizeof(int), st);
            if (e != cudaSuccess) return cuda_fail(e, "survey: resetting the work counters");
            a.work = sp.d_work;
            a.n_solo = c.n_solo * mpg;
        }
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
    gbk_status s = survey_plan_cached(geoms, n_gal, &sp);
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

size_t gbk_survey_jacobian_workspace_bytes(const gbk_geom *geoms, int32_t n_gal, uint32_t free_mask)
{
    ok();
    if (free_mask == 0 || (free_mask >> GBK_I0)) {
        fail(GBK_EINVAL, "free_mask must select parameters among x0 .. sigma0");
        return 0;
    }
    SurveyPlan sp;
    if (survey_plan(geoms, n_gal, &sp)) return 0;
    TsRaggedPlan rp;
    tsplit_ragged_plan(sp.geo, &rp);
    if (!rp.ok) {
        fail(GBK_EUNSUPPORTED, "the split Jacobian does not serve this batch (PSF radius <= 8, u = 1, cube model)");
        return 0;
    }
    return sp.table_bytes + rp.total;
}

gbk_status gbk_survey_jacobian(const gbk_geom *geoms, int32_t n_gal, const double *params, const gbk_obs *obs,
                               uint32_t free_mask, double *jtj, double *jtv, double *chi2, void *workspace,
                               size_t ws_bytes, void *stream)
{
    if (free_mask == 0 || (free_mask >> GBK_I0))
        return fail(GBK_EINVAL, "free_mask must select parameters among x0 .. sigma0");
    SurveyPlan sp;
    gbk_status s = survey_plan_cached(geoms, n_gal, &sp);
    if (s) return s;
    if (n_gal == 0) return ok();
    TsRaggedPlan rp;
    tsplit_ragged_plan(sp.geo, &rp);
    if (!rp.ok) return fail(GBK_EUNSUPPORTED, "the split Jacobian does not serve this batch (PSF radius <= 8, u = 1, cube model)");
    if ((s = check_device_ptr(params, "params", 8)) || (s = check_device_ptr(obs, "obs", 8))) return s;
    if (jtj && (s = check_device_ptr(jtj, "jtj", 8))) return s;
    if (jtv && (s = check_device_ptr(jtv, "jtv", 8))) return s;
    if (chi2 && (s = check_device_ptr(chi2, "chi2", 8))) return s;
    const size_t need = sp.table_bytes + rp.total;
    if (!workspace || ws_bytes < need)
        return fail(GBK_EWORKSPACE, "gbk_survey_jacobian needs %zu bytes of workspace (got %zu)", need, ws_bytes);
    if ((s = check_device_ptr(workspace, "workspace", 256))) return s;
    cudaStream_t st = (cudaStream_t)stream;
    char *ws = (char *)workspace;
    if ((s = survey_upload(&sp, ws, st)) || (s = tsplit_ragged_upload(rp, ws + sp.table_bytes, st))) return s;
    TsplitRaggedCall c = {};
    c.d_geo = sp.d_geo;
    c.params = params;
    c.obs_list = obs;
    c.skip = nullptr;
    for (int k = 0; k < GBK_I0; ++k)
        if (free_mask & (1u << k)) c.free_idx[c.np++] = k;
    c.jtj = jtj;
    c.jtv = jtv;
    c.chi2 = chi2;
    if ((s = launch_tsplit_ragged(rp, c, ws + sp.table_bytes, st))) return s;
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

gbk_status gbk_survey_autotune(const gbk_geom *geoms, int32_t n_gal, const double *params, const gbk_obs *obs,
                               double *chi2_scratch, void *workspace, size_t ws_bytes, gbk_tuning *best, void *stream)
{
    SurveyPlan base;
    gbk_status s = survey_plan(geoms, n_gal, &base);
    if (s) return s;
    if (n_gal < 1) return fail(GBK_EINVAL, "n_gal must be >= 1");
    if (!best) return fail(GBK_EINVAL, "best is NULL");
    if ((s = check_device_ptr(params, "params", 8)) || (s = check_device_ptr(chi2_scratch, "chi2_scratch", 8)) ||
        (s = check_device_ptr(obs, "obs", 8)))
        return s;
    if (!workspace || ws_bytes < base.table_bytes)
        return fail(GBK_EWORKSPACE, "gbk_survey_autotune needs %zu bytes of workspace (got %zu)", base.table_bytes,
                    ws_bytes);
    if ((s = check_device_ptr(workspace, "workspace", 256))) return s;
    // candidates: the per-class launches, and one launch with 256 or 512
    // threads and the four smallest cluster sizes that fit every galaxy
    std::vector<SurveyTuning> cand = {{0, 0, 0}};
    for (int threads : {512, 256}) {
        size_t smem;
        const int cs0 = one_launch_cs(base.geo, threads, &smem);
        for (int cs = cs0; cs0 > 0 && cs < cs0 + 4 && cs <= kFusedMaxCluster; ++cs)
            if (fused_config_ragged(base.geo.data(), n_gal, cs, threads, &smem)) cand.push_back({1, cs, threads});
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    SurveyTuning bt = {0, 0, 0};
    float best_ms = 0.f;
    int tried = 0;
    for (const SurveyTuning &c : cand) {
        SurveyPlan p;
        if (survey_plan(geoms, n_gal, &p, &c) || survey_upload(&p, (char *)workspace, st)) continue;
        if (survey_eval(p, 1, params, obs, nullptr, nullptr, chi2_scratch, nullptr, st)) {  // warm-up
            cudaGetLastError();
            continue;
        }
        float times[3];
        bool ok_run = true;
        for (int rep = 0; rep < 3 && ok_run; ++rep) {
            cudaEventRecord(t0, st);
            ok_run = survey_eval(p, 1, params, obs, nullptr, nullptr, chi2_scratch, nullptr, st) == GBK_OK;
            cudaEventRecord(t1, st);
            cudaEventSynchronize(t1);
            cudaEventElapsedTime(&times[rep], t0, t1);
        }
        if (!ok_run) {
            cudaGetLastError();
            continue;
        }
        const float med =
            std::fmax(std::fmin(times[0], times[1]), std::fmin(std::fmax(times[0], times[1]), times[2]));
        if (tried++ == 0 || med < best_ms) {
            best_ms = med;
            bt = p.tuning;
        }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "survey autotune");
    if (tried == 0) return fail(GBK_EUNSUPPORTED, "no survey launch shape could run");
    {
        std::lock_guard<std::mutex> lk(g_stune_mu);
        g_stune[survey_key(base.geo)] = bt;
        ++g_tune_gen;
    }
    best->cluster_ctas = bt.one ? bt.cs : 0;
    best->threads = bt.one ? bt.threads : 0;
    best->persistent = bt.one;
    best->ms = best_ms;
    best->candidates = tried;
    return ok();
}

gbk_status gbk_survey_get_tuning(const gbk_geom *geoms, int32_t n_gal, gbk_tuning *out)
{
    if (!out) return fail(GBK_EINVAL, "out is NULL");
    if (n_gal < 1) return fail(GBK_EINVAL, "n_gal must be >= 1");
    SurveyPlan sp;
    gbk_status s = survey_plan(geoms, n_gal, &sp);
    if (s) return s;
    out->cluster_ctas = sp.tuning.one ? sp.tuning.cs : 0;
    out->threads = sp.tuning.one ? sp.tuning.threads : 0;
    out->persistent = sp.tuning.one;
    out->ms = 0.f;
    out->candidates = 0;
    return ok();
}

gbk_status gbk_survey_set_tuning(const gbk_geom *geoms, int32_t n_gal, const gbk_tuning *t)
{
    if (n_gal < 1) return fail(GBK_EINVAL, "n_gal must be >= 1");
    SurveyPlan sp;
    gbk_status s = survey_plan(geoms, n_gal, &sp);
    if (s) return s;
    const uint64_t key = survey_key(sp.geo);
    if (!t) {
        std::lock_guard<std::mutex> lk(g_stune_mu);
        g_stune.erase(key);
        ++g_tune_gen;
        return ok();
    }
    if (t->persistent != 0 && t->persistent != 1) return fail(GBK_EINVAL, "persistent must be 0 or 1");
    SurveyTuning tu = {t->persistent, t->persistent ? t->cluster_ctas : 0, t->persistent ? t->threads : 0};
    if (tu.one && (tu.cs < 1 || (tu.threads != 512 && tu.threads != 384 && tu.threads != 256)))
        return fail(GBK_EINVAL, "one launch needs cluster_ctas >= 1 and 256, 384 or 512 threads");
    SurveyPlan check;
    if ((s = survey_plan(geoms, n_gal, &check, &tu))) return s;
    std::lock_guard<std::mutex> lk(g_stune_mu);
    g_stune[key] = tu;
    ++g_tune_gen;
    return ok();
}

}  // extern "C"
