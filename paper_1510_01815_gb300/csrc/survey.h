// survey.h -- ragged batches: galaxies of different geometry in one batch
// (host-side plan and launcher of the fused kernel's ragged mode).
#pragma once

#include <vector>

#include "gbk_internal.cuh"

namespace gbk {

// Galaxies served by one launch: the same cluster size and block size.
struct SurveyClass {
    int cs, threads;
    int beg, end;    // range of SurveyPlan::order
    size_t smem;     // dynamic shared memory of the launch
    int persistent;  // 1: one resident wave of clusters fed by the work counters
    int n_solo;      // persistent: the last n_solo galaxies of the range go to single CTAs
    int direct = 0;  // Jacobian classes: halo rows read in the neighbours' shared memory
};

// How the fused evaluator serves a survey: one launch per class (one = 0),
// or one persistent launch of cs-CTA clusters of `threads` threads over
// every galaxy (one = 1).
struct SurveyTuning {
    int one, cs, threads;
};

struct SurveyPlan {
    int n_gal = 0;
    std::vector<Geom> geo;          // derived geometry per galaxy
    std::vector<int64_t> pix_off;   // n_gal + 1 prefix sums of nx * ny
    std::vector<int32_t> order;     // galaxies grouped by class, costliest first
    std::vector<SurveyClass> classes;
    // the same for the analytic Jacobian kernel (larger per-spaxel records)
    std::vector<int32_t> torder;
    std::vector<SurveyClass> tclasses;
    bool tangent_ok = true;         // every galaxy fits the Jacobian kernel
    size_t table_bytes = 0;         // device tables at the start of the workspace
    // device copies (inside the workspace) after survey_upload
    Geom *d_geo = nullptr;
    int64_t *d_pix_off = nullptr;
    int32_t *d_order = nullptr;
    int32_t *d_torder = nullptr;
    int *d_work = nullptr;          // work counters of persistent launches
    std::vector<char> h_tables;     // host image of the device tables (built once)
    SurveyTuning tuning = {0, 0, 0};
    int64_t total_pix() const { return pix_off.empty() ? 0 : pix_off.back(); }
};

// `force` (optional) overrides the cached or default survey tuning.
gbk_status survey_plan(const gbk_geom *geoms, int n_gal, SurveyPlan *sp, const SurveyTuning *force = nullptr);
// survey_plan through a small cache of recent plans (same geometry bytes,
// same survey tunings): repeated calls over one survey skip the planning.
gbk_status survey_plan_cached(const gbk_geom *geoms, int n_gal, SurveyPlan *sp);
gbk_status survey_upload(SurveyPlan *sp, char *ws, cudaStream_t st);
// A plan's launches restricted to some of its galaxies (a batched fit's
// running ones): the classes' ranges index a compacted copy of the order
// (the device copy is the caller's).
struct SurveyLive {
    std::vector<SurveyClass> classes;
    std::vector<int32_t> rep;  // per class: the galaxy whose geometry the full plan's launch carries
    const int32_t *d_order = nullptr;
};
// Fills live->classes and the compacted order (host) for the galaxies with
// active[g] != 0; the caller uploads the order and sets live->d_order.
void survey_live(const SurveyPlan &sp, const std::vector<char> &active, SurveyLive *live,
                 std::vector<int32_t> *order);
// Models gal * mpg + s (s < mpg) of every galaxy (or of the galaxies of
// `live`): chi2 [n_gal * mpg] and the packed maps / residuals (galaxy gal at
// pixel offset pix_off[gal] * mpg).
gbk_status survey_eval(const SurveyPlan &sp, int mpg, const double *params, const gbk_obs *obs_list,
                       const int32_t *skip, float *maps, double *chi2, float *resid, cudaStream_t st,
                       const SurveyLive *live = nullptr);
struct TangentArgs;
// J^T J, J^T r and chi2 of one model per galaxy (the analytic Jacobian):
// `proto` supplies params, obs_list, skip, the free parameters and outputs.
gbk_status survey_tangent(const SurveyPlan &sp, const TangentArgs &proto, cudaStream_t st);

}  // namespace gbk
