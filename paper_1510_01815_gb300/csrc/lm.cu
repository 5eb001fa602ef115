// lm.cu -- gbk_fit_lm: Levenberg-Marquardt over the fused forward model
// (Sec. 2.3.1 of Bekiaris et al. 2015).
//
// Batched mode: every galaxy advances together.  One iteration is
//   Jacobian -> FP64 normal equations -> damped Cholesky solve -> fused
//   evaluation of the trial points -> accept/reject,
// where the Jacobian is either a finite-difference batch (evaluation of chi2
// and residual maps of 1 + P or 1 + 2P models per galaxy, then a reduction
// kernel) or the analytic tangent kernels, which reduce J^T J and J^T r
// directly;
// all on the device; it is captured once in a CUDA graph and replayed, and
// the host reads the number of running galaxies every kPoll iterations.  The
// evaluations and the analytic Jacobian take the two-stage (split) kernels
// where they serve the geometry and the caller's path allows, else the
// one-cluster-per-model kernels; chi2 values that accept/reject compares
// always come from one evaluator.
//
// Plain mode: the paper's arrangement -- one galaxy at a time, the model
// evaluations on the GPU, the residual maps copied to the host every
// iteration, the normal equations and the solve on the CPU in FP64.
#include <cmath>
#include <algorithm>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "gbk_api_internal.h"
#include "k_fused.h"
#include "k_lm.h"
#include "k_split.h"
#include "k_tangent.h"
#include "k_tsplit.h"
#include "survey.h"

namespace gbk {

constexpr int kPoll = 8;
constexpr int kCompactMin = 32;  // smallest batch of one geometry that is compacted

static size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

struct LmPlan {
    int np, m, central, tangent, idx[GBK_NPAR];
};

static gbk_status lm_plan(const gbk_lm_opts *o, LmPlan *pl)
{
    if (!o) return fail(GBK_EINVAL, "opts is NULL");
    if (o->max_iter < 1 || o->max_iter > 100000) return fail(GBK_EINVAL, "max_iter must be in 1..100000");
    if (o->mode != GBK_LM_BATCHED && o->mode != GBK_LM_PLAIN) return fail(GBK_EINVAL, "unknown LM mode %d", o->mode);
    if (o->jacobian != GBK_JAC_FD_FORWARD && o->jacobian != GBK_JAC_FD_CENTRAL && o->jacobian != GBK_JAC_TANGENT)
        return fail(GBK_EINVAL, "unknown Jacobian kind %d", o->jacobian);
    if (!(o->ftol >= 0.0) || !(o->xtol >= 0.0) || !(o->lambda0 > 0.0))
        return fail(GBK_EINVAL, "ftol, xtol must be >= 0 and lambda0 > 0");
    int np = 0;
    for (int k = 0; k < GBK_NPAR; ++k)
        if (o->free_mask & (1u << k)) {
            if (!(o->fd_step[k] > 0.0) || !std::isfinite(o->fd_step[k]))
                return fail(GBK_EINVAL, "fd_step[%d] must be finite and > 0", k);
            pl->idx[np++] = k;
        }
    if (np == 0) return fail(GBK_EINVAL, "free_mask selects no parameter");
    if (o->free_mask >> GBK_NPAR) return fail(GBK_EINVAL, "free_mask has bits beyond the %d parameters", GBK_NPAR);
    pl->np = np;
    pl->central = o->jacobian == GBK_JAC_FD_CENTRAL;
    pl->tangent = o->jacobian == GBK_JAC_TANGENT;
    pl->m = pl->tangent ? 1 : 1 + (pl->central ? 2 : 1) * np;
    if (pl->tangent && o->mode == GBK_LM_PLAIN)
        return fail(GBK_EINVAL, "the plain mode uses finite differences (the paper's arrangement)");
    return GBK_OK;
}

// Workspace layout; `ng` galaxies share one batch at a time (n_gal in the
// batched mode, 1 in the plain mode).
struct LmLayout {
    size_t pbatch, resid, chi2b, hstep, jtj, jtr, ptrial, chi2t, chi2cur, chi2best, lambda, dnorm, pnorm, pred, nu;
    size_t iters, status, done, jskip, nact, sws, sws_bytes, total;
    // tail compaction (one geometry): two sets of the moved per-galaxy
    // inputs, the running slots, and the moved state
    size_t cpar[2], clo[2], chi[2], cobs[2], cmap[2], clive, nlam, nnu, ncc, nit;
};

// pix_total: pixels of all ng galaxies together; split_bytes: the region the
// split evaluator and Jacobian share (they run one after the other).
static LmLayout lm_layout_pix(size_t pix_total, int ng, const LmPlan &pl, size_t split_bytes = 0)
{
    LmLayout L;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o += al256(bytes); return r; };
    L.pbatch = take(sizeof(double) * ng * pl.m * GBK_NPAR);
    L.resid = take(sizeof(float) * pl.m * 2 * pix_total);
    L.chi2b = take(sizeof(double) * ng * pl.m);
    L.hstep = take(sizeof(double) * ng * pl.np);
    L.jtj = take(sizeof(double) * ng * pl.np * pl.np);
    L.jtr = take(sizeof(double) * ng * pl.np);
    L.ptrial = take(sizeof(double) * ng * GBK_NPAR);
    L.chi2t = take(sizeof(double) * ng);
    L.chi2cur = take(sizeof(double) * ng);
    L.chi2best = take(sizeof(double) * ng);
    L.lambda = take(sizeof(double) * ng);
    L.dnorm = take(sizeof(double) * ng);
    L.pnorm = take(sizeof(double) * ng);
    L.pred = take(sizeof(double) * ng);
    L.nu = take(sizeof(double) * ng);
    L.iters = take(sizeof(int32_t) * ng);
    L.status = take(sizeof(int32_t) * ng);
    L.done = take(sizeof(int32_t) * ng);
    L.jskip = take(sizeof(int32_t) * ng);
    L.nact = take(sizeof(int32_t));
    for (int b = 0; b < 2; ++b) {
        L.cpar[b] = take(sizeof(double) * ng * GBK_NPAR);
        L.clo[b] = take(sizeof(double) * ng * GBK_NPAR);
        L.chi[b] = take(sizeof(double) * ng * GBK_NPAR);
        L.cobs[b] = take(sizeof(gbk_obs) * ng);
        L.cmap[b] = take(sizeof(int32_t) * ng);
    }
    L.clive = take(sizeof(int32_t) * ng);
    L.nlam = take(sizeof(double) * ng);
    L.nnu = take(sizeof(double) * ng);
    L.ncc = take(sizeof(double) * ng);
    L.nit = take(sizeof(int32_t) * ng);
    L.sws = take(split_bytes);
    L.sws_bytes = split_bytes;
    L.total = o;
    return L;
}

static LmLayout lm_layout(const Geom &g, int ng, const LmPlan &pl, size_t split_bytes = 0)
{
    return lm_layout_pix((size_t)ng * g.nx * g.ny, ng, pl, split_bytes);
}

// Which split kernels a batched fit of ng galaxies of one geometry uses
// (path: GBK_PATH_AUTO = where they serve, GBK_PATH_SPLIT = required,
// GBK_PATH_FUSED = never) and the workspace they share.
struct LmSplit {
    bool eval, jac;
    size_t bytes;
};

static gbk_status lm_split_plan(const Geom &g, int ng, const LmPlan &pl, int32_t path, LmSplit *sp)
{
    *sp = LmSplit{false, false, 0};
    if (path == (int32_t)GBK_PATH_FUSED) return GBK_OK;
    if (path != (int32_t)GBK_PATH_AUTO && path != (int32_t)GBK_PATH_SPLIT)
        return fail(GBK_EINVAL, "LM evaluates on GBK_PATH_AUTO, GBK_PATH_FUSED or GBK_PATH_SPLIT (got %d)", path);
    sp->eval = split_supported(g);
    sp->jac = pl.tangent && tsplit_supported(g, pl.np, pl.idx);
    if (path == (int32_t)GBK_PATH_SPLIT && (!sp->eval || (pl.tangent && !sp->jac)))
        return fail(GBK_EUNSUPPORTED, "the split kernels do not serve this geometry and free-parameter set");
    if (sp->eval) sp->bytes = split_workspace_bytes(g, ng * pl.m);
    if (sp->jac) sp->bytes = std::max(sp->bytes, tsplit_workspace_bytes(g, ng));
    return GBK_OK;
}

static gbk_status fused_for(const Geom &g, int n_models, const double *params, const gbk_obs *obs_list,
                            const gbk_obs *obs_one, int mpg, const int32_t *skip, double *chi2, float *resid,
                            cudaStream_t st)
{
    FusedConfig fc;
    if (!fused_config(g, &fc)) return fail(GBK_EUNSUPPORTED, "the fused path cannot serve this geometry");
    FusedArgs a = {};
    a.g = g;
    a.n_models = n_models;
    a.params = params;
    if (obs_one) a.obs = *obs_one;
    a.obs_list = obs_list;
    a.models_per_gal = mpg;
    a.skip = skip;
    a.chi2 = chi2;
    a.resid = resid;
    a.cs = fc.cs;
    a.band = fc.band;
    a.threads = fc.threads;
    a.persistent = fc.persistent;
    return launch_fused(a, st);
}

// What the batched LM evaluates: one geometry for every galaxy, or a ragged
// survey plan; for one geometry, whether the split evaluator and Jacobian
// serve it, and their workspace.
struct EvalTarget {
    const Geom *g;
    const SurveyPlan *sp;
    LmSplit split;
    void *sws;
    const TsRaggedPlan *rag = nullptr;  // survey: the ragged split Jacobian's plan (its region at sws)
    const SurveyLive *live = nullptr;   // survey: the evaluator's launches over the running galaxies
};

static gbk_status eval_for(const EvalTarget &t, int n_gal, int mpg, const double *params, const gbk_obs *obs_list,
                           const int32_t *skip, double *chi2, float *resid, cudaStream_t st)
{
    if (t.sp) return survey_eval(*t.sp, mpg, params, obs_list, skip, nullptr, chi2, resid, st, t.live);
    if (t.split.eval) {
        const SplitBatch b = {obs_list, skip, mpg};
        return launch_split(*t.g, n_gal * mpg, params, nullptr, nullptr, chi2, resid, t.sws, t.split.bytes, st,
                            nullptr, &b);
    }
    return fused_for(*t.g, n_gal * mpg, params, obs_list, nullptr, mpg, skip, chi2, resid, st);
}

// ----------------------------------------------------------------------------
// Host FP64 linear algebra of the plain mode (same damping rule as the device).
static bool host_solve(const std::vector<double> &JTJ, const std::vector<double> &JTr, int np, double &lam,
                       std::vector<double> &d)
{
    std::vector<double> L((size_t)np * np);
    bool ok = false;
    for (int attempt = 0; attempt < 12 && !ok; ++attempt) {
        ok = true;
        for (int j = 0; j < np && ok; ++j)
            for (int k = 0; k <= j; ++k) {
                double v = JTJ[j * np + k];
                if (j == k) v += lam * (JTJ[j * np + j] > 0.0 ? JTJ[j * np + j] : 1.0);
                for (int q = 0; q < k; ++q) v -= L[j * np + q] * L[k * np + q];
                if (j == k) {
                    if (!(v > 0.0)) { ok = false; break; }
                    L[j * np + j] = std::sqrt(v);
                } else {
                    L[j * np + k] = v / L[k * np + k];
                }
            }
        if (!ok) lam *= 10.0;
    }
    if (!ok) return false;
    std::vector<double> y(np);
    d.assign(np, 0.0);
    for (int j = 0; j < np; ++j) {
        double v = -JTr[j];
        for (int q = 0; q < j; ++q) v -= L[j * np + q] * y[q];
        y[j] = v / L[j * np + j];
    }
    for (int j = np - 1; j >= 0; --j) {
        double v = y[j];
        for (int q = j + 1; q < np; ++q) v -= L[q * np + j] * d[q];
        d[j] = v / L[j * np + j];
    }
    return true;
}

struct CudaGuard {
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    ~CudaGuard()
    {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (s) cudaStreamDestroy(s);
    }
};

static gbk_status lm_plain(const Geom &g, int n_gal, const gbk_obs *obs, const double *lo, const double *hi,
                           double *params, const gbk_lm_opts *o, const LmPlan &pl, double *chi2_out,
                           int32_t *iters_out, int32_t *status_out, char *ws, cudaStream_t st)
{
    LmLayout L = lm_layout(g, 1, pl);
    const size_t npix = (size_t)g.nx * g.ny, n2 = 2 * npix;
    const int np = pl.np, m = pl.m;
    std::vector<gbk_obs> h_obs(n_gal);
    std::vector<double> h_lo((size_t)n_gal * GBK_NPAR), h_hi(h_lo.size()), h_p(h_lo.size());
    std::vector<double> h_chi2(n_gal);
    std::vector<int32_t> h_it(n_gal), h_st(n_gal);
    cudaError_t e;
    if ((e = cudaMemcpyAsync(h_obs.data(), obs, sizeof(gbk_obs) * n_gal, cudaMemcpyDeviceToHost, st)) ||
        (e = cudaMemcpyAsync(h_lo.data(), lo, sizeof(double) * h_lo.size(), cudaMemcpyDeviceToHost, st)) ||
        (e = cudaMemcpyAsync(h_hi.data(), hi, sizeof(double) * h_hi.size(), cudaMemcpyDeviceToHost, st)) ||
        (e = cudaMemcpyAsync(h_p.data(), params, sizeof(double) * h_p.size(), cudaMemcpyDeviceToHost, st)) ||
        (e = cudaStreamSynchronize(st)))
        return cuda_fail(e, "plain LM: reading inputs");
    double *d_pb = (double *)(ws + L.pbatch), *d_chi2b = (double *)(ws + L.chi2b);
    float *d_res = (float *)(ws + L.resid);
    double *d_pt = (double *)(ws + L.ptrial), *d_ct = (double *)(ws + L.chi2t);
    std::vector<double> pb((size_t)m * GBK_NPAR), chi2b(m), hs(np), JTJ((size_t)np * np), JTr(np), dlt;
    std::vector<float> res((size_t)m * n2);
    for (int gal = 0; gal < n_gal; ++gal) {
        double *p = &h_p[(size_t)gal * GBK_NPAR];
        const double *plo = &h_lo[(size_t)gal * GBK_NPAR], *phi = &h_hi[(size_t)gal * GBK_NPAR];
        double lam = o->lambda0, nu = 2.0, best = NAN, cc = NAN;
        int it = 0, status = GBK_FIT_RUNNING;
        bool fresh = false;  // J^T J, J^T r and cc belong to p (kept after a rejected step)
        while (status == GBK_FIT_RUNNING) {
            if (!fresh) {
                // Jacobian batch
                for (int s = 0; s < m; ++s) std::memcpy(&pb[(size_t)s * GBK_NPAR], p, sizeof(double) * GBK_NPAR);
                for (int j = 0; j < np; ++j) {
                    int k = pl.idx[j];
                    double h = o->fd_step[k];
                    if (pl.central) {
                        pb[(size_t)(1 + j) * GBK_NPAR + k] = p[k] + h;
                        pb[(size_t)(1 + np + j) * GBK_NPAR + k] = p[k] - h;
                        hs[j] = 2.0 * h;
                    } else {
                        if (p[k] + h > phi[k] && p[k] - h >= plo[k]) h = -h;
                        pb[(size_t)(1 + j) * GBK_NPAR + k] = p[k] + h;
                        hs[j] = h;
                    }
                }
                if ((e = cudaMemcpyAsync(d_pb, pb.data(), sizeof(double) * pb.size(), cudaMemcpyHostToDevice, st)))
                    return cuda_fail(e, "plain LM: batch upload");
                gbk_status sb = fused_for(g, m, d_pb, nullptr, &h_obs[gal], m, nullptr, d_chi2b, d_res, st);
                if (sb) return sb;
                if ((e = cudaMemcpyAsync(res.data(), d_res, sizeof(float) * res.size(), cudaMemcpyDeviceToHost, st)) ||
                    (e = cudaMemcpyAsync(chi2b.data(), d_chi2b, sizeof(double) * m, cudaMemcpyDeviceToHost, st)) ||
                    (e = cudaStreamSynchronize(st)))
                    return cuda_fail(e, "plain LM: residual download");
                cc = chi2b[0];
                if (!std::isfinite(cc)) { ++it; status = GBK_FIT_NONFINITE; break; }
                std::fill(JTJ.begin(), JTJ.end(), 0.0);
                std::fill(JTr.begin(), JTr.end(), 0.0);
                std::vector<double> J(np);
                for (size_t i = 0; i < n2; ++i) {
                    double r0 = res[i];
                    for (int j = 0; j < np; ++j) {
                        double rm = pl.central ? res[(size_t)(1 + np + j) * n2 + i] : r0;
                        J[j] = ((double)res[(size_t)(1 + j) * n2 + i] - rm) / hs[j];
                    }
                    for (int j = 0; j < np; ++j) {
                        JTr[j] += J[j] * r0;
                        for (int k = 0; k <= j; ++k) JTJ[j * np + k] += J[j] * J[k];
                    }
                }
                for (int j = 0; j < np; ++j)
                    for (int k = 0; k < j; ++k) JTJ[k * np + j] = JTJ[j * np + k];
                fresh = true;
            }
            ++it;
            // damped solve and trial point
            std::vector<double> pt(p, p + GBK_NPAR);
            double dn = 0.0, pn = 0.0;
            bool solved = host_solve(JTJ, JTr, np, lam, dlt);
            if (solved)
                for (int j = 0; j < np; ++j) {
                    int k = pl.idx[j];
                    double v = std::fmin(std::fmax(p[k] + dlt[j], plo[k]), phi[k]);
                    dn += (v - p[k]) * (v - p[k]);
                    pn += p[k] * p[k];
                    pt[k] = v;
                }
            double ct = NAN;
            if (solved && dn > 0.0) {
                if ((e = cudaMemcpyAsync(d_pt, pt.data(), sizeof(double) * GBK_NPAR, cudaMemcpyHostToDevice, st)))
                    return cuda_fail(e, "plain LM: trial upload");
                gbk_status s = fused_for(g, 1, d_pt, nullptr, &h_obs[gal], 1, nullptr, d_ct, nullptr, st);
                if (s) return s;
                if ((e = cudaMemcpyAsync(&ct, d_ct, sizeof(double), cudaMemcpyDeviceToHost, st)) ||
                    (e = cudaStreamSynchronize(st)))
                    return cuda_fail(e, "plain LM: trial download");
            }
            if (std::isfinite(ct) && ct <= cc && dn > 0.0) {
                // gain ratio against the linearised model's decrease
                // -(2 s.J^T r + s.J^T J s) of the clipped step s
                double sg = 0.0, sas = 0.0;
                for (int j = 0; j < np; ++j) {
                    const double sj = pt[pl.idx[j]] - p[pl.idx[j]];
                    double as = 0.0;
                    for (int k = 0; k < np; ++k) as += JTJ[j * np + k] * (pt[pl.idx[k]] - p[pl.idx[k]]);
                    sg += sj * JTr[j];
                    sas += sj * as;
                }
                const double pred = -(2.0 * sg + sas);
                const double rho = pred > 0.0 ? (cc - ct) / pred : 0.0;
                const double q = 2.0 * rho - 1.0;
                lam = std::fmax(lam * std::fmax(0.1, 1.0 - q * q * q), 1e-12);
                nu = 2.0;
                std::memcpy(p, pt.data(), sizeof(double) * GBK_NPAR);
                best = ct;
                fresh = false;
                double rel = (cc - ct) / std::fmax(cc, 1e-300);
                if (rel < o->ftol) status = GBK_FIT_FTOL;
                else if (std::sqrt(dn) <= o->xtol * (std::sqrt(pn) + o->xtol)) status = GBK_FIT_XTOL;
            } else {
                best = cc;
                lam *= nu;
                nu *= 2.0;
                if (lam > 1e12) status = GBK_FIT_LAMBDA;
            }
            if (status == GBK_FIT_RUNNING && it >= o->max_iter) status = GBK_FIT_MAXITER;
        }
        h_chi2[gal] = best;
        h_it[gal] = it;
        h_st[gal] = status;
    }
    if ((e = cudaMemcpyAsync(params, h_p.data(), sizeof(double) * h_p.size(), cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(chi2_out, h_chi2.data(), sizeof(double) * n_gal, cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(iters_out, h_it.data(), sizeof(int32_t) * n_gal, cudaMemcpyHostToDevice, st)) ||
        (e = cudaMemcpyAsync(status_out, h_st.data(), sizeof(int32_t) * n_gal, cudaMemcpyHostToDevice, st)) ||
        (e = cudaStreamSynchronize(st)))
        return cuda_fail(e, "plain LM: writing results");
    return ok();
}

static gbk_status lm_iteration(const EvalTarget &t, const LmArgs &a, const gbk_obs *obs, bool tangent,
                               const TangentArgs &ta, const TsplitCall &tc, const TsplitRaggedCall &rc,
                               cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(a.n_active, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return cuda_fail(e, "LM: clearing the running count");
    gbk_status s;
    if (tangent) {
        // analytic J^T J and J^T r at the current point
        if (t.sp && t.rag) s = launch_tsplit_ragged(*t.rag, rc, (char *)t.sws, st);
        else if (t.sp) s = survey_tangent(*t.sp, ta, st);
        else if (t.split.jac) s = launch_tsplit(tc, t.sws, t.split.bytes, st);
        else s = launch_tangent(ta, st);
        if (s) return s;
    } else {
        lm_launch_build_fd(a, st);
        s = eval_for(t, a.n_gal, a.m, a.pbatch, obs, a.jskip, a.chi2_batch, a.resid, st);
        if (s) return s;
        lm_launch_normal_fd(a, st);
    }
    lm_launch_solve(a, st);
    s = eval_for(t, a.n_gal, 1, a.ptrial, obs, a.done, a.chi2_trial, nullptr, st);
    if (s) return s;
    lm_launch_accept(a, st);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "LM iteration launch");
    return GBK_OK;
}

static gbk_status lm_batched(const EvalTarget &t, int n_gal, const gbk_obs *obs, const double *lo, const double *hi,
                             double *params, const gbk_lm_opts *o, const LmPlan &pl, double *chi2_out,
                             int32_t *iters_out, int32_t *status_out, char *ws, cudaStream_t user)
{
    LmLayout L = t.sp ? lm_layout_pix((size_t)t.sp->total_pix(), n_gal, pl, t.split.bytes)
                      : lm_layout(*t.g, n_gal, pl, t.split.bytes);
    LmArgs a = {};
    a.n_gal = n_gal;
    a.np = pl.np;
    for (int j = 0; j < pl.np; ++j) a.free_idx[j] = pl.idx[j];
    for (int k = 0; k < GBK_NPAR; ++k) a.fd_step[k] = o->fd_step[k];
    a.m = pl.m;
    a.central = pl.central;
    a.np_pix = t.sp ? 0 : t.g->nx * t.g->ny;
    a.pix_off = t.sp ? t.sp->d_pix_off : nullptr;
    a.max_iter = o->max_iter;
    a.ftol = o->ftol;
    a.xtol = o->xtol;
    a.lo = lo;
    a.hi = hi;
    a.params = params;
    a.pbatch = (double *)(ws + L.pbatch);
    a.resid = (float *)(ws + L.resid);
    a.chi2_batch = (double *)(ws + L.chi2b);
    a.hstep = (double *)(ws + L.hstep);
    a.jtj = (double *)(ws + L.jtj);
    a.jtr = (double *)(ws + L.jtr);
    a.ptrial = (double *)(ws + L.ptrial);
    a.chi2_trial = (double *)(ws + L.chi2t);
    a.chi2_cur = (double *)(ws + L.chi2cur);
    a.chi2_best = (double *)(ws + L.chi2best);
    a.lambda = (double *)(ws + L.lambda);
    a.dnorm = (double *)(ws + L.dnorm);
    a.pnorm = (double *)(ws + L.pnorm);
    a.pred = (double *)(ws + L.pred);
    a.nu = (double *)(ws + L.nu);
    a.iters = (int32_t *)(ws + L.iters);
    a.status = (int32_t *)(ws + L.status);
    a.done = (int32_t *)(ws + L.done);
    a.jskip = (int32_t *)(ws + L.jskip);
    a.n_active = (int32_t *)(ws + L.nact);

    CudaGuard cg;
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&cg.s, cudaStreamNonBlocking)) ||
        (e = cudaEventCreateWithFlags(&cg.e0, cudaEventDisableTiming)) ||
        (e = cudaEventCreateWithFlags(&cg.e1, cudaEventDisableTiming)) || (e = cudaEventRecord(cg.e0, user)) ||
        (e = cudaStreamWaitEvent(cg.s, cg.e0, 0)))
        return cuda_fail(e, "LM: stream set-up");
    cudaStream_t st = cg.s;
    lm_launch_init(a, o->lambda0, st);
    TangentArgs ta = {};
    TsplitCall tc = {};
    TsplitRaggedCall rc = {};
    if (pl.tangent && t.sp && t.rag) {
        rc.d_geo = t.sp->d_geo;
        rc.params = params;
        rc.obs_list = obs;
        rc.skip = a.jskip;
        rc.np = pl.np;
        for (int j = 0; j < pl.np; ++j) rc.free_idx[j] = pl.idx[j];
        rc.jtj = a.jtj;
        rc.jtv = a.jtr;
        gbk_status s0 = eval_for(t, n_gal, 1, params, obs, nullptr, a.chi2_cur, nullptr, st);
        if (s0) return s0;
    } else if (pl.tangent && !t.sp && t.split.jac) {
        tc.g = *t.g;
        tc.n_models = n_gal;
        tc.params = params;
        tc.obs_list = obs;
        tc.skip = a.jskip;
        tc.np = pl.np;
        for (int j = 0; j < pl.np; ++j) tc.free_idx[j] = pl.idx[j];
        tc.jtj = a.jtj;
        tc.jtv = a.jtr;
        gbk_status s0 = eval_for(t, n_gal, 1, params, obs, nullptr, a.chi2_cur, nullptr, st);
        if (s0) return s0;
    } else if (pl.tangent) {
        ta.np = pl.np;
        for (int j = 0; j < pl.np; ++j) ta.free_idx[j] = pl.idx[j];
        if (t.sp) {
            if (!t.sp->tangent_ok || !tangent_narrow(ta))
                return fail(GBK_EUNSUPPORTED, "a galaxy of the batch is too large for the Jacobian kernel");
        } else {
            const Geom &g = *t.g;
            if (g.model == GBK_MODEL_CUBE && !tangent_config(g, &ta.cs, &ta.band, &ta.direct, tangent_narrow(ta)))
                return fail(GBK_EUNSUPPORTED, "geometry too large for the tangent Jacobian kernel");
            ta.g = g;
        }
        ta.n_models = n_gal;
        ta.params = params;
        ta.obs_list = obs;
        ta.models_per_gal = 1;
        ta.skip = a.jskip;
        ta.jtj = a.jtj;
        ta.jtv = a.jtr;
        // chi2 at the start point from the evaluator: accept/reject
        // decisions always compare that evaluator's chi2 values
        gbk_status s0 = eval_for(t, n_gal, 1, params, obs, nullptr, a.chi2_cur, nullptr, st);
        if (s0) return s0;
    }
    // The first iteration runs eagerly (it also settles the kernels' launch
    // configurations); the rest replay a captured graph.
    gbk_status s = lm_iteration(t, a, obs, pl.tangent, ta, tc, rc, st);
    if (s) return s;
    int32_t h_active = n_gal;
    int done_iters = 1;
    int planned = n_gal;   // galaxies of the current ragged Jacobian plan
    TsRaggedPlan live;     // its re-plan over the running galaxies
    SurveyLive slive;      // the survey evaluator's launches over them
    std::vector<int32_t> h_sorder;
    // one geometry: galaxies in slots 0 .. n_cur; after a compaction the
    // inputs live in the workspace and cmap gives each slot's caller index
    int n_cur = n_gal, flip = 0;
    bool compacted = false;
    const gbk_obs *obs_cur = obs;
    std::vector<int32_t> h_flags, h_live;
    if (o->max_iter > 1) {
        if ((e = cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed)))
            return cuda_fail(e, "LM: begin graph capture");
        s = lm_iteration(t, a, obs, pl.tangent, ta, tc, rc, st);
        e = cudaStreamEndCapture(st, &cg.graph);
        if (s) return s;
        if (e != cudaSuccess) return cuda_fail(e, "LM: end graph capture");
        if ((e = cudaGraphInstantiate(&cg.exec, cg.graph, 0))) return cuda_fail(e, "LM: graph instantiation");
        while (done_iters < o->max_iter) {
            int burst = kPoll;
            if (done_iters + burst > o->max_iter) burst = o->max_iter - done_iters;
            for (int b = 0; b < burst; ++b)
                if ((e = cudaGraphLaunch(cg.exec, st))) return cuda_fail(e, "LM: graph launch");
            done_iters += burst;
            if ((e = cudaMemcpyAsync(&h_active, a.n_active, sizeof(int32_t), cudaMemcpyDeviceToHost, st)) ||
                (e = cudaStreamSynchronize(st)))
                return cuda_fail(e, "LM: polling");
            if (h_active == 0) break;
            if (!t.sp && h_active * 4 <= n_cur && n_cur >= kCompactMin) {
                // Finished galaxies' CTAs only return at their skip test, but
                // at thousands per launch those returns cost most of a tail
                // iteration: move the running galaxies to the front of fresh
                // buffers and capture the iteration again for them alone.
                h_flags.resize(n_cur);
                if ((e = cudaMemcpyAsync(h_flags.data(), a.done, sizeof(int32_t) * n_cur, cudaMemcpyDeviceToHost,
                                         st)) ||
                    (e = cudaStreamSynchronize(st)))
                    return cuda_fail(e, "LM: reading the running galaxies");
                h_live.clear();
                for (int i = 0; i < n_cur; ++i)
                    if (h_flags[i] == 0) h_live.push_back(i);
                const int n_live = (int)h_live.size();
                const int nb = flip ^ 1;
                int32_t *d_live = (int32_t *)(ws + L.clive);
                if ((e = cudaMemcpyAsync(d_live, h_live.data(), sizeof(int32_t) * n_live, cudaMemcpyHostToDevice,
                                         st)))
                    return cuda_fail(e, "LM: uploading the running galaxies");
                const int32_t *map = compacted ? (const int32_t *)(ws + L.cmap[flip]) : nullptr;
                LmScatterArgs sc = {n_cur, map, a.params, a.chi2_best, a.iters, a.status,
                                    compacted ? params : nullptr, chi2_out, iters_out, status_out};
                lm_launch_scatter(sc, st);
                LmCompactArgs cp = {};
                cp.n_live = n_live;
                cp.live = d_live;
                cp.map = map;
                cp.params = a.params;
                cp.lo = a.lo;
                cp.hi = a.hi;
                cp.obs = obs_cur;
                cp.lambda = a.lambda;
                cp.nu = a.nu;
                cp.chi2_cur = a.chi2_cur;
                cp.iters = a.iters;
                cp.params_n = (double *)(ws + L.cpar[nb]);
                cp.lo_n = (double *)(ws + L.clo[nb]);
                cp.hi_n = (double *)(ws + L.chi[nb]);
                cp.obs_n = (gbk_obs *)(ws + L.cobs[nb]);
                cp.map_n = (int32_t *)(ws + L.cmap[nb]);
                cp.lambda_n = (double *)(ws + L.nlam);
                cp.nu_n = (double *)(ws + L.nnu);
                cp.chi2_cur_n = (double *)(ws + L.ncc);
                cp.iters_n = (int32_t *)(ws + L.nit);
                lm_launch_compact(cp, st);
                if ((e = cudaMemcpyAsync(a.lambda, cp.lambda_n, sizeof(double) * n_live, cudaMemcpyDeviceToDevice, st)) ||
                    (e = cudaMemcpyAsync(a.nu, cp.nu_n, sizeof(double) * n_live, cudaMemcpyDeviceToDevice, st)) ||
                    (e = cudaMemcpyAsync(a.chi2_cur, cp.chi2_cur_n, sizeof(double) * n_live, cudaMemcpyDeviceToDevice,
                                         st)) ||
                    (e = cudaMemcpyAsync(a.iters, cp.iters_n, sizeof(int32_t) * n_live, cudaMemcpyDeviceToDevice, st)) ||
                    (e = cudaMemsetAsync(a.status, 0, sizeof(int32_t) * n_live, st)) ||  // GBK_FIT_RUNNING
                    (e = cudaMemsetAsync(a.done, 0, sizeof(int32_t) * n_live, st)) ||
                    (e = cudaMemsetAsync(a.jskip, 0, sizeof(int32_t) * n_live, st)) ||
                    (e = cudaGetLastError()))
                    return cuda_fail(e, "LM: compacting the running galaxies");
                a.n_gal = n_live;
                a.params = cp.params_n;
                a.lo = cp.lo_n;
                a.hi = cp.hi_n;
                obs_cur = cp.obs_n;
                tc.n_models = n_live;
                tc.params = cp.params_n;
                tc.obs_list = cp.obs_n;
                ta.n_models = n_live;
                ta.params = cp.params_n;
                ta.obs_list = cp.obs_n;
                n_cur = n_live;
                flip = nb;
                compacted = true;
                cudaGraphExecDestroy(cg.exec);
                cudaGraphDestroy(cg.graph);
                cg.exec = nullptr;
                cg.graph = nullptr;
                if ((e = cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed)))
                    return cuda_fail(e, "LM: begin graph capture");
                s = lm_iteration(t, a, obs_cur, pl.tangent, ta, tc, rc, st);
                e = cudaStreamEndCapture(st, &cg.graph);
                if (s) return s;
                if (e != cudaSuccess) return cuda_fail(e, "LM: end graph capture");
                if ((e = cudaGraphInstantiate(&cg.exec, cg.graph, 0))) return cuda_fail(e, "LM: graph instantiation");
            }
            if (t.sp && h_active * 4 <= planned && planned > 16) {
                // Survey: the finished galaxies' CTAs (ragged split Jacobian)
                // and work items (evaluator) would only return at their skip
                // test, so once a quarter of the planned galaxies are still
                // running, plan the running ones alone and capture the
                // iteration again.
                std::vector<int32_t> h_done(n_gal);
                if ((e = cudaMemcpyAsync(h_done.data(), a.done, sizeof(int32_t) * n_gal, cudaMemcpyDeviceToHost,
                                         st)) ||
                    (e = cudaStreamSynchronize(st)))
                    return cuda_fail(e, "LM: reading the running galaxies");
                std::vector<char> act(n_gal);
                for (int i = 0; i < n_gal; ++i) act[i] = h_done[i] == 0;
                EvalTarget t2 = t;
                if (t.rag) {
                    tsplit_ragged_plan(t.sp->geo, &live, &act);
                    if (!live.ok || live.total > t.split.bytes)
                        return fail(GBK_EINVAL, "LM: re-planning the survey Jacobian");
                    if ((s = tsplit_ragged_upload(live, (char *)t.sws, st))) return s;
                    t2.rag = &live;
                }
                survey_live(*t.sp, act, &slive, &h_sorder);
                int32_t *d_sorder = (int32_t *)(ws + L.clive);
                if (!h_sorder.empty() &&
                    (e = cudaMemcpyAsync(d_sorder, h_sorder.data(), sizeof(int32_t) * h_sorder.size(),
                                         cudaMemcpyHostToDevice, st)))
                    return cuda_fail(e, "LM: uploading the running galaxies' order");
                slive.d_order = d_sorder;
                t2.live = &slive;
                planned = h_active;
                cudaGraphExecDestroy(cg.exec);
                cudaGraphDestroy(cg.graph);
                cg.exec = nullptr;
                cg.graph = nullptr;
                if ((e = cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed)))
                    return cuda_fail(e, "LM: begin graph capture");
                s = lm_iteration(t2, a, obs, pl.tangent, ta, tc, rc, st);
                e = cudaStreamEndCapture(st, &cg.graph);
                if (s) return s;
                if (e != cudaSuccess) return cuda_fail(e, "LM: end graph capture");
                if ((e = cudaGraphInstantiate(&cg.exec, cg.graph, 0))) return cuda_fail(e, "LM: graph instantiation");
            }
        }
    }
    if (compacted) {
        LmScatterArgs sc = {n_cur, (const int32_t *)(ws + L.cmap[flip]), a.params, a.chi2_best, a.iters, a.status,
                            params, chi2_out, iters_out, status_out};
        lm_launch_scatter(sc, st);
        if ((e = cudaGetLastError())) return cuda_fail(e, "LM: results");
    } else if ((e = cudaMemcpyAsync(chi2_out, a.chi2_best, sizeof(double) * n_gal, cudaMemcpyDeviceToDevice, st)) ||
               (e = cudaMemcpyAsync(iters_out, a.iters, sizeof(int32_t) * n_gal, cudaMemcpyDeviceToDevice, st)) ||
               (e = cudaMemcpyAsync(status_out, a.status, sizeof(int32_t) * n_gal, cudaMemcpyDeviceToDevice, st))) {
        return cuda_fail(e, "LM: results");
    }
    if ((e = cudaEventRecord(cg.e1, st)) || (e = cudaStreamWaitEvent(user, cg.e1, 0)) ||
        (e = cudaStreamSynchronize(st)))
        return cuda_fail(e, "LM: results");
    return ok();
}

// Whether the plan's free parameters are all among x0 .. sigma0 (the
// eight-derivative build of the Jacobian kernel serves them).
static bool lm_plan_narrow(const LmPlan &pl)
{
    for (int j = 0; j < pl.np; ++j)
        if (pl.idx[j] >= GBK_I0) return false;
    return true;
}

// Survey batches: the batched mode over a ragged plan, or the plain mode one
// galaxy (and geometry) at a time.
// Galaxies of a plan the Jacobian kernel serves with halo copies (A) and the
// rest (B), which the finite-difference Jacobian of the fused evaluator
// serves faster than the direct-halo shape.
static void tangent_split(const SurveyPlan &sp, std::vector<int32_t> &A, std::vector<int32_t> &B)
{
    A.clear();
    B.clear();
    for (int i = 0; i < sp.n_gal; ++i) {
        const int key = tangent_cluster_for(sp.geo[i]);
        (key > 0 && !tangent_key_direct(key) ? A : B).push_back(i);
    }
}

// Workspace of one batched part of a survey split: its plan's tables and LM state.
static size_t split_part_bytes(const gbk_geom *geoms, const std::vector<int32_t> &idx, const LmPlan &pl)
{
    if (idx.empty()) return 0;
    std::vector<gbk_geom> sub;
    for (int32_t i : idx) sub.push_back(geoms[i]);
    SurveyPlan p;
    if (survey_plan(sub.data(), (int)sub.size(), &p)) return 0;
    return p.table_bytes + lm_layout_pix((size_t)p.total_pix(), p.n_gal, pl).total;
}

// Gathered rows of one part: indices, parameters, bounds, observations and results.
static size_t split_rows_bytes(int n)
{
    return al256(sizeof(int32_t) * n) + 3 * al256(sizeof(double) * GBK_NPAR * n) + al256(sizeof(gbk_obs) * n) +
           al256(sizeof(double) * n) + 2 * al256(sizeof(int32_t) * n);
}

size_t lm_survey_workspace(const SurveyPlan &sp, const gbk_geom *geoms, const gbk_lm_opts *o)
{
    LmPlan pl;
    if (lm_plan(o, &pl)) return 0;
    if (o->mode == GBK_LM_PLAIN) {
        size_t m = 256;
        for (const Geom &g : sp.geo) m = std::max(m, lm_layout(g, 1, pl).total);
        return m;
    }
    if (pl.tangent && !lm_plan_narrow(pl)) {
        // survey batches carry the eight derivatives x0 .. sigma0; fits that
        // free I0 or h use finite differences throughout
        gbk_lm_opts ofd = *o;
        ofd.jacobian = GBK_JAC_FD_FORWARD;
        return lm_survey_workspace(sp, geoms, &ofd);
    }
    if (o->path != (int32_t)GBK_PATH_AUTO && o->path != (int32_t)GBK_PATH_FUSED && o->path != (int32_t)GBK_PATH_SPLIT) {
        fail(GBK_EINVAL, "LM evaluates on GBK_PATH_AUTO, GBK_PATH_FUSED or GBK_PATH_SPLIT (got %d)", o->path);
        return 0;
    }
    if (pl.tangent && o->path != (int32_t)GBK_PATH_FUSED) {
        // the ragged split Jacobian for every galaxy, where it serves the batch
        TsRaggedPlan rp;
        tsplit_ragged_plan(sp.geo, &rp);
        if (rp.ok) return lm_layout_pix((size_t)sp.total_pix(), sp.n_gal, pl, rp.total).total;
        if (o->path == (int32_t)GBK_PATH_SPLIT) {
            fail(GBK_EUNSUPPORTED, "the split Jacobian does not serve this batch (PSF radius <= 8, u = 1, cube model)");
            return 0;
        }
    }
    if (pl.tangent && !sp.tangent_ok) {
        // split: the Jacobian kernel where it fits, finite differences elsewhere
        std::vector<int32_t> A, B;
        tangent_split(sp, A, B);
        gbk_lm_opts ofd = *o;
        ofd.jacobian = GBK_JAC_FD_FORWARD;
        LmPlan pfd;
        lm_plan(&ofd, &pfd);
        size_t a = split_part_bytes(geoms, A, pl), b = split_part_bytes(geoms, B, pfd);
        if ((!A.empty() && a == 0) || b == 0) return 0;
        // the two parts run concurrently, each in its own region
        return al256(split_rows_bytes((int)A.size()) + a) + split_rows_bytes((int)B.size()) + b;
    }
    return lm_layout_pix((size_t)sp.total_pix(), sp.n_gal, pl).total;
}

__global__ void rows_copy_kernel(const uint32_t *src, uint32_t *dst, const int32_t *idx, int n, int row_words,
                                 int scatter)
{
    const long total = (long)n * row_words;
    for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const int r = (int)(t / row_words), w = (int)(t - (long)r * row_words);
        const long a = (long)idx[r] * row_words + w, b = (long)r * row_words + w;
        if (scatter) dst[a] = src[b];
        else dst[b] = src[a];
    }
}

static gbk_status rows_copy(const void *src, void *dst, const int32_t *idx, int n, size_t row_bytes, bool scatter,
                            cudaStream_t st)
{
    if (n == 0) return GBK_OK;
    const int words = (int)(row_bytes / 4);
    const long total = (long)n * words;
    const int blocks = (int)std::min<long>((total + 255) / 256, 152 * 8);
    rows_copy_kernel<<<blocks, 256, 0, st>>>((const uint32_t *)src, (uint32_t *)dst, idx, n, words, scatter ? 1 : 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "survey split: row copy");
    return GBK_OK;
}

// One part of a split survey fit: gather its rows, plan it, fit it batched,
// scatter the results back.
static gbk_status fit_part(const gbk_geom *geoms, const std::vector<int32_t> &idx, const gbk_obs *obs,
                           const double *lo, const double *hi, double *params, const gbk_lm_opts *o,
                           double *chi2_out, int32_t *iters_out, int32_t *status_out, char *ws, cudaStream_t st)
{
    const int n = (int)idx.size();
    if (n == 0) return GBK_OK;
    LmPlan pl;
    gbk_status s = lm_plan(o, &pl);
    if (s) return s;
    size_t off = 0;
    auto take = [&](size_t bytes) { char *p = ws + off; off += al256(bytes); return p; };
    int32_t *d_idx = (int32_t *)take(sizeof(int32_t) * n);
    double *d_p = (double *)take(sizeof(double) * GBK_NPAR * n);
    double *d_lo = (double *)take(sizeof(double) * GBK_NPAR * n);
    double *d_hi = (double *)take(sizeof(double) * GBK_NPAR * n);
    gbk_obs *d_obs = (gbk_obs *)take(sizeof(gbk_obs) * n);
    double *d_c = (double *)take(sizeof(double) * n);
    int32_t *d_it = (int32_t *)take(sizeof(int32_t) * n);
    int32_t *d_st = (int32_t *)take(sizeof(int32_t) * n);
    char *rest = ws + split_rows_bytes(n);
    cudaError_t e = cudaMemcpyAsync(d_idx, idx.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "survey split: index upload");
    const size_t prow = sizeof(double) * GBK_NPAR;
    if ((s = rows_copy(params, d_p, d_idx, n, prow, false, st)) || (s = rows_copy(lo, d_lo, d_idx, n, prow, false, st)) ||
        (s = rows_copy(hi, d_hi, d_idx, n, prow, false, st)) ||
        (s = rows_copy(obs, d_obs, d_idx, n, sizeof(gbk_obs), false, st)))
        return s;
    std::vector<gbk_geom> sub;
    for (int32_t i : idx) sub.push_back(geoms[i]);
    SurveyPlan sp;
    if ((s = survey_plan(sub.data(), n, &sp))) return s;
    if ((s = survey_upload(&sp, rest, st))) return s;
    EvalTarget t = {nullptr, &sp, LmSplit{false, false, 0}, nullptr};
    if ((s = lm_batched(t, n, d_obs, d_lo, d_hi, d_p, o, pl, d_c, d_it, d_st, rest + sp.table_bytes, st))) return s;
    if ((s = rows_copy(d_p, params, d_idx, n, prow, true, st)) || (s = rows_copy(d_c, chi2_out, d_idx, n, 8, true, st)) ||
        (s = rows_copy(d_it, iters_out, d_idx, n, 4, true, st)) || (s = rows_copy(d_st, status_out, d_idx, n, 4, true, st)))
        return s;
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "survey split: results");
    return GBK_OK;
}

gbk_status lm_survey(SurveyPlan &sp, const gbk_geom *geoms, const gbk_obs *obs, const double *lo, const double *hi,
                     double *params, const gbk_lm_opts *o, double *chi2_out, int32_t *iters_out, int32_t *status_out,
                     char *ws, size_t ws_bytes, cudaStream_t st)
{
    LmPlan pl;
    gbk_status s = lm_plan(o, &pl);
    if (s) return s;
    const size_t need = lm_survey_workspace(sp, geoms, o);
    if (need == 0 || ws_bytes < need) return fail(GBK_EWORKSPACE, "survey LM workspace too small");
    if (o->mode == GBK_LM_PLAIN) {
        for (int i = 0; i < sp.n_gal; ++i) {
            const size_t q = (size_t)i * GBK_NPAR;
            s = lm_plain(sp.geo[i], 1, obs + i, lo + q, hi + q, params + q, o, pl, chi2_out + i, iters_out + i,
                         status_out + i, ws, st);
            if (s) return s;
        }
        return ok();
    }
    if (pl.tangent && !lm_plan_narrow(pl)) {
        gbk_lm_opts ofd = *o;
        ofd.jacobian = GBK_JAC_FD_FORWARD;
        return lm_survey(sp, geoms, obs, lo, hi, params, &ofd, chi2_out, iters_out, status_out, ws, ws_bytes, st);
    }
    if (pl.tangent && o->path != (int32_t)GBK_PATH_FUSED) {
        // every galaxy on the ragged split Jacobian where it serves the batch
        // (the trial points on the survey's cluster evaluator)
        TsRaggedPlan rp;
        tsplit_ragged_plan(sp.geo, &rp);
        if (rp.ok) {
            const LmLayout L = lm_layout_pix((size_t)sp.total_pix(), sp.n_gal, pl, rp.total);
            char *rws = ws + L.sws;
            if ((s = tsplit_ragged_upload(rp, rws, st))) return s;
            EvalTarget t = {nullptr, &sp, LmSplit{false, true, rp.total}, rws, &rp};
            return lm_batched(t, sp.n_gal, obs, lo, hi, params, o, pl, chi2_out, iters_out, status_out, ws, st);
        }
        if (o->path == (int32_t)GBK_PATH_SPLIT)
            return fail(GBK_EUNSUPPORTED, "the split Jacobian does not serve this batch (PSF radius <= 8, u = 1, cube model)");
    }
    if (pl.tangent && !sp.tangent_ok) {
        // The Jacobian-kernel part (A) and the finite-difference part (B) are
        // independent batched LMs on disjoint galaxies and workspace regions;
        // B runs in a second host thread (its own LM stream) so that the two
        // overlap on the device, each while the other waits or polls.
        std::vector<int32_t> A, B;
        tangent_split(sp, A, B);
        gbk_lm_opts ofd = *o;
        ofd.jacobian = GBK_JAC_FD_FORWARD;
        LmPlan pfd;
        if ((s = lm_plan(&ofd, &pfd))) return s;
        char *wsB = ws + al256(split_rows_bytes((int)A.size()) + split_part_bytes(geoms, A, pl));
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return cuda_fail(e, "survey split: current device");
        gbk_status sb = GBK_OK;
        std::string eb;
        std::thread tb([&]() {
            cudaError_t ee = cudaSetDevice(dev);
            if (ee != cudaSuccess) {
                sb = GBK_ECUDA;
                eb = cudaGetErrorString(ee);
                return;
            }
            sb = fit_part(geoms, B, obs, lo, hi, params, &ofd, chi2_out, iters_out, status_out, wsB, st);
            if (sb) eb = gbk_last_error();
        });
        gbk_status sa = fit_part(geoms, A, obs, lo, hi, params, o, chi2_out, iters_out, status_out, ws, st);
        tb.join();
        if (sa) return sa;
        if (sb) return fail(sb, "survey split (finite-difference part): %s", eb.c_str());
        return ok();
    }
    EvalTarget t = {nullptr, &sp, LmSplit{false, false, 0}, nullptr};
    return lm_batched(t, sp.n_gal, obs, lo, hi, params, o, pl, chi2_out, iters_out, status_out, ws, st);
}

}  // namespace gbk

using namespace gbk;

// Keeps, for each galaxy r of a refitted part (galaxy idx[r]), the refit when
// its chi2 is lower than the first fit's (or the first is not finite).
__global__ void keep_better_kernel(const int32_t *idx, int n, const double *p_b, const double *c_b, const int32_t *it_b,
                                   const int32_t *st_b, double *params, double *chi2, int32_t *iters, int32_t *status,
                                   int32_t *used)
{
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        const int g = idx[r];
        const double ca = chi2[g], cb = c_b[r];
        const bool take_b = (cb < ca) || (!(ca == ca) && cb == cb);
        used[g] = take_b ? 1 : 2;
        if (!take_b) continue;
        for (int k = 0; k < GBK_NPAR; ++k) params[(size_t)g * GBK_NPAR + k] = p_b[(size_t)r * GBK_NPAR + k];
        chi2[g] = cb;
        iters[g] = it_b[r];
        status[g] = st_b[r];
    }
}

extern "C" {

size_t gbk_fit_lm_fallback_workspace_bytes(const gbk_geom *gin, int32_t n_gal, const gbk_lm_opts *opts)
{
    const size_t a = gbk_fit_lm_workspace_bytes(gin, n_gal, opts);
    if (a == 0) return 0;
    return al256(a) + split_rows_bytes(n_gal);
}

gbk_status gbk_fit_lm_fallback(const gbk_geom *gin, int32_t n_gal, const gbk_obs *obs, const double *lo,
                               const double *hi, double *params, const double *fallback_start,
                               const double *chi2_accept, const gbk_lm_opts *opts, double *chi2_out,
                               int32_t *iters_out, int32_t *status_out, int32_t *used_fallback, void *workspace,
                               size_t ws_bytes, void *stream)
{
    Geom g;
    gbk_status s = derive_geom(gin, &g);
    if (s) return s;
    if (n_gal < 0) return fail(GBK_EINVAL, "n_gal must be >= 0");
    if (n_gal == 0) return ok();
    const size_t need = gbk_fit_lm_fallback_workspace_bytes(gin, n_gal, opts);
    if (need == 0) return GBK_EINVAL;
    if (!workspace || ws_bytes < need)
        return fail(GBK_EWORKSPACE, "gbk_fit_lm_fallback needs %zu bytes of workspace (got %zu)", need, ws_bytes);
    if ((s = check_device_ptr(fallback_start, "fallback_start", 8)) ||
        (s = check_device_ptr(used_fallback, "used_fallback", 4)))
        return s;
    if (chi2_accept && (s = check_device_ptr(chi2_accept, "chi2_accept", 8))) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const size_t fit_bytes = gbk_fit_lm_workspace_bytes(gin, n_gal, opts);
    char *ws = (char *)workspace;
    // 1. every galaxy from the learned start
    if ((s = gbk_fit_lm(gin, n_gal, obs, lo, hi, params, opts, chi2_out, iters_out, status_out, ws, fit_bytes,
                        stream)))
        return s;
    cudaError_t e = cudaMemsetAsync(used_fallback, 0, sizeof(int32_t) * n_gal, st);
    if (e != cudaSuccess) return cuda_fail(e, "fallback: clearing used_fallback");
    // 2. the galaxies whose fit did not converge or ended above chi2_accept
    std::vector<int32_t> st_h(n_gal);
    std::vector<double> c_h(n_gal), acc_h;
    e = cudaMemcpyAsync(st_h.data(), status_out, sizeof(int32_t) * n_gal, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c_h.data(), chi2_out, sizeof(double) * n_gal, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && chi2_accept) {
        acc_h.resize(n_gal);
        e = cudaMemcpyAsync(acc_h.data(), chi2_accept, sizeof(double) * n_gal, cudaMemcpyDeviceToHost, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "fallback: reading the first fits");
    std::vector<int32_t> idx;
    for (int i = 0; i < n_gal; ++i) {
        const bool conv = st_h[i] == GBK_FIT_FTOL || st_h[i] == GBK_FIT_XTOL;
        const bool high = chi2_accept && !(c_h[i] <= acc_h[i]);
        if (!conv || high) idx.push_back(i);
    }
    const int n = (int)idx.size();
    if (n == 0) return ok();
    // 3. those galaxies from the fallback start, packed after the fit's region
    char *rows = ws + al256(fit_bytes);
    size_t off = 0;
    auto take = [&](size_t bytes) { char *p = rows + off; off += al256(bytes); return p; };
    int32_t *d_idx = (int32_t *)take(sizeof(int32_t) * n);
    double *d_p = (double *)take(sizeof(double) * GBK_NPAR * n);
    double *d_lo = (double *)take(sizeof(double) * GBK_NPAR * n);
    double *d_hi = (double *)take(sizeof(double) * GBK_NPAR * n);
    gbk_obs *d_obs = (gbk_obs *)take(sizeof(gbk_obs) * n);
    double *d_c = (double *)take(sizeof(double) * n);
    int32_t *d_it = (int32_t *)take(sizeof(int32_t) * n);
    int32_t *d_st = (int32_t *)take(sizeof(int32_t) * n);
    e = cudaMemcpyAsync(d_idx, idx.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "fallback: index upload");
    const size_t prow = sizeof(double) * GBK_NPAR;
    if ((s = rows_copy(fallback_start, d_p, d_idx, n, prow, false, st)) ||
        (s = rows_copy(lo, d_lo, d_idx, n, prow, false, st)) || (s = rows_copy(hi, d_hi, d_idx, n, prow, false, st)) ||
        (s = rows_copy(obs, d_obs, d_idx, n, sizeof(gbk_obs), false, st)))
        return s;
    const size_t part_bytes = gbk_fit_lm_workspace_bytes(gin, n, opts);
    if ((s = gbk_fit_lm(gin, n, d_obs, d_lo, d_hi, d_p, opts, d_c, d_it, d_st, ws, part_bytes, stream))) return s;
    // 4. keep the better of the two fits
    keep_better_kernel<<<(n + 255) / 256, 256, 0, st>>>(d_idx, n, d_p, d_c, d_it, d_st, params, chi2_out, iters_out,
                                                        status_out, used_fallback);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "fallback: merging the fits");
    return ok();
}

size_t gbk_fit_lm_workspace_bytes(const gbk_geom *gin, int32_t n_gal, const gbk_lm_opts *opts)
{
    ok();
    Geom g;
    if (derive_geom(gin, &g)) return 0;
    LmPlan pl;
    if (lm_plan(opts, &pl)) return 0;
    if (n_gal < 0) { fail(GBK_EINVAL, "n_gal must be >= 0"); return 0; }
    if (opts->mode == GBK_LM_PLAIN) return lm_layout(g, 1, pl).total;
    LmSplit spl;
    if (lm_split_plan(g, n_gal, pl, opts->path, &spl)) return 0;
    return lm_layout(g, n_gal, pl, spl.bytes).total;
}

gbk_status gbk_fit_lm(const gbk_geom *gin, int32_t n_gal, const gbk_obs *obs, const double *lo, const double *hi,
                      double *params, const gbk_lm_opts *opts, double *chi2_out, int32_t *iters_out,
                      int32_t *status_out, void *workspace, size_t ws_bytes, void *stream)
{
    Geom g;
    gbk_status s = derive_geom(gin, &g);
    if (s) return s;
    LmPlan pl;
    if ((s = lm_plan(opts, &pl))) return s;
    if (n_gal < 0) return fail(GBK_EINVAL, "n_gal must be >= 0");
    if (n_gal == 0) return ok();
    if (g.u != 1) return fail(GBK_EUNSUPPORTED, "LM fitting uses the fused path, which needs upsample == 1");
    FusedConfig fc;
    if (!fused_config(g, &fc)) return fail(GBK_EUNSUPPORTED, "the fused path cannot serve this geometry");
    if ((s = check_device_ptr(obs, "obs", 8)) || (s = check_device_ptr(lo, "lo", 8)) ||
        (s = check_device_ptr(hi, "hi", 8)) || (s = check_device_ptr(params, "params", 8)) ||
        (s = check_device_ptr(chi2_out, "chi2_out", 8)) || (s = check_device_ptr(iters_out, "iters_out", 4)) ||
        (s = check_device_ptr(status_out, "status_out", 4)))
        return s;
    LmSplit spl = {};
    if (opts->mode != GBK_LM_PLAIN && (s = lm_split_plan(g, n_gal, pl, opts->path, &spl))) return s;
    LmLayout L = lm_layout(g, opts->mode == GBK_LM_PLAIN ? 1 : n_gal, pl, spl.bytes);
    if (!workspace || ws_bytes < L.total)
        return fail(GBK_EWORKSPACE, "gbk_fit_lm needs %zu bytes of workspace (got %zu)", L.total, ws_bytes);
    if ((s = check_device_ptr(workspace, "workspace", 256))) return s;
    cudaStream_t st = (cudaStream_t)stream;
    if (opts->mode == GBK_LM_PLAIN)
        return lm_plain(g, n_gal, obs, lo, hi, params, opts, pl, chi2_out, iters_out, status_out, (char *)workspace, st);
    EvalTarget t = {&g, nullptr, spl, (char *)workspace + L.sws};
    return lm_batched(t, n_gal, obs, lo, hi, params, opts, pl, chi2_out, iters_out, status_out, (char *)workspace, st);
}

}  // extern "C"
