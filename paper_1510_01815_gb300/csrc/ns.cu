// ns.cu -- gbk_nested_sample: nested sampling (Sec. 2.3.2 of Bekiaris et al.
// 2015, which used MultiNest) with the likelihoods of each iteration's
// proposals evaluated in one batched launch (the split evaluator where it
// serves the geometry, else the cluster one).
//
// Readings (MultiNest's ellipsoidal clustering and importance weighting are
// not reproduced; the vanilla algorithm of Skilling 2004 with an ellipsoidal
// bound is):
//  - live points: n_live draws from the uniform prior over the free
//    parameters' box [lo, hi] (a parameter with lo == hi is fixed);
//  - each iteration draws `batch` proposals uniformly inside the bounding
//    ellipsoid of the live points (covariance-shaped, scaled to enclose every
//    live point, volume enlarged by 1.1 / efr), keeping those inside the
//    prior box, and evaluates their likelihood L = exp(-chi2 / 2) together;
//  - proposals are then taken in draw order: each one whose L exceeds the
//    current worst live point's replaces it; every replacement records the
//    worst point as dead with prior-volume shrinkage ln X -= 1 / n_live and
//    weight X_(i-1) - X_i;
//  - stop when ln(Z + L_max X) - ln Z < tol (MultiNest's evidence
//    tolerance) or after max_iter iterations; the remaining live points then
//    share X equally;
//  - random numbers: SplitMix64 (Steele, Lea & Flood 2014) seeded with
//    `seed`; uniforms use the top 53 bits; normals use Box-Muller.
#include <algorithm>
#include <cmath>
#include <vector>

#include "gbk_api_internal.h"
#include "k_fused.h"
#include "k_split.h"

namespace gbk {

struct SplitMix64 {
    uint64_t s;
    uint64_t next()
    {
        uint64_t z = (s += 0x9E3779B97F4A7C15ULL);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
        return z ^ (z >> 31);
    }
    double uniform() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }  // [0, 1)
    double normal()
    {
        double u1 = uniform(), u2 = uniform();
        if (u1 < 1e-300) u1 = 1e-300;
        return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
    }
};

static double logaddexp(double a, double b)
{
    if (a == -INFINITY) return b;
    if (b == -INFINITY) return a;
    double m = a > b ? a : b;
    return m + std::log(std::exp(a - m) + std::exp(b - m));
}

struct NsLayout {
    size_t params, chi2, split, split_bytes, total;
};

// The batch's parameters and chi2, then the split evaluator's workspace for
// a batch (0 where it does not serve the geometry: the cluster evaluator then
// takes the batches).
static NsLayout ns_layout(const Geom &g, int rows)
{
    NsLayout L;
    L.params = 0;
    L.chi2 = ((size_t)rows * GBK_NPAR * sizeof(double) + 255) & ~(size_t)255;
    L.split = L.chi2 + (((size_t)rows * sizeof(double) + 255) & ~(size_t)255);
    L.split_bytes = split_supported(g) ? split_workspace_bytes(g, rows) : 0;
    L.total = L.split + ((L.split_bytes + 255) & ~(size_t)255);
    return L;
}

static gbk_status ns_check(const gbk_ns_opts *o)
{
    if (!o) return fail(GBK_EINVAL, "opts is NULL");
    if (o->n_live < 2 || o->n_live > 1000000) return fail(GBK_EINVAL, "n_live must be in 2..1000000");
    if (o->batch < 1 || o->batch > 1000000) return fail(GBK_EINVAL, "batch must be in 1..1000000");
    if (!(o->tol > 0.0) || !(o->efr > 0.0)) return fail(GBK_EINVAL, "tol and efr must be > 0");
    if (o->max_iter < 1) return fail(GBK_EINVAL, "max_iter must be >= 1");
    return GBK_OK;
}

}  // namespace gbk

using namespace gbk;

extern "C" {

size_t gbk_nested_sample_workspace_bytes(const gbk_geom *gin, const gbk_ns_opts *opts)
{
    ok();
    Geom g;
    if (derive_geom(gin, &g) || ns_check(opts)) return 0;
    return ns_layout(g, std::max(opts->n_live, opts->batch)).total;
}

gbk_status gbk_nested_sample_traced(const gbk_geom *gin, const gbk_obs *obs, const double *lo, const double *hi,
                                    const gbk_ns_opts *opts, double *post_mean, double *post_std, double *log_z,
                                    int64_t *n_eval, int32_t *n_iter, void *workspace, size_t ws_bytes,
                                    void *stream, gbk_ns_trace *trace)
{
    if (trace && trace->max_iter < 0) return fail(GBK_EINVAL, "trace->max_iter must be >= 0");
    if (trace) trace->n_iter = 0;
    Geom g;
    gbk_status s = derive_geom(gin, &g);
    if (s) return s;
    if ((s = ns_check(opts))) return s;
    if (!lo || !hi || !post_mean || !post_std || !log_z || !n_eval || !n_iter)
        return fail(GBK_EINVAL, "a host argument is NULL");
    std::vector<int> ax;
    for (int k = 0; k < GBK_NPAR; ++k) {
        if (!(std::isfinite(lo[k]) && std::isfinite(hi[k]) && lo[k] <= hi[k]))
            return fail(GBK_EINVAL, "prior bounds of parameter %d are invalid", k);
        if (hi[k] > lo[k]) ax.push_back(k);
    }
    const int P = (int)ax.size();
    if (P == 0) return fail(GBK_EINVAL, "no free parameter (lo == hi everywhere)");
    FusedConfig fc;
    if (g.u != 1 || !fused_config(g, &fc)) return fail(GBK_EUNSUPPORTED, "nested sampling uses the fused path");
    if ((s = check_obs(obs))) return s;
    const int N = opts->n_live, K = opts->batch;
    NsLayout L = ns_layout(g, std::max(N, K));
    if (!workspace || ws_bytes < L.total)
        return fail(GBK_EWORKSPACE, "gbk_nested_sample needs %zu bytes of workspace (got %zu)", L.total, ws_bytes);
    if ((s = check_device_ptr(workspace, "workspace", 256))) return s;
    cudaStream_t st = (cudaStream_t)stream;
    double *d_p = (double *)((char *)workspace + L.params), *d_c = (double *)((char *)workspace + L.chi2);
    long long evals = 0;

    auto evaluate = [&](const std::vector<double> &pv, int n, std::vector<double> &chi2) -> gbk_status {
        cudaError_t e = cudaMemcpyAsync(d_p, pv.data(), sizeof(double) * GBK_NPAR * n, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "nested sampling: parameter upload");
        gbk_status s2;
        if (L.split_bytes) {
            s2 = launch_split(g, n, d_p, obs, nullptr, d_c, nullptr, (char *)workspace + L.split, L.split_bytes, st);
        } else {
            FusedArgs a = {};
            a.g = g;
            a.n_models = n;
            a.params = d_p;
            a.obs = *obs;
            a.chi2 = d_c;
            a.cs = fc.cs;
            a.band = fc.band;
            a.threads = fc.threads;
            a.persistent = fc.persistent;
            s2 = launch_fused(a, st);
        }
        if (s2) return s2;
        chi2.resize(n);
        e = cudaMemcpyAsync(chi2.data(), d_c, sizeof(double) * n, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "nested sampling: likelihood download");
        evals += n;
        return GBK_OK;
    };

    SplitMix64 rng{opts->seed};
    // live points
    std::vector<double> live((size_t)N * GBK_NPAR), logl(N), chi2;
    for (int i = 0; i < N; ++i)
        for (int k = 0; k < GBK_NPAR; ++k)
            live[(size_t)i * GBK_NPAR + k] = (hi[k] > lo[k]) ? lo[k] + (hi[k] - lo[k]) * rng.uniform() : lo[k];
    if ((s = evaluate(live, N, chi2))) return s;
    for (int i = 0; i < N; ++i) logl[i] = std::isfinite(chi2[i]) ? -0.5 * chi2[i] : -INFINITY;
    if (trace && trace->live0) std::copy(live.begin(), live.end(), trace->live0);
    if (trace && trace->live0_chi2) std::copy(chi2.begin(), chi2.begin() + N, trace->live0_chi2);

    // dead points: parameters and log weights (log L + log w)
    std::vector<double> dead_p, dead_lw;
    double logz = -INFINITY, logx = 0.0;
    const double log_shrink = std::log1p(-std::exp(-1.0 / N));  // log(1 - e^{-1/N})
    int it = 0;
    std::vector<double> prop((size_t)K * GBK_NPAR), mu(P), C((size_t)P * P), Lc((size_t)P * P), Ci((size_t)P * P);
    for (; it < opts->max_iter; ++it) {
        // stopping rule
        double lmax = *std::max_element(logl.begin(), logl.end());
        if (it > 0 && logaddexp(logz, lmax + logx) - logz < opts->tol) break;
        // bounding ellipsoid of the live points over the free axes
        std::fill(mu.begin(), mu.end(), 0.0);
        for (int i = 0; i < N; ++i)
            for (int a = 0; a < P; ++a) mu[a] += live[(size_t)i * GBK_NPAR + ax[a]];
        for (int a = 0; a < P; ++a) mu[a] /= N;
        std::fill(C.begin(), C.end(), 0.0);
        for (int i = 0; i < N; ++i)
            for (int a = 0; a < P; ++a)
                for (int b = 0; b <= a; ++b)
                    C[a * P + b] += (live[(size_t)i * GBK_NPAR + ax[a]] - mu[a]) * (live[(size_t)i * GBK_NPAR + ax[b]] - mu[b]);
        for (int a = 0; a < P; ++a) {
            for (int b = 0; b <= a; ++b) C[a * P + b] /= N;
            double span = hi[ax[a]] - lo[ax[a]];
            C[a * P + a] += 1e-12 * span * span;  // keeps the covariance positive definite
        }
        // Cholesky C = Lc Lc^T
        std::fill(Lc.begin(), Lc.end(), 0.0);
        for (int a = 0; a < P; ++a)
            for (int b = 0; b <= a; ++b) {
                double v = C[a * P + b];
                for (int q = 0; q < b; ++q) v -= Lc[a * P + q] * Lc[b * P + q];
                Lc[a * P + b] = (a == b) ? std::sqrt(std::fmax(v, 1e-300)) : v / Lc[b * P + b];
            }
        // scale so the ellipsoid encloses every live point: max of |Lc^-1 (x - mu)|^2
        double k2 = 0.0;
        std::vector<double> y(P);
        for (int i = 0; i < N; ++i) {
            for (int a = 0; a < P; ++a) {
                double v = live[(size_t)i * GBK_NPAR + ax[a]] - mu[a];
                for (int q = 0; q < a; ++q) v -= Lc[a * P + q] * y[q];
                y[a] = v / Lc[a * P + a];
            }
            double d2 = 0.0;
            for (int a = 0; a < P; ++a) d2 += y[a] * y[a];
            k2 = std::fmax(k2, d2);
        }
        double scale = std::sqrt(k2) * std::pow(1.1 / opts->efr, 1.0 / P);
        // proposals: uniform in the ellipsoid, kept if inside the prior box
        int made = 0;
        long long tries = 0;
        std::vector<double> z(P);
        while (made < K && tries < 1000LL * K) {
            ++tries;
            double r2 = 0.0;
            for (int a = 0; a < P; ++a) { z[a] = rng.normal(); r2 += z[a] * z[a]; }
            double rad = std::pow(rng.uniform(), 1.0 / P) / std::sqrt(std::fmax(r2, 1e-300));
            double *q = &prop[(size_t)made * GBK_NPAR];
            for (int k = 0; k < GBK_NPAR; ++k) q[k] = lo[k];
            bool inside = true;
            for (int a = 0; a < P; ++a) {
                double v = mu[a];
                for (int b = 0; b <= a; ++b) v += Lc[a * P + b] * z[b] * rad * scale;
                if (v < lo[ax[a]] || v > hi[ax[a]]) { inside = false; break; }
                q[ax[a]] = v;
            }
            if (inside) ++made;
        }
        if (made == 0) break;
        if ((s = evaluate(prop, made, chi2))) return s;
        // the iteration's record, when one is kept
        const bool rec = trace && it < trace->max_iter;
        if (rec) {
            const size_t t = (size_t)it;
            if (trace->n_props) trace->n_props[t] = made;
            if (trace->props) std::copy(prop.begin(), prop.begin() + (size_t)made * GBK_NPAR, trace->props + t * K * GBK_NPAR);
            if (trace->chi2) std::copy(chi2.begin(), chi2.begin() + made, trace->chi2 + t * K);
            if (trace->replaced) std::fill(trace->replaced + t * K, trace->replaced + t * K + made, -1);
            trace->n_iter = it + 1;
        }
        // replacements in draw order
        for (int j = 0; j < made; ++j) {
            double lj = std::isfinite(chi2[j]) ? -0.5 * chi2[j] : -INFINITY;
            int w = (int)(std::min_element(logl.begin(), logl.end()) - logl.begin());
            if (!(lj > logl[w])) continue;
            if (rec && trace->replaced) trace->replaced[(size_t)it * K + j] = w;
            double lw = logx + log_shrink + logl[w];  // log(L_w (X_{i-1} - X_i))
            logz = logaddexp(logz, lw);
            dead_p.insert(dead_p.end(), &live[(size_t)w * GBK_NPAR], &live[(size_t)w * GBK_NPAR] + GBK_NPAR);
            dead_lw.push_back(lw);
            logx -= 1.0 / N;
            std::copy(&prop[(size_t)j * GBK_NPAR], &prop[(size_t)j * GBK_NPAR] + GBK_NPAR, &live[(size_t)w * GBK_NPAR]);
            logl[w] = lj;
        }
    }
    // the remaining live points share X
    for (int i = 0; i < N; ++i) {
        double lw = logx - std::log((double)N) + logl[i];
        logz = logaddexp(logz, lw);
        dead_p.insert(dead_p.end(), &live[(size_t)i * GBK_NPAR], &live[(size_t)i * GBK_NPAR] + GBK_NPAR);
        dead_lw.push_back(lw);
    }
    // posterior moments
    for (int k = 0; k < GBK_NPAR; ++k) { post_mean[k] = 0.0; post_std[k] = 0.0; }
    size_t nd = dead_lw.size();
    for (size_t i = 0; i < nd; ++i) {
        double wgt = std::exp(dead_lw[i] - logz);
        for (int k = 0; k < GBK_NPAR; ++k) post_mean[k] += wgt * dead_p[i * GBK_NPAR + k];
    }
    for (size_t i = 0; i < nd; ++i) {
        double wgt = std::exp(dead_lw[i] - logz);
        for (int k = 0; k < GBK_NPAR; ++k) {
            double d = dead_p[i * GBK_NPAR + k] - post_mean[k];
            post_std[k] += wgt * d * d;
        }
    }
    for (int k = 0; k < GBK_NPAR; ++k) post_std[k] = std::sqrt(post_std[k]);
    *log_z = logz;
    *n_eval = evals;
    *n_iter = it;
    return ok();
}

gbk_status gbk_nested_sample(const gbk_geom *gin, const gbk_obs *obs, const double *lo, const double *hi,
                             const gbk_ns_opts *opts, double *post_mean, double *post_std, double *log_z,
                             int64_t *n_eval, int32_t *n_iter, void *workspace, size_t ws_bytes, void *stream)
{
    return gbk_nested_sample_traced(gin, obs, lo, hi, opts, post_mean, post_std, log_z, n_eval, n_iter, workspace,
                                    ws_bytes, stream, nullptr);
}

}  // extern "C"
