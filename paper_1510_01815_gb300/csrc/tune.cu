// tune.cu -- launch configuration of the fused kernel: a heuristic default
// and a measuring autotuner with a per-geometry cache.
//
// A configuration is (cluster size = CTAs per model, block size, grid shape).  The
// cluster size sets how many extended rows each CTA owns (its shared memory
// and the balance of the line-sampling work); the block size sets the
// register budget and the warps per SM.  The autotuner times every valid
// candidate on the caller's own batch and keeps the fastest for that
// geometry; later calls with the same geometry use it.
#include <algorithm>
#include <cmath>
#include <map>
#include <utility>
#include <vector>
#include <mutex>
#include <tuple>

#include "gbk_api_internal.h"
#include "k_fused.h"

namespace gbk {

using TuneKey = std::tuple<int, int, int, int, int, int>;

static std::mutex g_tune_mu;
static std::map<TuneKey, FusedConfig> g_tune_cache;

static TuneKey key_of(const Geom &g) { return TuneKey(g.nx, g.ny, g.nz, g.R, g.Rz, g.lsf_mode); }

static const int kBlockSizes[3] = {512, 384, 256};

static int min_blocks_per_sm(int threads) { (void)threads; return 2; }

// Shared memory per CTA that still lets min_blocks_per_sm CTAs share an SM
// (228 KB per SM, 1 KB reserved per CTA, 2 KB kept for static shared memory).
static size_t occupancy_smem(int threads)
{
    int b = min_blocks_per_sm(threads);
    return (size_t)(228 * 1024 / b) - 3 * 1024;
}

bool fused_config_valid(const Geom &g, int cs, int threads, int persistent, FusedConfig *cfg)
{
    if (persistent != 0 && persistent != 1) return false;
    if (g.model != GBK_MODEL_CUBE) {
        // the velocity-field kernel has one launch shape (one CTA per model)
        if (cs != 1 || threads != 256 || persistent != 0) return false;
        *cfg = FusedConfig{1, g.ey, 256, 0};
        return true;
    }
    if (g.u != 1 || cs < 1 || cs > kFusedMaxCluster || cs > g.ey) return false;
    if (threads != 512 && threads != 384 && threads != 256) return false;
    int band = (g.ey + cs - 1) / cs;
    if (fused_smem_bytes_host(g, band) > (size_t)kFusedMaxSmem) return false;
    cfg->cs = cs;
    cfg->band = band;
    cfg->threads = threads;
    cfg->persistent = persistent;
    return true;
}

// Fraction of the line-sampling rounds that do useful work in the CTA with
// the most extended rows (the cluster waits for it).
static double balance(const Geom &g, int cs, int threads)
{
    int band = (g.ey + cs - 1) / cs;
    double items = (double)band * g.ex;
    double rounds = std::ceil(items / threads);
    double avg = (double)g.ey * g.ex / cs;
    return avg / (rounds * threads);
}

static bool heuristic(const Geom &g, FusedConfig *cfg)
{
    const int threads = 512;
    double best = -1.0;
    for (int pass = 0; pass < 2 && best < 0.0; ++pass) {
        size_t cap = pass == 0 ? occupancy_smem(threads) : (size_t)kFusedMaxSmem;
        for (int cs = 1; cs <= kFusedMaxCluster; ++cs) {
            FusedConfig c;
            if (!fused_config_valid(g, cs, threads, 0, &c)) continue;
            if (fused_smem_bytes_host(g, c.band) > cap) continue;
            double b = balance(g, cs, threads);
            if (b > best + 1e-3) {
                best = b;
                *cfg = c;
            }
        }
    }
    return best > 0.0;
}

bool fused_config(const Geom &g, FusedConfig *cfg)
{
    if (g.u != 1) return false;
    if (g.model != GBK_MODEL_CUBE) return fused_config_valid(g, 1, 256, 0, cfg);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key_of(g));
        if (it != g_tune_cache.end()) {
            *cfg = it->second;
            return true;
        }
    }
    return heuristic(g, cfg);
}

}  // namespace gbk

using namespace gbk;

extern "C" {

gbk_status gbk_autotune(const gbk_geom *gin, int32_t n_models, const double *params, const gbk_obs *obs,
                        double *chi2_scratch, gbk_tuning *best, void *stream)
{
    Geom g;
    gbk_status s = derive_geom(gin, &g);
    if (s) return s;
    if (g.u != 1) return fail(GBK_EUNSUPPORTED, "the fused path (and its tuning) needs upsample == 1");
    if (n_models < 1) return fail(GBK_EINVAL, "n_models must be >= 1");
    if (!best) return fail(GBK_EINVAL, "best is NULL");
    if ((s = check_device_ptr(params, "params", 8))) return s;
    if ((s = check_device_ptr(chi2_scratch, "chi2_scratch", 8))) return s;
    if ((s = check_obs(obs))) return s;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    FusedConfig bestc = {0, 0, 0, 0};
    float best_ms = 0.f;
    int tried = 0;
    std::vector<std::pair<float, FusedConfig>> finalists;  // (screen median, configuration)
    for (int pers = 0; pers < 2; ++pers) {
    for (int ti = 0; ti < 3; ++ti) {
        for (int cs = 1; cs <= kFusedMaxCluster; ++cs) {
            FusedConfig c;
            if (!fused_config_valid(g, cs, kBlockSizes[ti], pers, &c)) continue;
            FusedArgs a = {};
            a.g = g;
            a.n_models = n_models;
            a.params = params;
            a.obs = *obs;
            a.chi2 = chi2_scratch;
            a.cs = c.cs;
            a.band = c.band;
            a.threads = c.threads;
            a.persistent = c.persistent;
            if (launch_fused(a, st) != GBK_OK) {  // e.g. a cluster shape the device cannot place
                cudaGetLastError();
                continue;
            }
            float times[3];
            bool ok_run = true;
            for (int rep = 0; rep < 3 && ok_run; ++rep) {
                cudaEventRecord(t0, st);
                ok_run = launch_fused(a, st) == GBK_OK;
                cudaEventRecord(t1, st);
                cudaEventSynchronize(t1);
                cudaEventElapsedTime(&times[rep], t0, t1);
            }
            if (!ok_run) {
                cudaGetLastError();
                continue;
            }
            float med = std::fmax(std::fmin(times[0], times[1]), std::fmin(std::fmax(times[0], times[1]), times[2]));
            ++tried;
            finalists.push_back({med, c});
            if (bestc.cs == 0 || med < best_ms) {
                best_ms = med;
                bestc = c;
            }
        }
    }
    }
    // The screen above takes a median of 3; its four fastest candidates,
    // often within a few per cent of each other, are re-timed with 9
    // launches each, interleaved so that clock or thermal drift affects them
    // alike, and the median decides.
    if (finalists.size() > 1) {
        std::sort(finalists.begin(), finalists.end(),
                  [](const std::pair<float, FusedConfig> &x, const std::pair<float, FusedConfig> &y) {
                      return x.first < y.first;
                  });
        if (finalists.size() > 4) finalists.resize(4);
        std::vector<std::vector<float>> reps(finalists.size());
        for (int rep = 0; rep < 9; ++rep) {
            for (size_t i = 0; i < finalists.size(); ++i) {
                const FusedConfig &c = finalists[i].second;
                FusedArgs a = {};
                a.g = g;
                a.n_models = n_models;
                a.params = params;
                a.obs = *obs;
                a.chi2 = chi2_scratch;
                a.cs = c.cs;
                a.band = c.band;
                a.threads = c.threads;
                a.persistent = c.persistent;
                float ms = 0.f;
                cudaEventRecord(t0, st);
                const bool ok_run = launch_fused(a, st) == GBK_OK;
                cudaEventRecord(t1, st);
                cudaEventSynchronize(t1);
                cudaEventElapsedTime(&ms, t0, t1);
                if (ok_run) reps[i].push_back(ms);
            }
        }
        for (size_t i = 0; i < finalists.size(); ++i) {
            if (reps[i].size() < 9) continue;
            std::nth_element(reps[i].begin(), reps[i].begin() + 4, reps[i].end());
            const float med = reps[i][4];
            if (i == 0 || med < best_ms) {
                best_ms = med;
                bestc = finalists[i].second;
            }
        }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "autotune");
    if (tried == 0) return fail(GBK_EUNSUPPORTED, "no fused configuration could run for this geometry");
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key_of(g)] = bestc;
    }
    best->cluster_ctas = bestc.cs;
    best->threads = bestc.threads;
    best->persistent = bestc.persistent;
    best->ms = best_ms;
    best->candidates = tried;
    return ok();
}

gbk_status gbk_get_tuning(const gbk_geom *gin, gbk_tuning *out)
{
    Geom g;
    gbk_status s = derive_geom(gin, &g);
    if (s) return s;
    if (!out) return fail(GBK_EINVAL, "out is NULL");
    FusedConfig c;
    if (!fused_config(g, &c)) return fail(GBK_EUNSUPPORTED, "the fused path cannot serve this geometry");
    out->cluster_ctas = c.cs;
    out->threads = c.threads;
    out->persistent = c.persistent;
    out->ms = 0.f;
    out->candidates = 0;
    return ok();
}

gbk_status gbk_set_tuning(const gbk_geom *gin, const gbk_tuning *t)
{
    Geom g;
    gbk_status s = derive_geom(gin, &g);
    if (s) return s;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    if (!t) {
        g_tune_cache.erase(key_of(g));
        return ok();
    }
    FusedConfig c;
    if (!fused_config_valid(g, t->cluster_ctas, t->threads, t->persistent, &c))
        return fail(GBK_EINVAL, "cluster_ctas %d / threads %d / persistent %d is not a valid fused configuration here",
                    t->cluster_ctas, t->threads, t->persistent);
    g_tune_cache[key_of(g)] = c;
    return ok();
}

}  // extern "C"
