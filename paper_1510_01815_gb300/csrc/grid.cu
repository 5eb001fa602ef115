// grid.cu -- gbk_grid: the nested-grids optimiser of Sec. 2.3.3 of Bekiaris
// et al. 2015.  Every node of a regular grid over the free parameters is
// evaluated (batched chi2: the split evaluator where it serves the geometry,
// else the cluster one), the best node is selected, and a new grid
// with the same number of nodes is built around it over a smaller volume.
//
// Readings: level 0 spans [lo, hi] with n_j nodes per parameter including
// both ends; level l+1 spans best_j +- one level-l step, clipped to [lo, hi];
// the linear node index is row-major in parameter order (the first free
// parameter varies slowest); ties go to the lowest index.  Node values are
// lo_j + i_j * ((hi_j - lo_j) / (n_j - 1)) in FP64, the same expression the
// oracle uses, so both sides evaluate identical parameter vectors.
#include <cmath>
#include <vector>

#include "gbk_api_internal.h"
#include "k_fused.h"
#include "k_split.h"

namespace gbk {

struct GridSpec {
    int nfree;
    int idx[GBK_NPAR];      // free parameter indices (grid axes), slowest first
    int n[GBK_NPAR];        // nodes per axis
    double lo[GBK_NPAR];    // axis start of this level
    double step[GBK_NPAR];  // axis step of this level
    double base[GBK_NPAR];  // values of every parameter (fixed ones used as is)
};

__global__ void grid_nodes_kernel(GridSpec s, long long first, int count, double *params)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    long long lin = first + t;
    double *p = params + (size_t)t * GBK_NPAR;
    for (int k = 0; k < GBK_NPAR; ++k) p[k] = s.base[k];
    for (int a = s.nfree - 1; a >= 0; --a) {
        long long i = lin % s.n[a];
        lin /= s.n[a];
        p[s.idx[a]] = s.lo[a] + (double)i * s.step[a];
    }
}

// Block-wise argmin with the lowest-index tie rule; NaN counts as +inf.
__device__ __forceinline__ bool better(double c1, long long i1, double c2, long long i2)
{
    bool n1 = !(c1 == c1), n2 = !(c2 == c2);
    if (n1 != n2) return n2;
    if (!n1 && c1 != c2) return c1 < c2;
    return i1 < i2;
}

__global__ void grid_argmin_kernel(const double *chi2, long long first, int count, double *best_c,
                                   long long *best_i, int slot)
{
    __shared__ double sc[256];
    __shared__ long long si[256];
    double c = INFINITY;
    long long i = -1;
    for (int t = threadIdx.x; t < count; t += blockDim.x) {
        double v = chi2[t];
        if (i < 0 || better(v, first + t, c, i)) {
            c = v;
            i = first + t;
        }
    }
    sc[threadIdx.x] = c;
    si[threadIdx.x] = i;
    __syncthreads();
    for (int off = blockDim.x / 2; off > 0; off >>= 1) {
        if (threadIdx.x < off) {
            double c2 = sc[threadIdx.x + off];
            long long i2 = si[threadIdx.x + off];
            if (i2 >= 0 && (si[threadIdx.x] < 0 || better(c2, i2, sc[threadIdx.x], si[threadIdx.x]))) {
                sc[threadIdx.x] = c2;
                si[threadIdx.x] = i2;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        best_c[slot] = sc[0];
        best_i[slot] = si[0];
    }
}

static size_t al256g(size_t b) { return (b + 255) & ~(size_t)255; }

struct GridLayout {
    size_t params, chi2, bc, bi, split, split_bytes, total;
};

// split_bytes: the split evaluator's workspace for a chunk (0 where it does
// not serve the geometry; the cluster evaluator then takes the chunks).
static GridLayout grid_layout(int chunk, long long nchunks, size_t split_bytes)
{
    GridLayout L;
    size_t o = 0;
    L.params = o; o += al256g(sizeof(double) * GBK_NPAR * chunk);
    L.chi2 = o; o += al256g(sizeof(double) * chunk);
    L.bc = o; o += al256g(sizeof(double) * nchunks);
    L.bi = o; o += al256g(sizeof(long long) * nchunks);
    L.split = o; o += al256g(split_bytes);
    L.split_bytes = split_bytes;
    L.total = o;
    return L;
}

static size_t grid_split_bytes(const Geom &g, int chunk)
{
    return split_supported(g) ? split_workspace_bytes(g, chunk) : 0;
}

static gbk_status grid_plan(const int32_t *nodes, int32_t chunk, GridSpec *s, long long *total)
{
    if (!nodes) return fail(GBK_EINVAL, "nodes is NULL");
    if (chunk < 1 || chunk > (1 << 22)) return fail(GBK_EINVAL, "chunk must be in 1..4194304");
    s->nfree = 0;
    long long N = 1;
    for (int k = 0; k < GBK_NPAR; ++k) {
        if (nodes[k] < 1) return fail(GBK_EINVAL, "nodes[%d] must be >= 1", k);
        if (nodes[k] > 1) {
            s->idx[s->nfree] = k;
            s->n[s->nfree] = nodes[k];
            s->nfree++;
            N *= nodes[k];
            if (N > (1LL << 40)) return fail(GBK_EINVAL, "too many grid nodes");
        }
    }
    if (s->nfree == 0) return fail(GBK_EINVAL, "no parameter has more than one node");
    *total = N;
    return GBK_OK;
}

}  // namespace gbk

using namespace gbk;

extern "C" {

size_t gbk_grid_workspace_bytes(const gbk_geom *gin, const int32_t *nodes, int32_t chunk)
{
    ok();
    Geom g;
    if (derive_geom(gin, &g)) return 0;
    GridSpec s;
    long long N;
    if (grid_plan(nodes, chunk, &s, &N)) return 0;
    long long nch = (N + chunk - 1) / chunk;
    return grid_layout(chunk, nch, grid_split_bytes(g, chunk)).total;
}

gbk_status gbk_grid(const gbk_geom *gin, const gbk_obs *obs, const double *lo, const double *hi,
                    const int32_t *nodes, const double *fixed, int32_t levels, int32_t chunk, double *best_params,
                    int64_t *best_index, double *best_chi2, void *workspace, size_t ws_bytes, void *stream)
{
    Geom g;
    gbk_status s = derive_geom(gin, &g);
    if (s) return s;
    GridSpec spec;
    long long N;
    if ((s = grid_plan(nodes, chunk, &spec, &N))) return s;
    if (!lo || !hi || !fixed || !best_params || !best_index || !best_chi2)
        return fail(GBK_EINVAL, "a host array argument is NULL");
    if (levels < 1 || levels > 64) return fail(GBK_EINVAL, "levels must be in 1..64");
    for (int a = 0; a < spec.nfree; ++a) {
        int k = spec.idx[a];
        if (!(std::isfinite(lo[k]) && std::isfinite(hi[k]) && lo[k] <= hi[k]))
            return fail(GBK_EINVAL, "bounds of parameter %d are invalid", k);
    }
    FusedConfig fc;
    if (g.u != 1 || !fused_config(g, &fc)) return fail(GBK_EUNSUPPORTED, "the grid search uses the fused path");
    if ((s = check_obs(obs))) return s;
    long long nch = (N + chunk - 1) / chunk;
    GridLayout L = grid_layout(chunk, nch, grid_split_bytes(g, chunk));
    if (!workspace || ws_bytes < L.total)
        return fail(GBK_EWORKSPACE, "gbk_grid needs %zu bytes of workspace (got %zu)", L.total, ws_bytes);
    if ((s = check_device_ptr(workspace, "workspace", 256))) return s;
    cudaStream_t st = (cudaStream_t)stream;
    char *ws = (char *)workspace;
    double *d_params = (double *)(ws + L.params), *d_chi2 = (double *)(ws + L.chi2);
    double *d_bc = (double *)(ws + L.bc);
    long long *d_bi = (long long *)(ws + L.bi);
    double llo[GBK_NPAR], lhi[GBK_NPAR];
    for (int k = 0; k < GBK_NPAR; ++k) {
        spec.base[k] = fixed[k];
        llo[k] = lo[k];
        lhi[k] = hi[k];
    }
    std::vector<double> h_bc(nch);
    std::vector<long long> h_bi(nch);
    for (int lev = 0; lev < levels; ++lev) {
        for (int a = 0; a < spec.nfree; ++a) {
            int k = spec.idx[a];
            spec.lo[a] = llo[k];
            spec.step[a] = (lhi[k] - llo[k]) / (double)(spec.n[a] - 1);
        }
        for (long long c = 0; c < nch; ++c) {
            long long first = c * chunk;
            int count = (int)((N - first) < chunk ? (N - first) : chunk);
            grid_nodes_kernel<<<(count + 127) / 128, 128, 0, st>>>(spec, first, count, d_params);
            if (L.split_bytes) {
                if ((s = launch_split(g, count, d_params, obs, nullptr, d_chi2, nullptr, ws + L.split, L.split_bytes,
                                      st)))
                    return s;
            } else {
                FusedArgs a = {};
                a.g = g;
                a.n_models = count;
                a.params = d_params;
                a.obs = *obs;
                a.chi2 = d_chi2;
                a.cs = fc.cs;
                a.band = fc.band;
                a.threads = fc.threads;
                a.persistent = fc.persistent;
                if ((s = launch_fused(a, st))) return s;
            }
            grid_argmin_kernel<<<1, 256, 0, st>>>(d_chi2, first, count, d_bc, d_bi, (int)c);
        }
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(h_bc.data(), d_bc, sizeof(double) * nch, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h_bi.data(), d_bi, sizeof(long long) * nch, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "grid level");
        // chunks in order: the lowest index wins ties
        double bc = h_bc[0];
        long long bi = h_bi[0];
        for (long long c = 1; c < nch; ++c) {
            double cc = h_bc[c];
            bool nb = !(bc == bc), nc = !(cc == cc);
            if ((nb && !nc) || (!nb && !nc && cc < bc)) {
                bc = cc;
                bi = h_bi[c];
            }
        }
        best_index[lev] = bi;
        best_chi2[lev] = bc;
        // best node's parameters, then the next level's box
        long long lin = bi;
        double bp[GBK_NPAR];
        for (int k = 0; k < GBK_NPAR; ++k) bp[k] = fixed[k];
        for (int a = spec.nfree - 1; a >= 0; --a) {
            long long i = lin % spec.n[a];
            lin /= spec.n[a];
            bp[spec.idx[a]] = spec.lo[a] + (double)i * spec.step[a];
        }
        for (int k = 0; k < GBK_NPAR; ++k) best_params[k] = bp[k];
        for (int a = 0; a < spec.nfree; ++a) {
            int k = spec.idx[a];
            double nlo = bp[k] - spec.step[a], nhi = bp[k] + spec.step[a];
            llo[k] = nlo < lo[k] ? lo[k] : nlo;
            lhi[k] = nhi > hi[k] ? hi[k] : nhi;
        }
    }
    return ok();
}

}  // extern "C"
