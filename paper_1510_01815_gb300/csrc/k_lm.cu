// k_lm.cu -- device side of batched Levenberg-Marquardt (Sec. 2.3.1):
// finite-difference batch construction, FP64 normal equations, the damped
// Cholesky solve and the accept/reject update, one galaxy per thread or CTA.
#include "gbk_internal.cuh"
#include "k_lm.h"

namespace gbk {

// ----------------------------------------------------------------------------
// Finite-difference batch: slot 0 holds p; slot 1 + j holds p + h_j e_j (and
// for central differences slot 1 + P + j holds p - h_j e_j).  A forward step
// that would leave the box is taken backwards instead.
__global__ void lm_build_fd_kernel(LmArgs a)
{
    int gal = blockIdx.x * blockDim.x + threadIdx.x;
    if (gal >= a.n_gal || a.jskip[gal]) return;
    const double *p = a.params + (size_t)gal * GBK_NPAR;
    const double *hi = a.hi + (size_t)gal * GBK_NPAR;
    const double *lo = a.lo + (size_t)gal * GBK_NPAR;
    double *pb = a.pbatch + (size_t)gal * a.m * GBK_NPAR;
    for (int s = 0; s < a.m; ++s)
        for (int k = 0; k < GBK_NPAR; ++k) pb[s * GBK_NPAR + k] = p[k];
    for (int j = 0; j < a.np; ++j) {
        int k = a.free_idx[j];
        double h = a.fd_step[k];
        if (a.central) {
            pb[(1 + j) * GBK_NPAR + k] = p[k] + h;
            pb[(1 + a.np + j) * GBK_NPAR + k] = p[k] - h;
            a.hstep[(size_t)gal * a.np + j] = 2.0 * h;
        } else {
            if (p[k] + h > hi[k] && p[k] - h >= lo[k]) h = -h;
            pb[(1 + j) * GBK_NPAR + k] = p[k] + h;
            a.hstep[(size_t)gal * a.np + j] = h;
        }
    }
}

// ----------------------------------------------------------------------------
// J^T J and J^T r from the batch residuals; one CTA per galaxy.  Products are
// accumulated in FP32 per thread (a few residuals each), summed over each
// warp in FP32 and over the warps in FP64, in a fixed order.
template <int NP>
__global__ void __launch_bounds__(256) lm_normal_fd_kernel(LmArgs a)
{
    const int gal = blockIdx.x;
    if (a.jskip[gal]) return;
    constexpr int NT = NP * (NP + 1) / 2;
    size_t n2, base;
    if (a.pix_off) {
        n2 = (size_t)2 * (a.pix_off[gal + 1] - a.pix_off[gal]);
        base = (size_t)2 * a.m * a.pix_off[gal];
    } else {
        n2 = (size_t)2 * a.np_pix;
        base = (size_t)gal * a.m * n2;
    }
    const float *R = a.resid + base;
    float inv_h[NP];
    for (int j = 0; j < NP; ++j) inv_h[j] = (float)(1.0 / a.hstep[(size_t)gal * NP + j]);
    float E[NT + NP];  // J^T J upper triangle, then J^T r
    float *const jtj = E, *const jtr = E + NT;
    for (int t = 0; t < NT + NP; ++t) E[t] = 0.f;
    for (size_t i = threadIdx.x; i < n2; i += blockDim.x) {
        float r0 = R[i];
        float J[NP];
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            float rp = R[(size_t)(1 + j) * n2 + i];
            float rm = a.central ? R[(size_t)(1 + NP + j) * n2 + i] : r0;
            J[j] = (rp - rm) * inv_h[j];
        }
        int t = 0;
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            jtr[j] = fmaf(J[j], r0, jtr[j]);
#pragma unroll
            for (int k = j; k < NP; ++k) {
                jtj[t] = fmaf(J[j], J[k], jtj[t]);
                ++t;
            }
        }
    }
    // each warp's sums in FP32 by a reduce-scatter, the warps in FP64 in order
    __shared__ float red[8][NT + NP];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    warp_sum_scatter<NT + NP>(E, lane, red[warp]);
    __syncthreads();
    for (int t = threadIdx.x; t < NT + NP; t += blockDim.x) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += (double)red[w][t];
        if (t < NT) {
            // upper-triangle index t -> (j, k)
            int j = 0, rem = t;
            while (rem >= NP - j) { rem -= NP - j; ++j; }
            int k = j + rem;
            a.jtj[(size_t)gal * NP * NP + j * NP + k] = s;
            a.jtj[(size_t)gal * NP * NP + k * NP + j] = s;
        } else {
            a.jtr[(size_t)gal * NP + (t - NT)] = s;
        }
    }
    if (threadIdx.x == 0) a.chi2_cur[gal] = a.chi2_batch[(size_t)gal * a.m];
}

// ----------------------------------------------------------------------------
// Damped solve and trial point; one thread per galaxy.  A Cholesky failure
// raises lambda tenfold and retries.  Also the chi2 decrease the linearised
// model predicts for the (box-clipped) step, for the gain ratio.
template <int NP>
__global__ void lm_solve_kernel(LmArgs a)
{
    int gal = blockIdx.x * blockDim.x + threadIdx.x;
    if (gal >= a.n_gal || a.done[gal]) return;
    const double *JTJ = a.jtj + (size_t)gal * NP * NP;
    const double *JTr = a.jtr + (size_t)gal * NP;
    double lam = a.lambda[gal];
    // the lower triangle in registers (its loads issue together), the
    // diagonal's reciprocals so that the factorisation and the two
    // substitutions multiply instead of dividing
    double A[NP][NP], L[NP][NP], rd[NP], d[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j)
#pragma unroll
        for (int k = 0; k <= j; ++k) A[j][k] = JTJ[j * NP + k];
    bool ok = false;
    for (int attempt = 0; attempt < 12 && !ok; ++attempt) {
        ok = true;
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            if (!ok) break;
#pragma unroll
            for (int k = 0; k <= j; ++k) {
                double v = A[j][k];
                if (j == k) v += lam * (A[j][j] > 0.0 ? A[j][j] : 1.0);
#pragma unroll
                for (int q = 0; q < k; ++q) v -= L[j][q] * L[k][q];
                if (j == k) {
                    if (!(v > 0.0)) { ok = false; break; }
                    L[j][j] = sqrt(v);
                    rd[j] = 1.0 / L[j][j];
                } else {
                    L[j][k] = v * rd[k];
                }
            }
        }
        if (!ok) lam *= 10.0;
    }
    a.lambda[gal] = lam;
    double *pt = a.ptrial + (size_t)gal * GBK_NPAR;
    const double *p = a.params + (size_t)gal * GBK_NPAR;
    for (int k = 0; k < GBK_NPAR; ++k) pt[k] = p[k];
    if (!ok) {  // no usable damping: the trial equals p and will be rejected
        a.dnorm[gal] = 0.0;
        a.pnorm[gal] = 1.0;
        a.pred[gal] = 0.0;
        return;
    }
    // forward then back substitution: L L^T d = -JTr
    double y[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        double v = -JTr[j];
#pragma unroll
        for (int q = 0; q < j; ++q) v -= L[j][q] * y[q];
        y[j] = v * rd[j];
    }
#pragma unroll
    for (int j = NP - 1; j >= 0; --j) {
        double v = y[j];
#pragma unroll
        for (int q = j + 1; q < NP; ++q) v -= L[q][j] * d[q];
        d[j] = v * rd[j];
    }
    double dn = 0.0, pn = 0.0, s[NP];
    for (int j = 0; j < NP; ++j) {
        int k = a.free_idx[j];
        double lo = a.lo[(size_t)gal * GBK_NPAR + k], hi = a.hi[(size_t)gal * GBK_NPAR + k];
        double v = p[k] + d[j];
        v = v < lo ? lo : (v > hi ? hi : v);
        double step = v - p[k];
        pt[k] = v;
        s[j] = step;
        dn += step * step;
        pn += p[k] * p[k];
    }
    // predicted chi2 decrease of the clipped step s: -(2 s.J^T r + s.J^T J s)
    double sg = 0.0, sas = 0.0;
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        sg += s[j] * JTr[j];
        double as = 0.0;
#pragma unroll
        for (int k = 0; k < NP; ++k) as += (k <= j ? A[j][k] : A[k][j]) * s[k];
        sas += s[j] * as;
    }
    a.pred[gal] = -(2.0 * sg + sas);
    a.dnorm[gal] = sqrt(dn);
    a.pnorm[gal] = sqrt(pn);
}

// ----------------------------------------------------------------------------
__global__ void lm_accept_kernel(LmArgs a)
{
    int gal = blockIdx.x * blockDim.x + threadIdx.x;
    if (gal >= a.n_gal || a.done[gal]) return;
    double cc = a.chi2_cur[gal], ct = a.chi2_trial[gal];
    int st = GBK_FIT_RUNNING;
    bool accepted = false;
    int it = a.iters[gal] + 1;
    a.iters[gal] = it;
    if (!isfinite(cc)) {
        st = GBK_FIT_NONFINITE;
    } else if (isfinite(ct) && ct <= cc && a.dnorm[gal] > 0.0) {
        accepted = true;
        double *p = a.params + (size_t)gal * GBK_NPAR;
        const double *pt = a.ptrial + (size_t)gal * GBK_NPAR;
        for (int k = 0; k < GBK_NPAR; ++k) p[k] = pt[k];
        a.chi2_best[gal] = ct;
        a.chi2_cur[gal] = ct;
        // gain ratio of the actual to the predicted decrease (0 when none is
        // predicted); lambda x max(1/10, 1 - (2 rho - 1)^3), floor 1e-12
        const double pr = a.pred[gal];
        const double rho = pr > 0.0 ? (cc - ct) / pr : 0.0;
        const double q = 2.0 * rho - 1.0;
        double lam = a.lambda[gal] * fmax(0.1, 1.0 - q * q * q);
        a.lambda[gal] = lam < 1e-12 ? 1e-12 : lam;
        a.nu[gal] = 2.0;
        double rel = (cc - ct) / (cc > 1e-300 ? cc : 1e-300);
        if (rel < a.ftol) st = GBK_FIT_FTOL;
        else if (a.dnorm[gal] <= a.xtol * (a.pnorm[gal] + a.xtol)) st = GBK_FIT_XTOL;
    } else {
        a.chi2_best[gal] = cc;
        // rejected: lambda x nu, nu doubles
        const double nu = a.nu[gal];
        double lam = a.lambda[gal] * nu;
        a.lambda[gal] = lam;
        a.nu[gal] = 2.0 * nu;
        if (lam > 1e12) st = GBK_FIT_LAMBDA;
    }
    if (st == GBK_FIT_RUNNING && it >= a.max_iter) st = GBK_FIT_MAXITER;
    a.status[gal] = st;
    // A rejected step leaves params, and so J^T J, J^T r and chi2_cur, as
    // they were: the next iteration's Jacobian stage skips the galaxy and
    // its solve reuses them with the larger lambda (the values a new
    // Jacobian would give, bit for bit: its kernels are deterministic).
    a.jskip[gal] = (st != GBK_FIT_RUNNING || !accepted) ? 1 : 0;
    if (st != GBK_FIT_RUNNING) a.done[gal] = 1;
    else atomicAdd(a.n_active, 1);
}

__global__ void lm_init_kernel(LmArgs a, double lambda0)
{
    int gal = blockIdx.x * blockDim.x + threadIdx.x;
    if (gal >= a.n_gal) return;
    a.lambda[gal] = lambda0;
    a.nu[gal] = 2.0;
    a.iters[gal] = 0;
    a.status[gal] = GBK_FIT_RUNNING;
    a.done[gal] = 0;
    a.jskip[gal] = 0;
    a.chi2_best[gal] = __longlong_as_double(0x7ff8000000000000LL);
}

// ----------------------------------------------------------------------------
__global__ void lm_compact_kernel(LmCompactArgs c)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= c.n_live) return;
    const int s = c.live[j];
    for (int k = 0; k < GBK_NPAR; ++k) {
        c.params_n[(size_t)j * GBK_NPAR + k] = c.params[(size_t)s * GBK_NPAR + k];
        c.lo_n[(size_t)j * GBK_NPAR + k] = c.lo[(size_t)s * GBK_NPAR + k];
        c.hi_n[(size_t)j * GBK_NPAR + k] = c.hi[(size_t)s * GBK_NPAR + k];
    }
    c.obs_n[j] = c.obs[s];
    c.map_n[j] = c.map ? c.map[s] : s;
    c.lambda_n[j] = c.lambda[s];
    c.nu_n[j] = c.nu[s];
    c.chi2_cur_n[j] = c.chi2_cur[s];
    c.iters_n[j] = c.iters[s];
}

__global__ void lm_scatter_kernel(LmScatterArgs a)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const int o = a.map ? a.map[i] : i;
    if (a.params_out)
        for (int k = 0; k < GBK_NPAR; ++k)
            a.params_out[(size_t)o * GBK_NPAR + k] = a.params[(size_t)i * GBK_NPAR + k];
    a.chi2_out[o] = a.chi2_best[i];
    a.iters_out[o] = a.iters[i];
    a.status_out[o] = a.status[i];
}

void lm_launch_compact(const LmCompactArgs &c, cudaStream_t st)
{
    if (c.n_live > 0) lm_compact_kernel<<<(c.n_live + 127) / 128, 128, 0, st>>>(c);
}

void lm_launch_scatter(const LmScatterArgs &s, cudaStream_t st)
{
    if (s.n > 0) lm_scatter_kernel<<<(s.n + 127) / 128, 128, 0, st>>>(s);
}

// ----------------------------------------------------------------------------
template <int NP>
static void launch_np(const LmArgs &a, int which, cudaStream_t st)
{
    if (which == 0) lm_normal_fd_kernel<NP><<<a.n_gal, 256, 0, st>>>(a);
    else lm_solve_kernel<NP><<<(a.n_gal + 31) / 32, 32, 0, st>>>(a);
}

static void dispatch_np(const LmArgs &a, int which, cudaStream_t st)
{
    switch (a.np) {
    case 1: launch_np<1>(a, which, st); break;
    case 2: launch_np<2>(a, which, st); break;
    case 3: launch_np<3>(a, which, st); break;
    case 4: launch_np<4>(a, which, st); break;
    case 5: launch_np<5>(a, which, st); break;
    case 6: launch_np<6>(a, which, st); break;
    case 7: launch_np<7>(a, which, st); break;
    case 8: launch_np<8>(a, which, st); break;
    case 9: launch_np<9>(a, which, st); break;
    default: launch_np<10>(a, which, st); break;
    }
}

void lm_launch_init(const LmArgs &a, double lambda0, cudaStream_t st)
{
    lm_init_kernel<<<(a.n_gal + 127) / 128, 128, 0, st>>>(a, lambda0);
}

void lm_launch_build_fd(const LmArgs &a, cudaStream_t st)
{
    lm_build_fd_kernel<<<(a.n_gal + 127) / 128, 128, 0, st>>>(a);
}

void lm_launch_normal_fd(const LmArgs &a, cudaStream_t st) { dispatch_np(a, 0, st); }

void lm_launch_solve(const LmArgs &a, cudaStream_t st) { dispatch_np(a, 1, st); }

void lm_launch_accept(const LmArgs &a, cudaStream_t st)
{
    lm_accept_kernel<<<(a.n_gal + 127) / 128, 128, 0, st>>>(a);
}

}  // namespace gbk
