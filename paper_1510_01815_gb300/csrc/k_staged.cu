// k_staged.cu -- the forward model as separate kernels that materialise the
// cube in HBM (Sec. 2.2.2-2.2.6 of Bekiaris et al. 2015):
//
//   model_cube_kernel   per-voxel model on the fine extended grid, written as
//                       coalesced float4 rows (Sec. 2.2.2)
//   conv3d_kernel       separable PSF x LSF valid convolution (Eq. 9,
//                       Sec. 2.2.3): x and y passes in shared memory on one
//                       extended z slice at a time, z pass over a shared ring
//                       of 2 Rz + 1 slices
//   downsample_kernel   mean of u^3 blocks (Sec. 2.2.4)
//   moments_kernel      moment maps, weighted residuals and per-block chi2
//                       partials (Sec. 2.2.5-2.2.6)
//   chi2_final_kernel   fixed-order FP64 sum of the partials
//   chi2_maps_kernel    Eq. 11 from caller-supplied maps, one block per model
#include "gbk_api_internal.h"
#include "gbk_internal.cuh"
#include "k_staged.h"

namespace gbk {

// ----------------------------------------------------------------------------
// Model cube.  One thread owns four consecutive x spaxels of one extended row
// and walks every extended channel, so the geometry (atan, sqrt, exp) is
// computed once per spaxel and each channel costs one ex2 per voxel.
__global__ void __launch_bounds__(256) model_cube_kernel(StagedArgs a)
{
    const Geom &g = a.g;
    const int pitch4 = a.e_pitch / 4;
    const long per_model = (long)g.ey * pitch4;
    const int blocks_per_model = (int)((per_model + blockDim.x - 1) / blockDim.x);
    const int model = blockIdx.x / blocks_per_model;
    const long item = (long)(blockIdx.x - model * blocks_per_model) * blockDim.x + threadIdx.x;
    __shared__ ModelConst mc;
    if (threadIdx.x == 0) mc = model_const(a.params + (size_t)model * GBK_NPAR, g);
    __syncthreads();
    if (item >= per_model) return;
    const ModelConst c = mc;
    const int ye = (int)(item / pitch4);
    const int xe0 = (int)(item - (long)ye * pitch4) * 4;
    const float inv_u = 1.f / (float)g.u;
    float y = ((float)(ye - g.R) + 0.5f) * inv_u - 0.5f;
    float vl[4], A[4];
    for (int q = 0; q < 4; ++q) {
        int xe = xe0 + q;
        float x = ((float)(xe - g.R) + 0.5f) * inv_u - 0.5f;
        float br;
        los(c, x, y, vl[q], br);
        A[q] = (xe < g.ex && c.valid) ? c.amp * br : 0.f;
        if (!c.valid) A[q] = __int_as_float(0x7fc00000);
    }
    float4 *out = reinterpret_cast<float4 *>(a.ext + (size_t)model * a.e_model_stride) + item;
    const size_t plane4 = (size_t)g.ey * pitch4;
    const float al = c.alpha;
    for (int e = 0; e < g.ez; ++e) {
        // velocity of fine channel e - Rz
        float kc = ((float)(e - g.Rz) + 0.5f) * inv_u - 0.5f;
        float v = g.vc + (kc - 0.5f * (float)(g.nz - 1)) * g.dv;
        float4 o;
        float u0 = al * (v - vl[0]), u1 = al * (v - vl[1]), u2 = al * (v - vl[2]), u3 = al * (v - vl[3]);
        o.x = A[0] * ex2_approx(-u0 * u0);
        o.y = A[1] * ex2_approx(-u1 * u1);
        o.z = A[2] * ex2_approx(-u2 * u2);
        o.w = A[3] * ex2_approx(-u3 * u3);
        out[(size_t)e * plane4] = o;
    }
}

// ----------------------------------------------------------------------------
// Separable valid convolution of the fine extended cube.  Block = TX x TY
// output spaxels; shared memory holds one input slice with its halo, the
// x-pass result and a ring of 2 Rz + 1 xy-convolved slices.
__global__ void __launch_bounds__(kConvTX * kConvTY) conv3d_kernel(StagedArgs a)
{
    const Geom &g = a.g;
    const int tiles_x = (g.nxf + kConvTX - 1) / kConvTX;
    const int tiles_y = (g.nyf + kConvTY - 1) / kConvTY;
    const int tiles = tiles_x * tiles_y;
    const int model = blockIdx.x / tiles;
    const int t = blockIdx.x - model * tiles;
    const int ty0 = (t / tiles_x) * kConvTY, tx0 = (t % tiles_x) * kConvTX;
    const int R = g.R, Rz = g.Rz, W = 2 * Rz + 1;
    const int SX = kConvTX + 2 * R, SY = kConvTY + 2 * R;

    extern __shared__ __align__(16) float sm[];
    float *wxy = sm;                          // 2R+1
    float *wz = wxy + 2 * R + 1;              // 2Rz+1
    float *slab = wz + W;                     // SY x SX
    float *xp = slab + SY * SX;               // SY x TX
    float *ring = xp + SY * kConvTX;          // W x TY x TX

    block_taps(g.sig_xy, R, wxy);
    block_taps(g.sig_z, Rz, wz);

    const float *E = a.ext + (size_t)model * a.e_model_stride;
    float *F = a.fine + (size_t)model * a.f_model_stride;
    const int tid = threadIdx.x;
    const int lx = tid % kConvTX, ly = tid / kConvTX;
    const size_t eplane = (size_t)g.ey * a.e_pitch;
    const size_t fplane = (size_t)g.nyf * g.nxf;

    for (int e = 0; e < g.ez; ++e) {
        // load slice e: extended rows ty0 .. ty0+SY-1, columns tx0 .. tx0+SX-1
        const float *Es = E + (size_t)e * eplane;
        for (int i = tid; i < SY * SX; i += blockDim.x) {
            int r = i / SX, cc = i - r * SX;
            int gy = ty0 + r, gx = tx0 + cc;
            slab[i] = (gy < g.ey && gx < g.ex) ? Es[(size_t)gy * a.e_pitch + gx] : 0.f;
        }
        __syncthreads();
        // x pass
        for (int i = tid; i < SY * kConvTX; i += blockDim.x) {
            int r = i / kConvTX, cc = i - r * kConvTX;
            const float *s = slab + r * SX + cc;
            float acc = 0.f;
            for (int j = 0; j <= 2 * R; ++j) acc = fmaf(wxy[j], s[j], acc);
            xp[i] = acc;
        }
        __syncthreads();
        // y pass into the ring
        {
            const float *s = xp + ly * kConvTX + lx;
            float acc = 0.f;
            for (int j = 0; j <= 2 * R; ++j) acc = fmaf(wxy[j], s[j * kConvTX], acc);
            ring[(e % W) * (kConvTX * kConvTY) + tid] = acc;
        }
        __syncthreads();
        // z pass: output fine channel k = e - 2 Rz once its window is complete
        int k = e - 2 * Rz;
        if (k >= 0) {
            int ox = tx0 + lx, oy = ty0 + ly;
            float acc = 0.f;
            for (int j = 0; j < W; ++j) acc = fmaf(wz[j], ring[((k + j) % W) * (kConvTX * kConvTY) + tid], acc);
            if (ox < g.nxf && oy < g.nyf) F[(size_t)k * fplane + (size_t)oy * g.nxf + ox] = acc;
        }
        // the ring slot written next iteration was last read in this one
        __syncthreads();
    }
}

// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(256) downsample_kernel(StagedArgs a)
{
    const Geom &g = a.g;
    const long nd = (long)g.nx * g.ny * g.nz;
    const long total = nd * a.n_models;
    const int u = g.u;
    const float inv = 1.f / (float)(u * u * u);
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long)gridDim.x * blockDim.x) {
        long m = i / nd, r = i - m * nd;
        int k = (int)(r / ((long)g.nx * g.ny));
        int rr = (int)(r - (long)k * g.nx * g.ny);
        int j = rr / g.nx, x = rr - j * g.nx;
        const float *F = a.fine + (size_t)m * a.f_model_stride;
        float acc = 0.f;
        for (int c = 0; c < u; ++c)
            for (int b = 0; b < u; ++b) {
                const float *row = F + ((size_t)(k * u + c) * g.nyf + (j * u + b)) * g.nxf + x * u;
                for (int q = 0; q < u; ++q) acc += row[q];
            }
        a.data[(size_t)m * a.d_model_stride + r] = acc * inv;
    }
}

// ----------------------------------------------------------------------------
// Moments of the data cube, one thread per spaxel.  Sums are taken about the
// spaxel's own line-of-sight velocity clamped into the band, which keeps the
// FP32 second moment free of cancellation.
__device__ __forceinline__ void finish_moments(float s0, float s1, float s2, float cen,
                                               const ModelConst &c, float &m0, float &m1, float &m2,
                                               bool &valid)
{
    valid = s0 > kInvalidFraction * c.i0;
    if (!c.valid) {
        m0 = m1 = m2 = __int_as_float(0x7fc00000);
    } else if (valid) {
        float mu = s1 / s0;
        m0 = s0;
        m1 = cen + mu;
        m2 = sqrtf(fmaxf(fmaf(-mu, mu, s2 / s0), 0.f));
    } else {
        m0 = 0.f; m1 = c.vsys; m2 = 0.f;
    }
}

// Block sum of one FP32 value per thread: FP32 within each warp (a fixed
// shuffle tree), the warps in FP64 in order.  Result in thread 0.
__device__ __forceinline__ double block_sum_f32(float v, double *red)
{
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[warp] = (double)v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    return s;
}

__device__ __forceinline__ double block_sum(double v, double *red)
{
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    return s;  // valid on thread 0
}

__global__ void __launch_bounds__(256) moments_kernel(StagedArgs a)
{
    const Geom &g = a.g;
    const int np = g.nx * g.ny;
    const int bpm = (np + blockDim.x - 1) / blockDim.x;
    const int model = blockIdx.x / bpm;
    const int pix = (blockIdx.x - model * bpm) * blockDim.x + threadIdx.x;
    __shared__ ModelConst mc;
    __shared__ double red[32];
    if (threadIdx.x == 0) mc = model_const(a.params + (size_t)model * GBK_NPAR, g);
    __syncthreads();
    const ModelConst c = mc;
    float acc = 0.f;
    if (pix < np) {
        int y = pix / g.nx, x = pix - y * g.nx;
        float vl, br;
        los(c, (float)x, (float)y, vl, br);
        // centre: v_los clamped into the band (see the fused kernel)
        float cen = fminf(fmaxf(vl, g.vc - 0.5f * (float)(g.nz - 1) * g.dv), g.vc + 0.5f * (float)(g.nz - 1) * g.dv);
        const float *D = a.data + (size_t)model * a.d_model_stride + pix;
        float base = g.vc - 0.5f * (float)(g.nz - 1) * g.dv - cen;
        float s0 = 0.f, s1 = 0.f, s2 = 0.f;
        // eight channel loads in flight per step; the sums stay in channel order
        int k = 0;
        for (; k + 8 <= g.nz; k += 8) {
            float cv[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) cv[q] = D[(size_t)(k + q) * np];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const float d = fmaf((float)(k + q), g.dv, base);
                const float t = cv[q] * d;
                s0 += cv[q]; s1 += t; s2 = fmaf(t, d, s2);
            }
        }
        for (; k < g.nz; ++k) {
            float cv = D[(size_t)k * np];
            float d = fmaf((float)k, g.dv, base);
            float t = cv * d;
            s0 += cv; s1 += t; s2 = fmaf(t, d, s2);
        }
        float m0, m1, m2;
        bool valid;
        finish_moments(s0, s1, s2, cen, c, m0, m1, m2, valid);
        if (a.maps) {
            float *mp = a.maps + (size_t)model * 3 * np;
            mp[pix] = m0; mp[np + pix] = m1; mp[2 * np + pix] = m2;
        }
        if (a.chi2 || a.resid) {
            float rv = 0.f, rs = 0.f;
            if (a.obs.mask[pix] != 0 && (valid || !c.valid)) {
                rv = a.obs.w_v[pix] * (m1 - a.obs.v_obs[pix]);
                rs = a.obs.w_s[pix] * (m2 - a.obs.s_obs[pix]);
            }
            acc = rv * rv + rs * rs;
            if (a.resid) {
                float *rp = a.resid + (size_t)model * 2 * np;
                rp[pix] = rv; rp[np + pix] = rs;
            }
        }
    }
    if (a.chi2) {
        double s = block_sum_f32(acc, red);
        if (threadIdx.x == 0) a.partials[blockIdx.x] = c.valid ? s : (double)__int_as_float(0x7fc00000);
    }
}

__global__ void chi2_final_kernel(const double *partials, int bpm, int n_models, double *chi2)
{
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= n_models) return;
    double s = 0.0;
    for (int b = 0; b < bpm; ++b) s += partials[(size_t)m * bpm + b];
    chi2[m] = s;
}

// ----------------------------------------------------------------------------
// Eq. 11 from caller-supplied maps; one block per model, fixed-order sum.
__global__ void __launch_bounds__(512) chi2_maps_kernel(int np, const float *maps, gbk_obs obs,
                                                        double *chi2, float *resid)
{
    const int model = blockIdx.x;
    const float *mp = maps + (size_t)model * 3 * np;
    __shared__ double red[32];
    double acc = 0.0;
    for (int pix = threadIdx.x; pix < np; pix += blockDim.x) {
        float rv = 0.f, rs = 0.f;
        if (obs.mask[pix] != 0 && mp[pix] > 0.f) {
            rv = obs.w_v[pix] * (mp[np + pix] - obs.v_obs[pix]);
            rs = obs.w_s[pix] * (mp[2 * np + pix] - obs.s_obs[pix]);
        }
        acc += (double)(rv * rv) + (double)(rs * rs);
        if (resid) {
            resid[(size_t)model * 2 * np + pix] = rv;
            resid[(size_t)model * 2 * np + np + pix] = rs;
        }
    }
    double s = block_sum(acc, red);
    if (threadIdx.x == 0) chi2[model] = s;
}

// ----------------------------------------------------------------------------
size_t conv_smem_bytes(const Geom &g)
{
    int SX = kConvTX + 2 * g.R, SY = kConvTY + 2 * g.R, W = 2 * g.Rz + 1;
    return sizeof(float) * (size_t)((2 * g.R + 1) + W + SY * SX + SY * kConvTX + W * kConvTX * kConvTY);
}

gbk_status launch_staged(const StagedArgs &a, bool want_moments, cudaStream_t stream, cudaEvent_t *ev)
{
    const Geom &g = a.g;
    if (a.n_models == 0) return GBK_OK;
    cudaError_t e;
    auto mark = [&](int i) -> gbk_status {
        if (ev && (e = cudaEventRecord(ev[i], stream)) != cudaSuccess) return cuda_fail(e, "stage event");
        return GBK_OK;
    };
    gbk_status sm;
    if ((sm = mark(0))) return sm;
    {
        long per_model = (long)g.ey * (a.e_pitch / 4);
        long bpm = (per_model + 255) / 256;
        model_cube_kernel<<<(unsigned)(bpm * a.n_models), 256, 0, stream>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "model cube kernel launch");
    }
    if ((sm = mark(1))) return sm;
    if (conv_fir_supported(g)) {
        gbk_status s = launch_conv_fir(a, stream);
        if (s) return s;
    } else if (conv_tma_supported(g)) {
        gbk_status s = launch_conv_tma(a, stream);
        if (s) return s;
    } else {
        size_t smem = conv_smem_bytes(g);
        static KernelAttrMemo memo;
        if (smem > 48 * 1024) {
            gbk_status s = ensure_kernel_attrs((const void *)conv3d_kernel, smem, false, memo,
                                               "conv kernel: setting dynamic shared memory");
            if (s) return s;
        }
        int tiles = ((g.nxf + kConvTX - 1) / kConvTX) * ((g.nyf + kConvTY - 1) / kConvTY);
        conv3d_kernel<<<(unsigned)(tiles * a.n_models), kConvTX * kConvTY, smem, stream>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "conv kernel launch");
    }
    if ((sm = mark(2))) return sm;
    if (g.u > 1) {
        long total = (long)g.nx * g.ny * g.nz * a.n_models;
        long blocks = (total + 255) / 256;
        if (blocks > 152L * 64) blocks = 152L * 64;
        downsample_kernel<<<(unsigned)blocks, 256, 0, stream>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "down-sampling kernel launch");
    }
    if ((sm = mark(3))) return sm;
    if (want_moments) {
        int np = g.nx * g.ny;
        int bpm = (np + 255) / 256;
        moments_kernel<<<(unsigned)(bpm * a.n_models), 256, 0, stream>>>(a);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "moments kernel launch");
        if (a.chi2) {
            chi2_final_kernel<<<(a.n_models + 127) / 128, 128, 0, stream>>>(a.partials, bpm, a.n_models, a.chi2);
            if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "chi2 final kernel launch");
        }
    }
    return mark(4);
}

cudaError_t launch_chi2_maps(int nx, int ny, int n_models, const float *maps, const gbk_obs &obs,
                             double *chi2, float *resid, cudaStream_t stream)
{
    if (n_models == 0) return cudaSuccess;
    chi2_maps_kernel<<<(unsigned)n_models, 512, 0, stream>>>(nx * ny, maps, obs, chi2, resid);
    return cudaGetLastError();
}

}  // namespace gbk
