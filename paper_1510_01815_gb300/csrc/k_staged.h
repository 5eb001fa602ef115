// k_staged.h -- launchers of the staged (cube-materialising) kernels.
#pragma once

#include "gbk_internal.cuh"

namespace gbk {

constexpr int kConvTX = 32;
constexpr int kConvTY = 8;

struct StagedArgs {
    Geom g;
    int n_models;
    const double *params;    // [n][GBK_NPAR]
    float *ext;              // fine extended model cube, [n][ez][ey][e_pitch]
    int e_pitch;             // row pitch of ext in floats (multiple of 4, >= ex)
    size_t e_model_stride;   // floats per model in ext
    float *fine;             // convolved fine cube [n][nzf][nyf][nxf]
    size_t f_model_stride;
    float *data;             // data-resolution cube [n][nz][ny][nx] (== fine when u == 1)
    size_t d_model_stride;
    float *maps;             // [n][3][ny][nx] or null
    double *chi2;            // [n] or null
    float *resid;            // [n][2][ny][nx] or null
    double *partials;        // [n][ceil(nx*ny/256)] when chi2 is set
    gbk_obs obs;
};

size_t conv_smem_bytes(const Geom &g);
bool conv_tma_supported(const Geom &g);
gbk_status launch_conv_tma(const StagedArgs &a, cudaStream_t stream);
// ev (optional): five events recorded at the stage boundaries -- before the
// model cube, after it, after the convolution, after the down-sampling and
// after the moments and chi2.
gbk_status launch_staged(const StagedArgs &a, bool want_moments, cudaStream_t stream,
                         cudaEvent_t *ev = nullptr);
cudaError_t launch_chi2_maps(int nx, int ny, int n_models, const float *maps, const gbk_obs &obs,
                             double *chi2, float *resid, cudaStream_t stream);

gbk_status conv_status_read(int *v);
// Register-FIR convolution for PSF and LSF radii up to 8 (k_conv_fir.cu).
bool conv_fir_supported(const Geom &g);
gbk_status launch_conv_fir(const StagedArgs &a, cudaStream_t stream);
gbk_status conv_fir_status_read(int *v);

}  // namespace gbk
