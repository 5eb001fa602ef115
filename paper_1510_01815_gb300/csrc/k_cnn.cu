// k_cnn.cu -- a convolutional network that maps a galaxy's observed velocity
// and dispersion maps (64 x 64) to the model parameters, used as the initial
// guess of the fits.  The paper starts its optimisers from a heuristic guess
// (Sec. 2.1.9); this learned guess replaces it.  Every dense operation runs
// on the tensor cores through the tcgen05 GEMM of k_gemm.cu.
//
// Network (all convolutions have stride = kernel size), 1.23 M parameters:
//   input  64 x 64 x 4   (v / 200 km/s, sigma / 100 km/s, mask, 0; masked -> 0)
//   conv   2 x 2 -> 32 x 32 x 32,  ReLU
//   conv   2 x 2 -> 16 x 16 x 64,  ReLU
//   conv   2 x 2 ->  8 x  8 x 128, ReLU
//   conv   2 x 2 ->  4 x  4 x 256, ReLU
//   dense  4096  -> 256, ReLU       (flatten index = morton(y, x) * 256 + c)
//   dense  256   -> 16              (outputs 0..9 are used, see targets)
// Weights W_l [C_l][K_l] with the patch index k = (dy * p + dx) * C_in + c.
//
// Layout trick: the rows of every activation matrix are ordered by the
// Morton (bit-interleaved) index of the pixel within its sample, so the p x p
// patches of the next layer are runs of consecutive rows and each patch
// matrix is a plain reshape of the previous layer's output -- no im2col pass.
// The weight gradients dW = dZ^T A contract over rows, so the forward and
// backward GEMM epilogues also write transposed copies; each transposed
// activation carries an extra row of ones so that the same GEMM yields the
// bias gradient as an extra column.  Long contractions are split over K into
// FP32 slices summed in a fixed order.
#include <cuda_bf16.h>

#include <cmath>

#include "gbk_api_internal.h"
#include "k_gemm.h"

namespace gbk {

constexpr int kCnnMap = 64;
constexpr int kCnnL = 6;
constexpr int kCnnC[kCnnL] = {32, 64, 128, 256, 256, 16};      // outputs per layer
constexpr int kCnnK[kCnnL] = {16, 128, 256, 512, 4096, 256};   // inputs per layer
constexpr int kCnnRows[kCnnL] = {1024, 256, 64, 16, 1, 1};     // matrix rows per sample
constexpr int kCnnIn = 4;                                      // input channels
constexpr int kCnnOut = 16, kCnnTargets = 10;
constexpr float kVScale = 200.f, kSScale = 100.f;
constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;

// ---------------------------------------------------------------------------
// parameter layout: layer l is P_l [C_l][K_l + 1] (weights, then the bias)
static size_t param_offset(int l)
{
    size_t o = 0;
    for (int i = 0; i < l; ++i) o += (size_t)kCnnC[i] * (kCnnK[i] + 1);
    return o;
}
static size_t param_count() { return param_offset(kCnnL); }

struct CnnTables {
    int C[kCnnL], K[kCnnL];
    size_t off[kCnnL + 1];
    __nv_bfloat16 *W[kCnnL], *WT[kCnnL];
    float *bias[kCnnL];
};

__device__ __forceinline__ uint64_t sm_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Normal number i of a stream: outputs 2i+1 and 2i+2 of SplitMix64 seeded
// with `seed` (the k-th output is mix(seed + k * golden)), Box-Muller cosine
// branch, u1 in (0, 1].
__device__ __forceinline__ double sm_normal(uint64_t seed, uint64_t i)
{
    uint64_t z1 = sm_mix(seed + (2 * i + 1) * kGolden), z2 = sm_mix(seed + (2 * i + 2) * kGolden);
    double u1 = (double)((z1 >> 11) + 1) * (1.0 / 9007199254740992.0);
    double u2 = (double)(z2 >> 11) * (1.0 / 9007199254740992.0);
    return sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
}

__device__ __forceinline__ double sm_uniform(uint64_t seed, uint64_t i)
{
    return (double)(sm_mix(seed + (i + 1) * kGolden) >> 11) * (1.0 / 9007199254740992.0);
}

// Morton index of (y, x) with `bits` bits per coordinate: x bit i -> bit 2i,
// y bit i -> bit 2i + 1.
__host__ __device__ __forceinline__ int morton(int y, int x, int bits)
{
    int q = 0;
    for (int i = 0; i < bits; ++i) q |= (((x >> i) & 1) << (2 * i)) | (((y >> i) & 1) << (2 * i + 1));
    return q;
}

// He-normal weights (std sqrt(2 / K), the last layer sqrt(1 / K)), zero biases.
__global__ void cnn_init_kernel(float *P, CnnTables t, uint64_t seed)
{
    const size_t n = t.off[kCnnL];
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        int l = 0;
        while (i >= t.off[l + 1]) ++l;
        const size_t j = i - t.off[l];
        const int k = (int)(j % (size_t)(t.K[l] + 1));
        if (k == t.K[l]) {
            P[i] = 0.f;
        } else {
            double sd = sqrt((l == kCnnL - 1 ? 1.0 : 2.0) / t.K[l]);
            P[i] = (float)(sd * sm_normal(seed, i));
        }
    }
}

// BF16 copies of the weights (row-major and transposed) and FP32 biases.
__global__ void cnn_publish_kernel(const float *P, CnnTables t)
{
    const size_t n = t.off[kCnnL];
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        int l = 0;
        while (i >= t.off[l + 1]) ++l;
        const size_t j = i - t.off[l];
        const int K = t.K[l], C = t.C[l];
        const int o = (int)(j / (size_t)(K + 1)), k = (int)(j % (size_t)(K + 1));
        const float v = P[i];
        if (k == K) {
            t.bias[l][o] = v;
        } else {
            const __nv_bfloat16 h = __float2bfloat16_rn(v);
            t.W[l][(size_t)o * K + k] = h;
            t.WT[l][(size_t)k * C + o] = h;
        }
    }
}

// Input encoding: sample b, 2 x 2 patch (Y, X) -> row b * 1024 + morton(Y, X);
// column (dy * 2 + dx) * 4 + ch.  Also the transposed matrix with a row of
// ones at index 16.  One thread per patch: two 8-byte loads each of v and
// sigma and two 2-byte mask loads, one 32-byte row store, and 17 transposed
// stores that are coalesced across the warp (consecutive threads, consecutive
// rows).
__global__ void cnn_encode_kernel(int n, const float *v, const float *s, const uint8_t *mask, __nv_bfloat16 *A,
                                  __nv_bfloat16 *AT)
{
    constexpr int kRows = kCnnRows[0], kK = kCnnK[0];
    const size_t rows = (size_t)n * kRows;
    for (size_t r = blockIdx.x * (size_t)blockDim.x + threadIdx.x; r < rows; r += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(r / kRows), q = (int)(r % kRows);
        int Y = 0, X = 0;
        for (int k = 0; k < 5; ++k) {
            X |= ((q >> (2 * k)) & 1) << k;
            Y |= ((q >> (2 * k + 1)) & 1) << k;
        }
        __align__(16) __nv_bfloat16 h[kK];
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
            const size_t pix = (size_t)b * kCnnMap * kCnnMap + (size_t)(2 * Y + dy) * kCnnMap + 2 * X;
            const float2 vv = *reinterpret_cast<const float2 *>(v + pix);
            const float2 ss = *reinterpret_cast<const float2 *>(s + pix);
            const uchar2 mm = *reinterpret_cast<const uchar2 *>(mask + pix);
            const float vx[2] = {vv.x, vv.y}, sx[2] = {ss.x, ss.y};
            const unsigned char mx[2] = {mm.x, mm.y};
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
                const bool on = mx[dx] != 0;
                const int e = (dy * 2 + dx) * kCnnIn;
                h[e] = __float2bfloat16_rn(on ? vx[dx] / kVScale : 0.f);
                h[e + 1] = __float2bfloat16_rn(on ? sx[dx] / kSScale : 0.f);
                h[e + 2] = __float2bfloat16_rn(on ? 1.f : 0.f);
                h[e + 3] = __float2bfloat16_rn(0.f);
            }
        }
        uint4 *dst = reinterpret_cast<uint4 *>(A + r * kK);
        const uint4 *src = reinterpret_cast<const uint4 *>(h);
        dst[0] = src[0];
        dst[1] = src[1];
#pragma unroll
        for (int e = 0; e < kK; ++e) AT[(size_t)e * rows + r] = h[e];
        AT[(size_t)kK * rows + r] = __float2bfloat16_rn(1.f);
    }
}

__global__ void cnn_ones_kernel(__nv_bfloat16 *row, size_t n)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        row[i] = __float2bfloat16_rn(1.f);
}

// Loss = mean over samples and the 10 used outputs of (y - t)^2; dY = dL/dy
// (BF16, plain and transposed).  One block; fixed-order reduction.
__global__ void cnn_loss_kernel(const float *Y, const float *T, int B, __nv_bfloat16 *dY, __nv_bfloat16 *dYT,
                                float *loss)
{
    __shared__ double red[32];
    double acc = 0.0;
    const float g = 2.f / (float)(B * kCnnTargets);
    for (int i = threadIdx.x; i < B * kCnnOut; i += blockDim.x) {
        const int b = i / kCnnOut, j = i % kCnnOut;
        float d = 0.f;
        if (j < kCnnTargets) {
            d = Y[(size_t)b * kCnnOut + j] - T[(size_t)b * kCnnTargets + j];
            acc += (double)d * d;
        }
        const __nv_bfloat16 h = __float2bfloat16_rn(g * d);
        dY[(size_t)b * kCnnOut + j] = h;
        dYT[(size_t)j * B + b] = h;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        if (loss) *loss = (float)(s / (double)(B * kCnnTargets));
    }
}

__global__ void cnn_adam_kernel(float *P, float *Mo, float *Vo, const float *G, size_t n, float lr, float b1, float b2,
                                float eps, float bc1, float bc2)
{
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float g = G[i];
        const float m = b1 * Mo[i] + (1.f - b1) * g;
        const float v = b2 * Vo[i] + (1.f - b2) * g * g;
        Mo[i] = m;
        Vo[i] = v;
        P[i] -= lr * (m / bc1) / (sqrtf(v / bc2) + eps);
    }
}

// Targets (the network's outputs 0..9) from parameter vectors, and back.
//  t0 = (x0 - 31.5) / 8, t1 = (y0 - 31.5) / 8, t2 = cos PA, t3 = sin PA,
//  t4 = (i - 50) / 20, t5 = Vsys / 30, t6 = (Vmax - 175) / 75,
//  t7 = (r_t - 4.5) / 2.5, t8 = (sigma0 - 45) / 25, t9 = (h - 7) / 3.
// I0 cannot be recovered from v and sigma maps; decoding sets it to 1.
__global__ void cnn_targets_kernel(int n, const double *p, float *t)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    const double *q = p + (size_t)b * GBK_NPAR;
    float *o = t + (size_t)b * kCnnTargets;
    const double pa = q[GBK_PA] * (M_PI / 180.0);
    o[0] = (float)((q[GBK_X0] - 31.5) / 8.0);
    o[1] = (float)((q[GBK_Y0] - 31.5) / 8.0);
    o[2] = (float)cos(pa);
    o[3] = (float)sin(pa);
    o[4] = (float)((q[GBK_INCL] - 50.0) / 20.0);
    o[5] = (float)(q[GBK_VSYS] / 30.0);
    o[6] = (float)((q[GBK_VMAX] - 175.0) / 75.0);
    o[7] = (float)((q[GBK_RT] - 4.5) / 2.5);
    o[8] = (float)((q[GBK_SIG0] - 45.0) / 25.0);
    o[9] = (float)((q[GBK_H] - 7.0) / 3.0);
}

__global__ void cnn_decode_kernel(int n, const float *y, double *p)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n) return;
    const float *o = y + (size_t)b * kCnnOut;
    double *q = p + (size_t)b * GBK_NPAR;
    q[GBK_X0] = 31.5 + 8.0 * o[0];
    q[GBK_Y0] = 31.5 + 8.0 * o[1];
    double pa = atan2((double)o[3], (double)o[2]) * (180.0 / M_PI);
    q[GBK_PA] = pa < 0.0 ? pa + 360.0 : pa;
    q[GBK_INCL] = 50.0 + 20.0 * o[4];
    q[GBK_VSYS] = 30.0 * o[5];
    q[GBK_VMAX] = 175.0 + 75.0 * o[6];
    q[GBK_RT] = 4.5 + 2.5 * o[7];
    q[GBK_SIG0] = 45.0 + 25.0 * o[8];
    q[GBK_I0] = 1.0;
    q[GBK_H] = 7.0 + 3.0 * o[9];
}

// Observed maps from model maps [n][3][64][64]: v = m1 + N(0, noise_v),
// sigma = m2 + N(0, sqrt(2) noise_v) (normal streams 2 idx and 2 idx + 1),
// mask = 0 with probability dead_frac (uniform stream of seed ^ 0xD1B54A32D192ED03)
// or where the model spectrum is invalid (m0 == 0).
__global__ void cnn_synth_obs_kernel(int n, const float *maps, uint64_t seed, float noise_v, float dead_frac, float *v,
                                     float *s, uint8_t *mask)
{
    const size_t np = (size_t)kCnnMap * kCnnMap, total = (size_t)n * np;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t b = i / np, pix = i % np;
        const float *m = maps + b * 3 * np;
        v[i] = m[np + pix] + (float)(noise_v * sm_normal(seed, 2 * i));
        s[i] = m[2 * np + pix] + (float)(1.4142135623730951 * noise_v * sm_normal(seed, 2 * i + 1));
        const bool dead = sm_uniform(seed ^ 0xD1B54A32D192ED03ull, i) < (double)dead_frac;
        mask[i] = (dead || !(m[pix] > 0.f)) ? 0 : 1;
    }
}

// ---------------------------------------------------------------------------
static size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

struct CnnWs {
    __nv_bfloat16 *A[kCnnL];    // A_l [M_l][K_l]; A_{l+1} is H_l
    __nv_bfloat16 *AT[kCnnL];   // [K_l + 1][M_l], last row ones
    float *Y;                   // [B][16]
    __nv_bfloat16 *dY, *dYT;    // [B][16], [16][B]
    __nv_bfloat16 *dZ[kCnnL];   // dZ_l (l < L - 1) stored in A_{l+1}'s layout
    __nv_bfloat16 *dZT[kCnnL];  // [C_l][M_l]
    float *G;                   // gradient, parameter layout
    float *part;                // split-K slices
    size_t part_floats;
    float *loss;
    CnnTables t;
    size_t total;
};

static int split_of(int l, int B, int *kt_split)
{
    const int M = kCnnC[l], N = kCnnK[l] + 1, Kc = B * kCnnRows[l];
    const int bn = N >= 256 ? 256 : (N >= 128 ? 128 : ((N + 15) / 16) * 16);
    const int tiles = ((M + 127) / 128) * ((N + bn - 1) / bn);
    const int KT = (Kc + 63) / 64;
    int splits = (2 * 152 + tiles - 1) / tiles;
    if (splits > 128) splits = 128;  // bounds the slices the reduction reads
    if (splits > KT) splits = KT;
    if (splits < 1) splits = 1;
    *kt_split = (KT + splits - 1) / splits;
    return (KT + *kt_split - 1) / *kt_split;
}

static CnnWs cnn_layout(int B, char *base)
{
    CnnWs w = {};
    size_t o = 0;
    auto take = [&](size_t bytes) { char *p = base ? base + o : nullptr; o += al256(bytes); return p; };
    const size_t bf = sizeof(__nv_bfloat16);
    for (int l = 0; l < kCnnL; ++l) {
        const size_t M = (size_t)B * kCnnRows[l];
        w.A[l] = (__nv_bfloat16 *)take(bf * M * kCnnK[l]);
        w.AT[l] = (__nv_bfloat16 *)take(bf * (kCnnK[l] + 1) * M);
        w.dZT[l] = (__nv_bfloat16 *)take(bf * kCnnC[l] * M);
        if (l < kCnnL - 1) w.dZ[l] = (__nv_bfloat16 *)take(bf * M * kCnnC[l]);
    }
    w.Y = (float *)take(sizeof(float) * B * kCnnOut);
    w.dY = (__nv_bfloat16 *)take(bf * B * kCnnOut);
    w.dYT = (__nv_bfloat16 *)take(bf * B * kCnnOut);
    w.G = (float *)take(sizeof(float) * param_count());
    w.part_floats = 0;
    for (int l = 0; l < kCnnL; ++l) {
        int kts;
        const int sp = split_of(l, B, &kts);
        const size_t need = (size_t)sp * kCnnC[l] * (kCnnK[l] + 1);
        if (need > w.part_floats) w.part_floats = need;
    }
    w.part = (float *)take(sizeof(float) * w.part_floats);
    w.loss = (float *)take(sizeof(float));
    for (int l = 0; l < kCnnL; ++l) {
        w.t.C[l] = kCnnC[l];
        w.t.K[l] = kCnnK[l];
        w.t.off[l] = param_offset(l);
        w.t.W[l] = (__nv_bfloat16 *)take(bf * kCnnC[l] * kCnnK[l]);
        w.t.WT[l] = (__nv_bfloat16 *)take(bf * kCnnC[l] * kCnnK[l]);
        w.t.bias[l] = (float *)take(sizeof(float) * kCnnC[l]);
    }
    w.t.off[kCnnL] = param_count();
    w.total = o;
    return w;
}

static int grid_for(size_t n) { return (int)std::min<size_t>((n + 255) / 256, 152 * 16); }

static gbk_status gemm(const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, int ldb, GemmArgs a, cudaStream_t st)
{
    if (a.alpha == 0.f) a.alpha = 1.f;
    return launch_gemm_bf16(A, lda, B, ldb, a, st);
}

static int ilog2(int v)
{
    int r = 0;
    while ((1 << r) < v) ++r;
    return r;
}

// Forward pass of B encoded samples (w.A[0], w.AT[0] filled); logits in w.Y.
static gbk_status cnn_forward_ws(const CnnWs &w, int B, bool want_transposed, cudaStream_t st)
{
    gbk_status s;
    for (int l = 0; l < kCnnL; ++l) {
        GemmArgs a = {};
        a.M = B * kCnnRows[l];
        a.N = kCnnC[l];
        a.K = kCnnK[l];
        a.alpha = 1.f;
        a.bias = w.t.bias[l];
        if (l < kCnnL - 1) {
            a.relu = 1;
            a.out_bf16 = w.A[l + 1];
            a.ldo = kCnnC[l];
            if (want_transposed) {
                const int q = kCnnK[l + 1] / kCnnC[l];
                a.out_t = w.AT[l + 1];
                a.ldt = B * kCnnRows[l + 1];
                a.t_mode = 1;
                a.t_log2 = ilog2(q);
            }
        } else {
            a.out_f32 = w.Y;
            a.ldo = kCnnOut;
        }
        if ((s = gemm(w.A[l], kCnnK[l], w.t.W[l], kCnnK[l], a, st))) return s;
    }
    return GBK_OK;
}

static gbk_status cnn_encode(const CnnWs &w, int B, const float *v, const float *sg, const uint8_t *mask,
                             cudaStream_t st)
{
    cnn_encode_kernel<<<grid_for((size_t)B * kCnnRows[0]), 256, 0, st>>>(B, v, sg, mask, w.A[0], w.AT[0]);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "CNN encode launch");
    return GBK_OK;
}

// Forward + backward: gradient of the loss in w.G, loss in w.loss.
static gbk_status cnn_grad_ws(const CnnWs &w, const float *P, int B, const float *v, const float *sg,
                              const uint8_t *mask, const float *T, cudaStream_t st)
{
    gbk_status s;
    const size_t np = param_count();
    cnn_publish_kernel<<<grid_for(np), 256, 0, st>>>(P, w.t);
    for (int l = 1; l < kCnnL; ++l) {
        const size_t M = (size_t)B * kCnnRows[l];
        cnn_ones_kernel<<<grid_for(M), 256, 0, st>>>(w.AT[l] + (size_t)kCnnK[l] * M, M);
    }
    if ((s = cnn_encode(w, B, v, sg, mask, st))) return s;
    if ((s = cnn_forward_ws(w, B, true, st))) return s;
    cnn_loss_kernel<<<1, 1024, 0, st>>>(w.Y, T, B, w.dY, w.dYT, w.loss);
    for (int l = kCnnL - 1; l >= 0; --l) {
        const int M = B * kCnnRows[l], C = kCnnC[l], K = kCnnK[l];
        const __nv_bfloat16 *dZ = (l == kCnnL - 1) ? w.dY : w.dZ[l];
        const __nv_bfloat16 *dZT = (l == kCnnL - 1) ? w.dYT : w.dZT[l];
        // dW_l (and db_l as column K) = dZ_l^T [A_l | 1]
        GemmArgs g = {};
        g.M = C;
        g.N = K + 1;
        g.K = M;
        g.alpha = 1.f;
        g.out_f32 = w.part;
        g.ldo = K + 1;
        int kts;
        const int splits = split_of(l, B, &kts);
        g.kt_split = kts;
        g.split_stride = (size_t)C * (K + 1);
        if ((s = gemm(dZT, M, w.AT[l], M, g, st))) return s;
        if ((s = launch_splitk_reduce(w.part, splits, g.split_stride, C, K + 1, K + 1, w.G + param_offset(l), st)))
            return s;
        if (l == 0) break;
        // dZ_{l-1} = (dZ_l W_l) * [A_l > 0], in A_l's layout, plus its transpose
        GemmArgs d = {};
        d.M = M;
        d.N = K;
        d.K = C;
        d.alpha = 1.f;
        d.mask = w.A[l];
        d.ldm = K;
        d.out_bf16 = w.dZ[l - 1];
        d.ldo = K;
        d.out_t = w.dZT[l - 1];
        d.ldt = B * kCnnRows[l - 1];
        d.t_mode = 2;
        d.t_log2 = ilog2(kCnnC[l - 1]);
        const int lda = (l == kCnnL - 1) ? kCnnOut : C;
        if ((s = gemm(dZ, lda, w.t.WT[l], C, d, st))) return s;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "CNN gradient launches");
    return GBK_OK;
}

static gbk_status check_batch(int B)
{
    if (B < 8 || B % 8 != 0) return fail(GBK_EINVAL, "batch must be a positive multiple of 8 (got %d)", B);
    // every activation matrix (and its transpose) stays below 2^31 elements
    for (int l = 0; l < kCnnL; ++l)
        if ((size_t)B * kCnnRows[l] * (kCnnK[l] + 1) >= (size_t)1 << 31 ||
            (size_t)B * kCnnRows[l] * kCnnC[l] >= (size_t)1 << 31)
            return fail(GBK_EINVAL, "batch too large");
    return GBK_OK;
}

}  // namespace gbk

using namespace gbk;

extern "C" {

size_t gbk_cnn_param_count(void) { return param_count(); }

size_t gbk_cnn_workspace_bytes(int32_t batch)
{
    ok();
    if (check_batch(batch)) return 0;
    return cnn_layout(batch, nullptr).total;
}

gbk_status gbk_cnn_init(float *params, uint64_t seed, void *stream)
{
    gbk_status s = check_device_ptr(params, "params", 4);
    if (s) return s;
    CnnWs w = cnn_layout(8, nullptr);
    cnn_init_kernel<<<grid_for(param_count()), 256, 0, (cudaStream_t)stream>>>(params, w.t, seed);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "CNN init launch");
    return ok();
}

gbk_status gbk_cnn_targets(int32_t n, const double *params, float *targets, void *stream)
{
    if (n < 0) return fail(GBK_EINVAL, "n must be >= 0");
    if (n == 0) return ok();
    gbk_status s;
    if ((s = check_device_ptr(params, "params", 8)) || (s = check_device_ptr(targets, "targets", 4))) return s;
    cnn_targets_kernel<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(n, params, targets);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "CNN targets launch");
    return ok();
}

gbk_status gbk_cnn_decode(int32_t n, const float *out, double *params, void *stream)
{
    if (n < 0) return fail(GBK_EINVAL, "n must be >= 0");
    if (n == 0) return ok();
    gbk_status s;
    if ((s = check_device_ptr(out, "out", 4)) || (s = check_device_ptr(params, "params", 8))) return s;
    cnn_decode_kernel<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(n, out, params);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "CNN decode launch");
    return ok();
}

gbk_status gbk_cnn_synth_obs(int32_t n, const float *maps, uint64_t seed, float noise_v, float dead_frac, float *v,
                             float *sigma, uint8_t *mask, void *stream)
{
    if (n < 0) return fail(GBK_EINVAL, "n must be >= 0");
    if (n == 0) return ok();
    if (!(noise_v >= 0.f) || !(dead_frac >= 0.f && dead_frac <= 1.f))
        return fail(GBK_EINVAL, "noise_v must be >= 0 and dead_frac in [0, 1]");
    gbk_status s;
    if ((s = check_device_ptr(maps, "maps", 4)) || (s = check_device_ptr(v, "v", 4)) ||
        (s = check_device_ptr(sigma, "sigma", 4)) || (s = check_device_ptr(mask, "mask", 1)))
        return s;
    cnn_synth_obs_kernel<<<grid_for((size_t)n * kCnnMap * kCnnMap), 256, 0, (cudaStream_t)stream>>>(
        n, maps, seed, noise_v, dead_frac, v, sigma, mask);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "CNN observation synthesis launch");
    return ok();
}

// The encoding reads 2-pixel runs as 8-byte (maps) and 2-byte (mask) vectors;
// the contract asks for 16- and 4-byte alignment.
static gbk_status check_maps_in(const float *v, const float *sg, const uint8_t *mask)
{
    gbk_status s;
    if ((s = check_device_ptr(v, "v", 16)) || (s = check_device_ptr(sg, "sigma", 16)) ||
        (s = check_device_ptr(mask, "mask", 4)))
        return s;
    return GBK_OK;
}

gbk_status gbk_cnn_forward(const float *params, int32_t n, const float *v, const float *sigma, const uint8_t *mask,
                           float *out, void *workspace, size_t ws_bytes, void *stream)
{
    gbk_status s;
    if ((s = check_batch(n))) return s;
    if ((s = check_device_ptr(params, "params", 4)) || (s = check_maps_in(v, sigma, mask)) ||
        (s = check_device_ptr(out, "out", 4)))
        return s;
    CnnWs w = cnn_layout(n, nullptr);
    if (!workspace || ws_bytes < w.total)
        return fail(GBK_EWORKSPACE, "gbk_cnn_forward needs %zu bytes of workspace (got %zu)", w.total, ws_bytes);
    if ((s = check_device_ptr(workspace, "workspace", 256))) return s;
    w = cnn_layout(n, (char *)workspace);
    cudaStream_t st = (cudaStream_t)stream;
    cnn_publish_kernel<<<grid_for(param_count()), 256, 0, st>>>(params, w.t);
    if ((s = cnn_encode(w, n, v, sigma, mask, st))) return s;
    if ((s = cnn_forward_ws(w, n, false, st))) return s;
    cudaError_t e = cudaMemcpyAsync(out, w.Y, sizeof(float) * n * kCnnOut, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "CNN output copy");
    return ok();
}

gbk_status gbk_cnn_grad(const float *params, int32_t B, const float *v, const float *sigma, const uint8_t *mask,
                        const float *targets, float *grad, float *loss, void *workspace, size_t ws_bytes, void *stream)
{
    gbk_status s;
    if ((s = check_batch(B))) return s;
    if ((s = check_device_ptr(params, "params", 4)) || (s = check_maps_in(v, sigma, mask)) ||
        (s = check_device_ptr(targets, "targets", 4)))
        return s;
    if (grad && (s = check_device_ptr(grad, "grad", 4))) return s;
    if (loss && (s = check_device_ptr(loss, "loss", 4))) return s;
    CnnWs w = cnn_layout(B, nullptr);
    if (!workspace || ws_bytes < w.total)
        return fail(GBK_EWORKSPACE, "gbk_cnn_grad needs %zu bytes of workspace (got %zu)", w.total, ws_bytes);
    if ((s = check_device_ptr(workspace, "workspace", 256))) return s;
    w = cnn_layout(B, (char *)workspace);
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = cnn_grad_ws(w, params, B, v, sigma, mask, targets, st))) return s;
    cudaError_t e = cudaSuccess;
    if (grad) e = cudaMemcpyAsync(grad, w.G, sizeof(float) * param_count(), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && loss) e = cudaMemcpyAsync(loss, w.loss, sizeof(float), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "CNN gradient copy");
    return ok();
}

gbk_status gbk_cnn_train_step(float *params, float *adam_m, float *adam_v, int32_t step, float lr, int32_t B,
                              const float *v, const float *sigma, const uint8_t *mask, const float *targets,
                              float *loss, void *workspace, size_t ws_bytes, void *stream)
{
    gbk_status s;
    if (step < 1) return fail(GBK_EINVAL, "step counts from 1");
    if (!(lr >= 0.f)) return fail(GBK_EINVAL, "lr must be >= 0");
    if ((s = check_device_ptr(adam_m, "adam_m", 4)) || (s = check_device_ptr(adam_v, "adam_v", 4))) return s;
    if ((s = gbk_cnn_grad(params, B, v, sigma, mask, targets, nullptr, loss, workspace, ws_bytes, stream))) return s;
    CnnWs w = cnn_layout(B, (char *)workspace);
    const float b1 = 0.9f, b2 = 0.999f;
    const float bc1 = 1.f - powf(b1, (float)step), bc2 = 1.f - powf(b2, (float)step);
    cnn_adam_kernel<<<grid_for(param_count()), 256, 0, (cudaStream_t)stream>>>(params, adam_m, adam_v, w.G,
                                                                              param_count(), lr, b1, b2, 1e-8f, bc1,
                                                                              bc2);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "CNN Adam launch");
    return ok();
}

}  // extern "C"
