// residual.cu -- the QFCA+ features (arXiv 2510.15602, Sec. 3.3): the input
// features minus their PCA reconstruction from the top dres components,
//     F = (X - mean) - (X - mean) V V^T,
// for all C channels, with each channel's image-wide min/max (order-preserving
// u32 keys) for the per-channel quantisation that follows.
//
// k_residual: one thread per pixel.  The thread forms the dres projections
// y_k = sum_c (x_c - mean_c) V_ck in FP32 registers (mean and V staged in
// shared memory as FP32), then walks the channels again (the CTA's pixels are
// still in L2) to write f_c = (x_c - mean_c) - sum_k V_ck y_k.  Per channel,
// a warp reduces the keys with one hardware min and one max reduction, lane 0
// folds them into the CTA's shared-memory keys, and the CTA adds its C minima
// and maxima to the image's keys once.  The work is 4 C dres flops per pixel;
// the traffic, X read once from HBM and F written once, bounds it.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.cuh"

namespace qfca {
namespace {

constexpr int kResThreads = 256;

struct ResP {
    const float *X;
    int layout, H, W, C, dres;
    const double *mean, *V;  // [C], [C][dres]
    float *F;                // [C][N]
    uint32_t *mm;            // keys: min of channel c at c*kKeyStride, max at (C+c)*kKeyStride
};

__global__ void __launch_bounds__(kResThreads) k_residual(const __grid_constant__ ResP p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int C = p.C, dr = p.dres;
    float *mu = reinterpret_cast<float *>(smem_raw);   // [C]
    float *Vs = mu + C;                                 // [C][dres]
    uint32_t *mn = reinterpret_cast<uint32_t *>(Vs + (size_t)C * dr);  // [C]
    uint32_t *mx = mn + C;                              // [C]
    for (int c = threadIdx.x; c < C; c += kResThreads) {
        mu[c] = (float)p.mean[c];
        mn[c] = 0xffffffffu;
        mx[c] = 0u;
    }
    for (int e = threadIdx.x; e < C * dr; e += kResThreads) Vs[e] = (float)p.V[e];
    __syncthreads();
    const long N = (long)p.H * p.W;
    const long px = (long)blockIdx.x * kResThreads + threadIdx.x;
    const bool ok = px < N;
    const long q = ok ? px : 0;
    auto xval = [&](int c) -> float {
        return p.layout == 0 ? p.X[(size_t)c * N + q] : p.X[(size_t)q * C + c];
    };
    float y[kMaxResidual];
#pragma unroll
    for (int k = 0; k < kMaxResidual; k++) y[k] = 0.0f;
    // eight channels' loads in flight at a time (few warps per SM: latency, not bandwidth, is the limit)
    int c = 0;
    for (; c + 8 <= C; c += 8) {
        float xs[8];
#pragma unroll
        for (int u = 0; u < 8; u++) xs[u] = xval(c + u);
#pragma unroll
        for (int u = 0; u < 8; u++) {
            const float xc = xs[u] - mu[c + u];
            const float *v = Vs + (size_t)(c + u) * dr;
#pragma unroll
            for (int k = 0; k < kMaxResidual; k++)
                if (k < dr) y[k] = fmaf(xc, v[k], y[k]);
        }
    }
    for (; c < C; c++) {
        const float xc = xval(c) - mu[c];
        const float *v = Vs + (size_t)c * dr;
#pragma unroll
        for (int k = 0; k < kMaxResidual; k++)
            if (k < dr) y[k] = fmaf(xc, v[k], y[k]);
    }
    const int lane = threadIdx.x & 31;
    auto emit = [&](int cc, float xv) {
        float f = xv - mu[cc];
        const float *v = Vs + (size_t)cc * dr;
#pragma unroll
        for (int k = 0; k < kMaxResidual; k++)
            if (k < dr) f = fmaf(-v[k], y[k], f);
        const uint32_t key = f2key(f);
        if (ok) p.F[(size_t)cc * N + px] = f;
        const uint32_t kmin = __reduce_min_sync(0xffffffffu, ok ? key : 0xffffffffu);
        const uint32_t kmax = __reduce_max_sync(0xffffffffu, ok ? key : 0u);
        if (lane == 0) {
            atomicMin(&mn[cc], kmin);
            atomicMax(&mx[cc], kmax);
        }
    };
    c = 0;
    for (; c + 8 <= C; c += 8) {
        float xs[8];
#pragma unroll
        for (int u = 0; u < 8; u++) xs[u] = xval(c + u);
#pragma unroll
        for (int u = 0; u < 8; u++) emit(c + u, xs[u]);
    }
    for (; c < C; c++) emit(c, xval(c));
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += kResThreads) {
        atomicMin(&p.mm[(size_t)c * kKeyStride], mn[c]);
        atomicMax(&p.mm[(size_t)(C + c) * kKeyStride], mx[c]);
    }
}

int g_attr_dev_res = -1;

}  // namespace

size_t residual_smem(int C, int dres) { return sizeof(float) * ((size_t)C + (size_t)C * dres) + 2 * sizeof(uint32_t) * C; }

cudaError_t launch_residual(const float *X, int layout, int H, int W, int C, const double *mean, const double *V,
                            int dres, float *F, uint32_t *mm, cudaStream_t st) {
    if (dres < 0 || dres > kMaxResidual) return cudaErrorInvalidValue;
    int dev = 0;
    cudaGetDevice(&dev);
    if (g_attr_dev_res != dev) {
        cudaFuncSetAttribute(k_residual, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        g_attr_dev_res = dev;
    }
    cudaError_t e = launch_init_keys(mm, C, 1, st);
    if (e != cudaSuccess) return e;
    ResP p{X, layout, H, W, C, dres, mean, V, F, mm};
    const long N = (long)H * W;
    const unsigned grid = (unsigned)((N + kResThreads - 1) / kResThreads);
    QFCA_LAUNCH("k_residual", st, (k_residual<<<grid, kResThreads, residual_smem(C, dres), st>>>(p)));
    return cudaGetLastError();
}

}  // namespace qfca
