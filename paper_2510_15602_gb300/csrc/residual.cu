// residual.cu -- the QFCA+ features (arXiv 2510.15602, Sec. 3.3): the input
// features minus their PCA reconstruction from the top dres components,
//     F = (X - mean) - (X - mean) V V^T,
// for all C channels, with each channel's image-wide min/max (order-preserving
// u32 keys) for the per-channel quantisation that follows.
//
// k_residual: one thread per pixel (or four adjacent pixels, one 16-byte load
// per channel, when the layout allows).  The thread forms the dres projections
// y_k = sum_c (x_c - mean_c) V_ck in FP32 registers (mean and V staged in
// shared memory as FP32), then walks the channels again to write
// f_c = (x_c - mean_c) - sum_k V_ck y_k; on a 1 GB batch the second walk misses
// L2 (measured: the features are read twice from DRAM).  Per channel,
// a warp reduces the keys with one hardware min and one max reduction, lane 0
// folds them into the CTA's shared-memory keys, and the CTA adds its C minima
// and maxima to the image's keys once.  The work is 4 C dres flops per pixel;
// the traffic bounds it: algorithmically X read once and F written once.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.cuh"

namespace qfca {
namespace {

constexpr int kResThreads = 256;

struct ResP {
    const float *X;          // image i at X + i C N
    int layout, H, W, C, dres, tiles;  // tiles: CTAs per image
    const double *mean, *V;  // image i: mean + i C, V + i C dres ([C][dres])
    float *F;                // image i: [C][N] at F + i C N
    uint32_t *mm;            // image i at mm + i 2 C kKeyStride: min of channel c at c*kKeyStride, max at (C+c)*kKeyStride
};

// PX pixels per thread (4: NCHW with N % 4 == 0 and 16-byte aligned X, one
// 16-byte load per channel; else 1); DRM >= dres bounds the registers of the
// projections.
template <int PX, int DRM>
__global__ void __launch_bounds__(kResThreads) k_residual(const __grid_constant__ ResP p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int C = p.C, dr = p.dres;
    const int img = blockIdx.x / p.tiles, tile = blockIdx.x % p.tiles;
    const long N = (long)p.H * p.W;
    const float *X = p.X + (size_t)img * C * N;
    const double *mean = p.mean + (size_t)img * C, *Vg = p.V + (size_t)img * C * dr;
    float *Fo = p.F + (size_t)img * C * N;
    uint32_t *mm = p.mm + (size_t)img * 2 * C * kKeyStride;
    float *mu = reinterpret_cast<float *>(smem_raw);   // [C]
    float *Vs = mu + C;                                 // [C][dres]
    uint32_t *mn = reinterpret_cast<uint32_t *>(Vs + (size_t)C * dr);  // [C]
    uint32_t *mx = mn + C;                              // [C]
    for (int c = threadIdx.x; c < C; c += kResThreads) {
        mu[c] = (float)mean[c];
        mn[c] = 0xffffffffu;
        mx[c] = 0u;
    }
    for (int e = threadIdx.x; e < C * dr; e += kResThreads) Vs[e] = (float)Vg[e];
    __syncthreads();
    const long px = ((long)tile * kResThreads + threadIdx.x) * PX;  // first pixel of this thread
    const bool ok = px < N;                                          // PX = 4: N % 4 == 0, so all four are valid
    const long q = ok ? px : 0;
    auto load = [&](int c, float *xs) {
        if (PX == 4) {
            const float4 v = *reinterpret_cast<const float4 *>(X + (size_t)c * N + q);
            xs[0] = v.x, xs[1] = v.y, xs[2] = v.z, xs[3] = v.w;
        } else {
            xs[0] = p.layout == 0 ? X[(size_t)c * N + q] : X[(size_t)q * C + c];
        }
    };
    float y[PX][DRM];
#pragma unroll
    for (int j = 0; j < PX; j++)
#pragma unroll
        for (int k = 0; k < DRM; k++) y[j][k] = 0.0f;
    constexpr int U = PX == 4 ? 4 : 8;  // channels whose loads are in flight together
    auto accumulate = [&](int c, const float *xs) {
        const float *v = Vs + (size_t)c * dr;
        const float m = mu[c];
#pragma unroll
        for (int k = 0; k < DRM; k++)
            if (k < dr) {
                const float vk = v[k];
#pragma unroll
                for (int j = 0; j < PX; j++) y[j][k] = fmaf(xs[j] - m, vk, y[j][k]);
            }
    };
    int c = 0;
    for (; c + U <= C; c += U) {
        float xs[U][PX];
#pragma unroll
        for (int u = 0; u < U; u++) load(c + u, xs[u]);
#pragma unroll
        for (int u = 0; u < U; u++) accumulate(c + u, xs[u]);
    }
    for (; c < C; c++) {
        float xs[PX];
        load(c, xs);
        accumulate(c, xs);
    }
    const int lane = threadIdx.x & 31;
    auto emit = [&](int cc, const float *xs) {
        const float *v = Vs + (size_t)cc * dr;
        const float m = mu[cc];
        float f[PX];
#pragma unroll
        for (int j = 0; j < PX; j++) f[j] = xs[j] - m;
#pragma unroll
        for (int k = 0; k < DRM; k++)
            if (k < dr) {
                const float vk = v[k];
#pragma unroll
                for (int j = 0; j < PX; j++) f[j] = fmaf(-vk, y[j][k], f[j]);
            }
        uint32_t kmin = 0xffffffffu, kmax = 0u;
#pragma unroll
        for (int j = 0; j < PX; j++) {
            const uint32_t key = f2key(f[j]);
            kmin = min(kmin, key);
            kmax = max(kmax, key);
        }
        if (ok) {
            if (PX == 4) *reinterpret_cast<float4 *>(Fo + (size_t)cc * N + px) = make_float4(f[0], f[1], f[2], f[3]);
            else Fo[(size_t)cc * N + px] = f[0];
        }
        kmin = __reduce_min_sync(0xffffffffu, ok ? kmin : 0xffffffffu);
        kmax = __reduce_max_sync(0xffffffffu, ok ? kmax : 0u);
        if (lane == 0) {
            atomicMin(&mn[cc], kmin);
            atomicMax(&mx[cc], kmax);
        }
    };
    c = 0;
    for (; c + U <= C; c += U) {
        float xs[U][PX];
#pragma unroll
        for (int u = 0; u < U; u++) load(c + u, xs[u]);
#pragma unroll
        for (int u = 0; u < U; u++) emit(c + u, xs[u]);
    }
    for (; c < C; c++) {
        float xs[PX];
        load(c, xs);
        emit(c, xs);
    }
    __syncthreads();
    for (int c2 = threadIdx.x; c2 < C; c2 += kResThreads) {
        atomicMin(&mm[(size_t)c2 * kKeyStride], mn[c2]);
        atomicMax(&mm[(size_t)(C + c2) * kKeyStride], mx[c2]);
    }
}

DeviceOnce g_attrs_res;

}  // namespace

size_t residual_smem(int C, int dres) { return sizeof(float) * ((size_t)C + (size_t)C * dres) + 2 * sizeof(uint32_t) * C; }

cudaError_t launch_residual(const float *X, int layout, int H, int W, int C, const double *mean, const double *V,
                            int dres, int nimg, float *F, uint32_t *mm, cudaStream_t st) {
    if (dres < 0 || dres > kMaxResidual) return cudaErrorInvalidValue;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaError_t e = device_once(g_attrs_res, dev, [] {
        const int lim = 200 * 1024;
        cudaError_t r = cudaFuncSetAttribute(k_residual<1, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        if (r == cudaSuccess) r = cudaFuncSetAttribute(k_residual<1, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        if (r == cudaSuccess) r = cudaFuncSetAttribute(k_residual<4, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        if (r == cudaSuccess) r = cudaFuncSetAttribute(k_residual<4, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        if (r == cudaSuccess) r = cudaFuncSetAttribute(k_residual<4, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        return r;
    });
    if (e != cudaSuccess) return e;
    e = launch_init_keys(mm, C, nimg, st);
    if (e != cudaSuccess) return e;
    const long N = (long)H * W;
    // four pixels per thread only when that still leaves about two waves of CTAs
    const bool wide = layout == 0 && N % 4 == 0 && ((uintptr_t)X & 15) == 0 && ((uintptr_t)F & 15) == 0 &&
                      (N / (4L * kResThreads)) * nimg >= 300;
    const int PX = wide ? 4 : 1;
    const int tiles = (int)((N + (long)kResThreads * PX - 1) / ((long)kResThreads * PX));
    ResP p{X, layout, H, W, C, dres, tiles, mean, V, F, mm};
    const unsigned grid = (unsigned)((long)tiles * nimg);
    const size_t smem = residual_smem(C, dres);
    if (wide && dres <= 8) QFCA_LAUNCH("k_residual", st, (k_residual<4, 8><<<grid, kResThreads, smem, st>>>(p)));
    else if (wide && dres <= 16) QFCA_LAUNCH("k_residual", st, (k_residual<4, 16><<<grid, kResThreads, smem, st>>>(p)));
    else if (wide) QFCA_LAUNCH("k_residual", st, (k_residual<4, 32><<<grid, kResThreads, smem, st>>>(p)));
    else if (dres <= 8) QFCA_LAUNCH("k_residual", st, (k_residual<1, 8><<<grid, kResThreads, smem, st>>>(p)));
    else QFCA_LAUNCH("k_residual", st, (k_residual<1, 32><<<grid, kResThreads, smem, st>>>(p)));
    return cudaGetLastError();
}

}  // namespace qfca
