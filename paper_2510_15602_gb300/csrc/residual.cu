// residual.cu -- the QFCA+ features (arXiv 2510.15602, Sec. 3.3): the input
// features minus their PCA reconstruction from the top dres components,
//     F = (X - mean) - (X - mean) V V^T,
// for all C channels, with each channel's image-wide min/max (order-preserving
// u32 keys) for the per-channel quantisation that follows.
//
// k_residual_tiled (NCHW maps whose rows allow 16-byte copies): a tile of
// pixels with all channels in shared memory, both channel walks from there.
// k_residual (other layouts): one thread per pixel (or four adjacent pixels,
// one 16-byte load per channel, when the layout allows).  The thread forms the dres projections
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

#include <algorithm>

#include "internal.cuh"
#include "tc.cuh"

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

// The tiled form (NCHW, N % 4 == 0, X 16-byte aligned): persistent CTAs, each
// over a contiguous range of TP-pixel tiles of the batch, with ALL C channels of
// a tile staged in shared memory by 16-byte cp.async copies, double-buffered
// (the next tile loads while this one is computed), so the second walk over the
// channels reads shared memory, not DRAM (features read once, residual written
// once).  Thread t owns pixel t % TP and the channels congruent to
// g = t / TP (mod G): the projections are summed over its channels in registers
// (DRM >= dres accumulators), the G partial sums of a pixel are added in a
// fixed order in shared memory, and the residual of its channels is formed
// with the pixel's projections held in registers.  A CTA reloads the mean and
// basis when its range enters a new image and flushes that image's keys when
// it leaves it.
constexpr int kTileThreads = 256;

size_t residual_tiled_smem(int C, int dres, int TP) {
    const int G = kTileThreads / TP;
    return sizeof(float) * (2 * (size_t)C * TP + C + (size_t)C * dres + (size_t)G * dres * TP) +
           2 * sizeof(uint32_t) * C;
}

template <int TP, int DRM>
__global__ void __launch_bounds__(kTileThreads) k_residual_tiled(const __grid_constant__ ResP p, long total_tiles) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int G = kTileThreads / TP;
    constexpr int CH = TP / 4;  // 16-byte chunks per channel row of a tile
    const int C = p.C, dr = p.dres;
    const long N = (long)p.H * p.W;
    float *xs = reinterpret_cast<float *>(smem_raw);    // [2][C][TP]
    float *mu = xs + 2 * (size_t)C * TP;                // [C]
    float *Vs = mu + C;                                 // [C][dres]
    float *part = Vs + (size_t)C * dr;                  // [G][dres][TP] partial projections
    uint32_t *mn = reinterpret_cast<uint32_t *>(part + (size_t)G * dr * TP);  // [C]
    uint32_t *mx = mn + C;                                                    // [C]
    const int tid = threadIdx.x, lane = tid & 31;
    const int pl = tid % TP, grp = tid / TP;  // a warp shares grp (TP >= 32), so basis reads broadcast
    const long t_begin = total_tiles * blockIdx.x / gridDim.x, t_end = total_tiles * (blockIdx.x + 1) / gridDim.x;

    auto issue_load = [&](long t, int b) {
        const int img = (int)(t / p.tiles);
        const long p0 = (t % p.tiles) * TP;
        const float *X = p.X + (size_t)img * C * N;
        float *buf = xs + (size_t)b * C * TP;
        for (int e = tid; e < C * CH; e += kTileThreads) {
            const int c = e / CH, q4 = e % CH;
            const long px = p0 + 4 * q4;
            float *dst = buf + (size_t)c * TP + 4 * q4;
            if (px < N) tc::cp_async16(tc::smem_u32(dst), X + (size_t)c * N + px);
            else *reinterpret_cast<float4 *>(dst) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    auto flush_keys = [&](int img) {
        uint32_t *mm = p.mm + (size_t)img * 2 * C * kKeyStride;
        for (int c = tid; c < C; c += kTileThreads) {
            atomicMin(&mm[(size_t)c * kKeyStride], mn[c]);
            atomicMax(&mm[(size_t)(C + c) * kKeyStride], mx[c]);
        }
    };
    if (t_begin < t_end) issue_load(t_begin, 0);
    tc::cp_async_commit();
    int cur = -1;
    for (long t = t_begin; t < t_end; t++) {
        const int b = (int)((t - t_begin) & 1);
        if (t + 1 < t_end) issue_load(t + 1, b ^ 1);
        tc::cp_async_commit();
        const int img = (int)(t / p.tiles);
        if (img != cur) {  // the same in every thread
            __syncthreads();
            if (cur >= 0) flush_keys(cur);
            __syncthreads();
            const double *mean = p.mean + (size_t)img * C, *Vg = p.V + (size_t)img * C * dr;
            for (int c = tid; c < C; c += kTileThreads) {
                mu[c] = (float)mean[c];
                mn[c] = 0xffffffffu;
                mx[c] = 0u;
            }
            for (int e = tid; e < C * dr; e += kTileThreads) Vs[e] = (float)Vg[e];
            cur = img;
        }
        tc::cp_async_wait<1>();  // tile t has landed (tile t+1 may still be in flight)
        __syncthreads();
        const float *xt = xs + (size_t)b * C * TP;
        const long p0 = (t % p.tiles) * TP;
        const bool ok = p0 + pl < N;
        float y[DRM];
#pragma unroll
        for (int k = 0; k < DRM; k++) y[k] = 0.0f;
        for (int c = grp; c < C; c += G) {
            const float xm = xt[(size_t)c * TP + pl] - mu[c];
            const float *v = Vs + (size_t)c * dr;
#pragma unroll
            for (int k = 0; k < DRM; k++)
                if (k < dr) y[k] = fmaf(xm, v[k], y[k]);
        }
#pragma unroll
        for (int k = 0; k < DRM; k++)
            if (k < dr) part[((size_t)grp * dr + k) * TP + pl] = y[k];
        __syncthreads();
        // the pixel's projections: the G partial sums in a fixed order
#pragma unroll
        for (int k = 0; k < DRM; k++)
            if (k < dr) {
                float s = part[(size_t)k * TP + pl];
                for (int g = 1; g < G; g++) s += part[((size_t)g * dr + k) * TP + pl];
                y[k] = s;
            }
        // residual f_c = (x_c - mean_c) - sum_k V_ck y_k for the thread's channels; per-channel keys
        float *Fo = p.F + (size_t)img * C * N;
        for (int c = grp; c < C; c += G) {
            const float *v = Vs + (size_t)c * dr;
            float f = xt[(size_t)c * TP + pl] - mu[c];
#pragma unroll
            for (int k = 0; k < DRM; k++)
                if (k < dr) f = fmaf(-v[k], y[k], f);
            if (ok) Fo[(size_t)c * N + p0 + pl] = f;
            const uint32_t key = f2key(f);
            const uint32_t kmin = __reduce_min_sync(0xffffffffu, ok ? key : 0xffffffffu);
            const uint32_t kmax = __reduce_max_sync(0xffffffffu, ok ? key : 0u);
            if (lane == 0) {
                atomicMin(&mn[c], kmin);
                atomicMax(&mx[c], kmax);
            }
        }
        __syncthreads();  // buffer b and the partial sums are free again
    }
    tc::cp_async_wait<0>();
    if (cur >= 0) {
        __syncthreads();
        flush_keys(cur);
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
        auto tiled = [&](auto kern) {
            if (r == cudaSuccess) r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
        };
        tiled(k_residual_tiled<64, 8>);
        tiled(k_residual_tiled<64, 16>);
        tiled(k_residual_tiled<64, 32>);
        tiled(k_residual_tiled<32, 8>);
        tiled(k_residual_tiled<32, 16>);
        tiled(k_residual_tiled<32, 32>);
        return r;
    });
    if (e != cudaSuccess) return e;
    e = launch_init_keys(mm, C, nimg, st);
    if (e != cudaSuccess) return e;
    const long N = (long)H * W;
    // the tiled form when every feature row can be copied in 16-byte pieces
    if (layout == 0 && N % 4 == 0 && ((uintptr_t)X & 15) == 0) {
        const int TP = 32;
        const size_t smem = residual_tiled_smem(C, dres, TP);
        if (smem <= 110 * 1024) {  // two CTAs per SM
            const int tiles = (int)((N + TP - 1) / TP);
            ResP p{X, layout, H, W, C, dres, tiles, mean, V, F, mm};
            int n_sm = 0;
            e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
            if (e != cudaSuccess) return e;
            const long total = (long)tiles * nimg;
            const unsigned grid = (unsigned)std::min<long>(total, 2L * n_sm);
            auto go = [&](auto kern) {
                QFCA_LAUNCH("k_residual", st, (kern<<<grid, kTileThreads, smem, st>>>(p, total)));
            };
            if (TP == 64) {
                if (dres <= 8) go(k_residual_tiled<64, 8>);
                else if (dres <= 16) go(k_residual_tiled<64, 16>);
                else go(k_residual_tiled<64, 32>);
            } else {
                if (dres <= 8) go(k_residual_tiled<32, 8>);
                else if (dres <= 16) go(k_residual_tiled<32, 16>);
                else go(k_residual_tiled<32, 32>);
            }
            return cudaGetLastError();
        }
    }
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
