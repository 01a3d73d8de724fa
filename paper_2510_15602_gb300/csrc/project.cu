// project.cu -- principal-component projection Y = (X - mean) V (arXiv 2510.15602,
// Sec. 3.3) with per-component min/max for the image-wide quantisation range.
//
// FP32 path: SIMT FFMA.  One CTA = 128 pixels x DT components (DT in {16,32,64}
// >= d, extra columns zero).  Channels are staged 32 at a time in shared memory
// (coalesced along pixels for NCHW, along channels for NHWC); each thread owns
// one pixel and DT FP32 accumulators; the basis chunk is read as broadcasts.
// Output Y is component-major [d][N] so quantisation and the window stage read
// it coalesced.  min/max per component: warp reductions, then one atomicMin /
// atomicMax per warp on order-preserving u32 keys.
#include <cuda_runtime.h>

#include <algorithm>
#include <stdint.h>

#include "internal.cuh"

namespace qfca {

// tcgen05 BF16 projection (project_tc.cu)
cudaError_t launch_project_bf16(const float *X, int layout, int H, int W, int C, const double *mean,
                                const double *V, int d, int nimg, float *Y, uint32_t *mm_keys, void *ws,
                                int *status, cudaStream_t st);
size_t project_bf16_workspace_bytes(int C, long N, int d, int nimg);

namespace {

constexpr int kPix = 128;
constexpr int kCh = 32;

// Per image (grid.y): mean32[c] = (float)mean[c];  V32[c][j] = (float)V[c][j] for j < d, 0 for d <= j < DT.
__global__ void k_prep_f32(const double *__restrict__ mean, const double *__restrict__ V, int C, int d, int DT,
                           int Cs, float *__restrict__ mean32, float *__restrict__ V32) {
    const long img = blockIdx.y;
    mean += img * C;
    V += img * C * d;
    mean32 += img * Cs;
    V32 += img * C * DT;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < C * DT; e += gridDim.x * blockDim.x) {
        const int c = e / DT, j = e % DT;
        V32[e] = j < d ? (float)V[(long)c * d + j] : 0.0f;
        if (j == 0) mean32[c] = (float)mean[c];
    }
}

// min keys start at the largest key, max keys at the smallest (per image: d min keys, then d max keys)
__global__ void k_init_keys(uint32_t *__restrict__ keys, int d, int nimg) {
    const long total = (long)nimg * 2 * d * kKeyStride;
    for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < total; e += (long)gridDim.x * blockDim.x) {
        const long within = e % (2L * d * kKeyStride);
        keys[e] = within < (long)d * kKeyStride ? 0xffffffffu : 0u;
    }
}

template <int DT>
__global__ void __launch_bounds__(kPix) k_project_f32(const float *__restrict__ X, int layout, int C, long N,
                                                     const float *__restrict__ mean32, const float *__restrict__ V32,
                                                     int d, int Cs, long tiles, float *__restrict__ Y,
                                                     uint32_t *__restrict__ mm_keys) {
    __shared__ float Xs[kCh][kPix + 1];
    __shared__ __align__(16) float Vs[kCh][DT];
    __shared__ float Ms[kCh];
    __shared__ uint32_t kmin[DT], kmax[DT];
    const int tid = threadIdx.x;
    if (tid < DT) { kmin[tid] = 0xffffffffu; kmax[tid] = 0u; }
    const long img = blockIdx.x / tiles;
    X += img * C * N;
    mean32 += img * Cs;
    V32 += img * C * DT;
    Y += img * d * N;
    mm_keys += img * 2 * d * kKeyStride;
    const long p0 = (blockIdx.x % tiles) * kPix;
    const long p = p0 + tid;
    float acc[DT];
#pragma unroll
    for (int j = 0; j < DT; j++) acc[j] = 0.0f;

    for (int c0 = 0; c0 < C; c0 += kCh) {
        const int nc = min(kCh, C - c0);
        if (layout == QFCA_NCHW) {
            for (int cl = 0; cl < kCh; cl++) {
                float v = 0.0f;
                if (cl < nc && p < N) v = X[(long)(c0 + cl) * N + p];
                Xs[cl][tid] = v;
            }
        } else {
            // 32 consecutive channels of one pixel per warp pass
            const int lane = tid & 31, warp = tid >> 5;
            for (int pp = warp; pp < kPix; pp += kPix / 32) {
                const long q = p0 + pp;
                float v = 0.0f;
                if (lane < nc && q < N) v = X[q * C + c0 + lane];
                Xs[lane][pp] = v;
            }
        }
        for (int e = tid; e < kCh * DT; e += kPix) {
            const int cl = e / DT, j = e % DT;
            Vs[cl][j] = cl < nc ? V32[(long)(c0 + cl) * DT + j] : 0.0f;
        }
        if (tid < kCh) Ms[tid] = tid < nc ? mean32[c0 + tid] : 0.0f;
        __syncthreads();
#pragma unroll 4
        for (int cl = 0; cl < kCh; cl++) {
            const float x = Xs[cl][tid] - Ms[cl];
            const float4 *vr = reinterpret_cast<const float4 *>(&Vs[cl][0]);
#pragma unroll
            for (int j4 = 0; j4 < DT / 4; j4++) {
                const float4 v = vr[j4];
                acc[4 * j4 + 0] = fmaf(x, v.x, acc[4 * j4 + 0]);
                acc[4 * j4 + 1] = fmaf(x, v.y, acc[4 * j4 + 1]);
                acc[4 * j4 + 2] = fmaf(x, v.z, acc[4 * j4 + 2]);
                acc[4 * j4 + 3] = fmaf(x, v.w, acc[4 * j4 + 3]);
            }
        }
        __syncthreads();
    }
    const bool valid = p < N;
    const int lane = tid & 31;
#pragma unroll
    for (int j = 0; j < DT; j++) {
        if (j >= d) break;
        if (valid) Y[(long)j * N + p] = acc[j];
        float mn = valid ? acc[j] : __int_as_float(0x7f800000);
        float mx = valid ? acc[j] : -__int_as_float(0x7f800000);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        }
        if (lane == 0) {
            atomicMin(&kmin[j], f2key(mn));
            atomicMax(&kmax[j], f2key(mx));
        }
    }
    __syncthreads();
    if (tid < d) {
        atomicMin(&mm_keys[tid * kKeyStride], kmin[tid]);
        atomicMax(&mm_keys[(d + tid) * kKeyStride], kmax[tid]);
    }
}

int pick_dt(int d) { return d <= 16 ? 16 : (d <= 32 ? 32 : 64); }

}  // namespace

cudaError_t launch_init_keys(uint32_t *mm_keys, int d, int nimg, cudaStream_t st) {
    const long nkeys = (long)nimg * 2 * d * kKeyStride;
    QFCA_LAUNCH("k_init_keys", st, k_init_keys<<<(unsigned)((nkeys + 255) / 256), 256, 0, st>>>(mm_keys, d, nimg));
    return cudaGetLastError();
}

size_t project_workspace_bytes(int C, long N, int d, int nimg) {
    const size_t f32 = align_up(sizeof(float) * (align_up(C, 64) + (size_t)C * 64) * nimg, 256);
    const size_t bf = project_bf16_workspace_bytes(C, N, d, nimg);
    const size_t f8 = project_fp8_workspace_bytes(C, d, nimg);
    return std::max(f32, std::max(bf, f8));
}

cudaError_t launch_project(const float *X, int layout, int H, int W, int C, const double *mean,
                           const double *V, int d, int nimg, int precision, float *Y, uint32_t *mm_keys, void *ws,
                           int *status, cudaStream_t st) {
    const long N = (long)H * W;
    const long nkeys = (long)nimg * 2 * d * kKeyStride;
    QFCA_LAUNCH("k_init_keys", st,
                k_init_keys<<<(unsigned)((nkeys + 255) / 256), 256, 0, st>>>(mm_keys, d, nimg));
    if (precision == QFCA_BF16)
        return launch_project_bf16(X, layout, H, W, C, mean, V, d, nimg, Y, mm_keys, ws, status, st);
    if (precision == QFCA_FP8_E4M3)
        return launch_project_fp8(X, layout, N, C, mean, V, d, nimg, Y, mm_keys, ws, status, st);
    const int DT = pick_dt(d);
    const int Cs = (int)align_up(C, 64);
    float *mean32 = (float *)ws;
    float *V32 = mean32 + (size_t)Cs * nimg;
    QFCA_LAUNCH("k_prep_f32", st,
                k_prep_f32<<<dim3((C * DT + 255) / 256, nimg), 256, 0, st>>>(mean, V, C, d, DT, Cs, mean32, V32));
    const long tiles = (N + kPix - 1) / kPix;
    const unsigned grid = (unsigned)(tiles * nimg);
    switch (DT) {
        case 16:
            QFCA_LAUNCH("k_project_f32", st,
                        k_project_f32<16><<<grid, kPix, 0, st>>>(X, layout, C, N, mean32, V32, d, Cs, tiles, Y, mm_keys));
            break;
        case 32:
            QFCA_LAUNCH("k_project_f32", st,
                        k_project_f32<32><<<grid, kPix, 0, st>>>(X, layout, C, N, mean32, V32, d, Cs, tiles, Y, mm_keys));
            break;
        default:
            QFCA_LAUNCH("k_project_f32", st,
                        k_project_f32<64><<<grid, kPix, 0, st>>>(X, layout, C, N, mean32, V32, d, Cs, tiles, Y, mm_keys));
            break;
    }
    return cudaGetLastError();
}

}  // namespace qfca
