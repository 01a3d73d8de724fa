// quantize.cu -- uniform quantisation of each principal component into B
// equally spaced bins (arXiv 2510.15602, Sec. 3.1) and the reference histogram
// R_k[b] (the image-global histogram of component k).
//
// One CTA = one component k x a band of rows.  The bin decision is taken in
// FP32 with IEEE-rounded operations in a fixed order:
//     t = (y - lo) / (hi - lo);  v = t * B;  q = clamp((int)v, 0, B-1)
// (hi == lo gives q = 0).  Histogram: shared-memory counters per CTA, then one
// global atomicAdd per bin (integer adds: order-independent, exact).
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.cuh"

namespace qfca {
namespace {

constexpr int kThreads = 256;
constexpr int kRowsPerCta = 8;

__device__ __forceinline__ int bin_of(float y, float lo, float hi, float fB, int B) {
    if (!(hi > lo)) return 0;
    const float t = __fdiv_rn(__fsub_rn(y, lo), __fsub_rn(hi, lo));
    const float v = __fmul_rn(t, fB);
    int q = v < 0.0f ? 0 : (int)v;
    return q > B - 1 ? B - 1 : q;
}

// Grid (row bands, d, images).
__global__ void __launch_bounds__(kThreads) k_quantize(const float *__restrict__ Y, long N, int H, int W, int d,
                                                       int B, int range_mode, const uint32_t *__restrict__ mm_keys,
                                                       const float *__restrict__ lo_in,
                                                       const float *__restrict__ hi_in, uint8_t *__restrict__ bins,
                                                       int pitch, float *__restrict__ lo_out,
                                                       float *__restrict__ hi_out, uint32_t *__restrict__ hist) {
    __shared__ uint32_t sh[256];
    const int k = blockIdx.y;
    const long img = blockIdx.z;
    Y += img * d * N;
    mm_keys += img * 2 * d * kKeyStride;
    bins += img * d * H * (long)pitch;
    if (lo_out) lo_out += img * d;
    if (hi_out) hi_out += img * d;
    if (hist) hist += img * d * B;
    float lo, hi;
    if (range_mode == QFCA_RANGE_IMAGE) {
        lo = key2f(mm_keys[k * kKeyStride]);
        hi = key2f(mm_keys[(d + k) * kKeyStride]);
    } else {
        lo = lo_in[k];
        hi = hi_in[k];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (lo_out) lo_out[k] = lo;
        if (hi_out) hi_out[k] = hi;
    }
    for (int b = threadIdx.x; b < B; b += kThreads) sh[b] = 0;
    __syncthreads();
    const float fB = (float)B;
    const float *yk = Y + (long)k * N;
    uint8_t *bk = bins + (long)k * H * pitch;
    const int y0 = blockIdx.x * kRowsPerCta;
    const int y1 = min(H, y0 + kRowsPerCta);
    for (int yy = y0; yy < y1; yy++) {
        for (int x = threadIdx.x; x < W; x += kThreads) {
            const int q = bin_of(yk[(long)yy * W + x], lo, hi, fB, B);
            bk[(long)yy * pitch + x] = (uint8_t)q;
            if (hist) atomicAdd(&sh[q], 1u);
        }
    }
    __syncthreads();
    if (hist)
        for (int b = threadIdx.x; b < B; b += kThreads)
            if (sh[b]) atomicAdd(&hist[(long)k * B + b], sh[b]);
}

}  // namespace

cudaError_t launch_quantize(const float *Y, long N, int H, int W, int d, int nimg, int B, int range_mode,
                            const uint32_t *mm_keys, const float *lo_in, const float *hi_in, uint8_t *bins,
                            int pitch, float *lo_out, float *hi_out, uint32_t *hist, cudaStream_t st) {
    if (hist) {
        cudaError_t err = cudaMemsetAsync(hist, 0, sizeof(uint32_t) * (size_t)d * B * nimg, st);
        if (err != cudaSuccess) return err;
    }
    dim3 grid((H + kRowsPerCta - 1) / kRowsPerCta, d, nimg);
    QFCA_LAUNCH("k_quantize", st,
                k_quantize<<<grid, kThreads, 0, st>>>(Y, N, H, W, d, B, range_mode, mm_keys, lo_in, hi_in, bins,
                                                      pitch, lo_out, hi_out, hist));
    return cudaGetLastError();
}

}  // namespace qfca
