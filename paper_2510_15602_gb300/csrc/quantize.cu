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

struct QuantImgP {
    const float *Y;           // [d][N]
    int H, W;
    long cta0;                // first CTA of this image
    const uint32_t *mm;       // min/max keys (image range) or NULL
    const float *lo_in, *hi_in;  // fixed range [d] when mm is NULL
    uint8_t *bins;            // [d][H][pitch]
    int pitch;
    float *lo_out, *hi_out;   // [d] or NULL
    uint32_t *hist;           // [d][B] or NULL
};

struct QuantParams {
    int n, d, B;
    QuantImgP img[kMaxBatch];
};

// One CTA = one component x a band of rows of one image of the table.
__global__ void __launch_bounds__(kThreads) k_quantize(const __grid_constant__ QuantParams p) {
    __shared__ uint32_t sh[256];
    const long cta = blockIdx.x;
    int ii = 0;
    while (ii + 1 < p.n && p.img[ii + 1].cta0 <= cta) ii++;
    const QuantImgP &im = p.img[ii];
    const int d = p.d, B = p.B, H = im.H, W = im.W;
    const long N = (long)H * W;
    const long local = cta - im.cta0;
    const int k = (int)(local % d), band = (int)(local / d);
    float lo, hi;
    if (im.mm) {
        lo = key2f(im.mm[k * kKeyStride]);
        hi = key2f(im.mm[(d + k) * kKeyStride]);
    } else {
        lo = im.lo_in[k];
        hi = im.hi_in[k];
    }
    if (band == 0 && threadIdx.x == 0) {
        if (im.lo_out) im.lo_out[k] = lo;
        if (im.hi_out) im.hi_out[k] = hi;
    }
    for (int b = threadIdx.x; b < B; b += kThreads) sh[b] = 0;
    __syncthreads();
    const float fB = (float)B;
    const float *yk = im.Y + (long)k * N;
    uint8_t *bk = im.bins + (long)k * H * im.pitch;
    const int y0 = band * kRowsPerCta;
    const int y1 = min(H, y0 + kRowsPerCta);
    // a thread's pixels of the band's rows are loaded before any is used: eight loads in flight
    // per thread (the bins and counts written in between would otherwise keep them in order)
    for (int x = threadIdx.x; x < W; x += kThreads) {
        float v[kRowsPerCta];
#pragma unroll
        for (int i = 0; i < kRowsPerCta; i++) v[i] = y0 + i < y1 ? __ldg(yk + (long)(y0 + i) * W + x) : 0.0f;
#pragma unroll
        for (int i = 0; i < kRowsPerCta; i++) {
            if (y0 + i >= y1) break;
            const int q = quant_bin(v[i], lo, hi, fB, B);
            bk[(long)(y0 + i) * im.pitch + x] = (uint8_t)q;
            if (im.hist) atomicAdd(&sh[q], 1u);
        }
    }
    __syncthreads();
    if (im.hist)
        for (int b = threadIdx.x; b < B; b += kThreads)
            if (sh[b]) atomicAdd(&im.hist[(long)k * B + b], sh[b]);
}

}  // namespace

cudaError_t launch_quantize_jobs(const QuantJob *jobs, int n, int d, int B, bool zero_hist, cudaStream_t st) {
    for (int i0 = 0; i0 < n; i0 += kMaxBatch) {
        const int m = n - i0 < kMaxBatch ? n - i0 : kMaxBatch;
        QuantParams p;
        memset(&p, 0, sizeof(p));
        p.n = m, p.d = d, p.B = B;
        long cta = 0;
        for (int i = 0; i < m; i++) {
            const QuantJob &j = jobs[i0 + i];
            QuantImgP &im = p.img[i];
            im.Y = j.Y, im.H = j.H, im.W = j.W, im.cta0 = cta;
            cta += (long)((j.H + kRowsPerCta - 1) / kRowsPerCta) * d;
            im.mm = j.mm, im.lo_in = j.lo_in, im.hi_in = j.hi_in;
            im.bins = j.bins, im.pitch = j.pitch, im.lo_out = j.lo_out, im.hi_out = j.hi_out, im.hist = j.hist;
            if (j.hist && zero_hist) {
                cudaError_t err = cudaMemsetAsync(j.hist, 0, sizeof(uint32_t) * (size_t)d * B, st);
                if (err != cudaSuccess) return err;
            }
        }
        QFCA_LAUNCH("k_quantize", st, k_quantize<<<(unsigned)cta, kThreads, 0, st>>>(p));
        cudaError_t err = cudaGetLastError();
        if (err != cudaSuccess) return err;
    }
    return cudaSuccess;
}

cudaError_t launch_quantize(const float *Y, long N, int H, int W, int d, int nimg, int B, int range_mode,
                            const uint32_t *mm_keys, const float *lo_in, const float *hi_in, uint8_t *bins,
                            int pitch, float *lo_out, float *hi_out, uint32_t *hist, cudaStream_t st) {
    if (hist) {
        cudaError_t err = cudaMemsetAsync(hist, 0, sizeof(uint32_t) * (size_t)d * B * nimg, st);
        if (err != cudaSuccess) return err;
    }
    QuantJob jobs[kMaxBatch];
    for (int i0 = 0; i0 < nimg; i0 += kMaxBatch) {
        const int m = nimg - i0 < kMaxBatch ? nimg - i0 : kMaxBatch;
        for (int i = 0; i < m; i++) {
            const long img = i0 + i;
            QuantJob &j = jobs[i];
            j.Y = Y + img * d * N;
            j.H = H, j.W = W;
            j.mm = range_mode == QFCA_RANGE_IMAGE ? mm_keys + img * 2 * d * kKeyStride : nullptr;
            j.lo_in = lo_in, j.hi_in = hi_in;
            j.bins = bins + img * d * H * (long)pitch, j.pitch = pitch;
            j.lo_out = lo_out ? lo_out + img * d : nullptr;
            j.hi_out = hi_out ? hi_out + img * d : nullptr;
            j.hist = hist ? hist + img * d * B : nullptr;
        }
        cudaError_t e = launch_quantize_jobs(jobs, m, d, B, false, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace qfca
