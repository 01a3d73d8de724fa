// quantize.cu -- uniform quantisation of each principal component into B
// equally spaced bins (arXiv 2510.15602, Sec. 3.1) and the reference histogram
// R_k[b] (the image-global histogram of component k).
//
// One CTA = one component k x a band of rows.  The bin decision is taken in
// FP32 with IEEE-rounded operations in a fixed order:
//     t = (y - lo) / (hi - lo);  v = t * B;  q = clamp((int)v, 0, B-1)
// (hi == lo gives q = 0).  Every rounded step is monotone in y, so q(y) is a
// non-decreasing step function of y: q(y) = #{j in 1..B-1 : y >= e_j} with
// e_j the smallest float whose decision is >= j.  Each CTA finds its
// component's B-1 edges by bisection over the order-preserving keys of the
// floats, evaluating the decision itself (so the edges are exact by
// construction), and each pixel's bin is then a branch-free search of that
// table: the same bins as evaluating the division per pixel, at a fraction of
// its instructions.  Histogram: shared-memory counters per CTA, then one
// global atomicAdd per bin (integer adds: order-independent, exact).
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.cuh"

namespace qfca {
namespace {

constexpr int kThreads = 256;
constexpr int kRowsPerCta = 32;  // rows per CTA (the edge search is amortised over them)
constexpr int kLoadRows = 8;     // rows whose pixels a thread loads before using any

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

// e_j = the smallest float y with quant_bin(y) >= j (1 <= j <= B-1; needs hi > lo): bisection on the
// order-preserving keys, q(key2f(a)) < j <= q(key2f(b)) throughout (q(-inf) = 0, q(+inf) = B-1).
__device__ float bin_edge(int j, float lo, float hi, float fB, int B) {
    uint32_t a = f2key(-INFINITY), b = f2key(INFINITY);
    for (int it = 0; it < 33 && b - a > 1; it++) {
        const uint32_t m = a + ((b - a) >> 1);
        if (quant_bin(key2f(m), lo, hi, fB, B) >= j) b = m;
        else a = m;
    }
    return key2f(b);
}

// The bin of y from the edge table E[0..P-1] (E[j-1] = e_j, NaN past B-1; P a power of two >= B):
// the number of edges <= y (NaN compares false, so a NaN y gets 0 as quant_bin gives it).
template <int P>
__device__ __forceinline__ int edge_bin(float y, const float *E) {
    int q = 0;
#pragma unroll
    for (int s = P >> 1; s > 0; s >>= 1)
        if (y >= E[q + s - 1]) q += s;
    return q;
}

// One CTA = one component x a band of rows of one image of the table.
__global__ void __launch_bounds__(kThreads) k_quantize(const __grid_constant__ QuantParams p) {
    __shared__ uint32_t sh[256];
    __shared__ float edge[256];
    const long cta = blockIdx.x;
    const int ii = table_image(p.n, cta, [&](int i) { return p.img[i].cta0; });
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
    const float fB = (float)B;
    {  // the component's bin edges, one per thread (kThreads >= 256 >= P)
        const int j = threadIdx.x;
        edge[j] = (j < B - 1 && hi > lo) ? bin_edge(j + 1, lo, hi, fB, B) : __int_as_float(0x7fc00000);
    }
    __syncthreads();
    const float *yk = im.Y + (long)k * N;
    uint8_t *bk = im.bins + (long)k * H * im.pitch;
    const int y0 = band * kRowsPerCta;
    const int y1 = min(H, y0 + kRowsPerCta);
    // a thread's pixels of kLoadRows rows are loaded before any is used (the bins and counts
    // written in between would otherwise keep the loads in order)
    for (int x = threadIdx.x; x < W; x += kThreads)
        for (int g = y0; g < y1; g += kLoadRows) {
            float v[kLoadRows];
#pragma unroll
            for (int i = 0; i < kLoadRows; i++) v[i] = g + i < y1 ? __ldg(yk + (long)(g + i) * W + x) : 0.0f;
#pragma unroll
            for (int i = 0; i < kLoadRows; i++) {
                if (g + i >= y1) break;
                const int q = B <= 32 ? edge_bin<32>(v[i], edge) : edge_bin<256>(v[i], edge);
                bk[(long)(g + i) * im.pitch + x] = (uint8_t)q;
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
