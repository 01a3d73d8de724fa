// median.cu -- the median reference (arXiv 2510.15602, Sec. 3.2): for each
// component, the reference's m-th value is the median over all full windows
// ((2r+1)^2 pixels, centre at least r from every border) of their m-th
// smallest value, m = 1..T^2; the reference is the histogram of those T^2
// values (N_ref = T^2).  On bin indices: a non-decreasing quantiser commutes
// with order statistics, so this is also the quantised median of the values.
//
// With cumP_b(p) the window's cumulative count up to bin b, the m-th smallest
// value of window p is <= b exactly when cumP_b(p) >= m, so
//     G[b][m] = #{p : cumP_b(p) >= m},   median_m = min{b : G[b][m] >= ceil(Np/2)}
// (the lower median of Np windows).  k_median_ref slides each window column's
// histogram down the image and, per full window, adds one count at
// D[b][cumP_b] for every bin (shared memory, then the CTA's table is added
// into the image's table in global memory); G is the suffix sum of D over the
// count.  k_median_fin forms G, the per-rank medians and their histogram.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"

namespace qfca {
namespace {

struct MedImgP {
    const uint8_t *bins;   // [d][H][pitch]
    int H, W, pitch, r;
    int nstrip, sw;        // strips of window centres, centres per strip
    long cta0;
    uint32_t *D;           // [d][B][T^2 + 1] counts (zeroed by the launcher)
    uint32_t *ref;         // [d][B] output
};

struct MedParams {
    int n, d, B, nt;
    MedImgP img[kMaxBatch];
};

size_t med_smem(int nt, int B, int r) {
    const int T2 = (2 * r + 1) * (2 * r + 1);
    const int rw = (nt + 2 * r + 15) & ~15;
    return sizeof(uint32_t) * ((size_t)B * nt + (size_t)B * (T2 + 1)) + (size_t)(2 * r + 2) * rw + 16;
}

constexpr size_t kMedSmemMax = 200 * 1024;

__global__ void __launch_bounds__(256) k_median_ref(const __grid_constant__ MedParams p) {
    const int B = p.B, nt = p.nt;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const long cta = blockIdx.x;
    const int ii = table_image(p.n, cta, [&](int i) { return p.img[i].cta0; });
    const MedImgP &im = p.img[ii];
    const int H = im.H, W = im.W, r = im.r, span = 2 * r + 1, T2 = span * span;
    const long local = cta - im.cta0;
    const int strip = (int)(local % im.nstrip), k = (int)(local / im.nstrip);
    const int cx0 = r + strip * im.sw;             // first window centre column of the strip
    const int ncen = min(im.sw, W - r - cx0);      // centres in this strip
    const int px0 = cx0 - r;                       // image column of ring column 0
    const int rw = (nt + 2 * r + 15) & ~15;
    const int RR = 2 * r + 2;
    uint32_t *hist = reinterpret_cast<uint32_t *>(smem_raw);  // [B][nt]
    uint32_t *D = hist + (size_t)B * nt;                       // [B][T2 + 1]
    uint8_t *ring = reinterpret_cast<uint8_t *>(D + (size_t)B * (T2 + 1));  // [RR][rw]
    const int t = threadIdx.x;
    const uint8_t *plane = im.bins + (size_t)k * H * im.pitch;
    for (int e = t; e < B * nt + B * (T2 + 1); e += nt) hist[e] = 0;
    auto load_row = [&](int yy, int slot) {
        uint8_t *dst = ring + (size_t)slot * rw;
        for (int col = t; col < rw; col += nt) {
            const int x = px0 + col;
            dst[col] = (x < W && col < ncen + 2 * r) ? (uint8_t)min((int)plane[(size_t)yy * im.pitch + x], B - 1) : 0;
        }
    };
    // rows 0 .. 2r-1 of the first window, then one row per step
    for (int yy = 0; yy < 2 * r; yy++) load_row(yy, yy % RR);
    __syncthreads();
    const bool on = t < ncen;
    if (on)
        for (int yy = 0; yy < 2 * r; yy++) {
            const uint8_t *rp = ring + (size_t)(yy % RR) * rw + t;
            for (int u = 0; u < span; u++) atomicAdd(&hist[(size_t)rp[u] * nt + t], 1u);
        }
    for (int y = r; y < H - r; y++) {
        // row y + r enters (loaded now), row y - r - 1 leaves
        load_row(y + r, (y + r) % RR);
        __syncthreads();
        if (on) {
            const uint8_t *ra = ring + (size_t)((y + r) % RR) * rw + t;
            for (int u = 0; u < span; u++) atomicAdd(&hist[(size_t)ra[u] * nt + t], 1u);
            if (y - r - 1 >= 0) {
                const uint8_t *rb = ring + (size_t)((y - r - 1) % RR) * rw + t;
                for (int u = 0; u < span; u++) atomicAdd(&hist[(size_t)rb[u] * nt + t], 0xffffffffu);
            }
            uint32_t cum = 0;
            for (int b = 0; b < B; b++) {
                cum += hist[(size_t)b * nt + t];
                if (cum) atomicAdd(&D[(size_t)b * (T2 + 1) + cum], 1u);
            }
        }
        __syncthreads();
    }
    uint32_t *Dg = im.D + (size_t)k * B * (T2 + 1);
    for (int e = t; e < B * (T2 + 1); e += nt)
        if (D[e]) atomicAdd(&Dg[e], D[e]);
}

// One CTA per (image, component): G = suffix sums of D over the count, the
// lower median per rank, and their histogram.
__global__ void __launch_bounds__(256) k_median_fin(const __grid_constant__ MedParams p) {
    const int B = p.B;
    const int ii = blockIdx.x / p.d, k = blockIdx.x % p.d;
    const MedImgP &im = p.img[ii];
    const int r = im.r, T2 = (2 * r + 1) * (2 * r + 1);
    const long Np = (long)(im.H - 2 * r) * (im.W - 2 * r);
    const uint32_t half = (uint32_t)((Np + 1) / 2);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    uint32_t *G = reinterpret_cast<uint32_t *>(smem_raw);  // [B][T2 + 1]
    uint32_t *R = G + (size_t)B * (T2 + 1);                  // [B]
    const uint32_t *D = im.D + (size_t)k * B * (T2 + 1);
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        uint32_t s = 0;
        for (int c = T2; c >= 0; c--) {
            s += D[(size_t)b * (T2 + 1) + c];
            G[(size_t)b * (T2 + 1) + c] = s;
        }
        R[b] = 0;
    }
    __syncthreads();
    for (int m = 1 + threadIdx.x; m <= T2; m += blockDim.x) {
        int b = 0;
        while (b < B - 1 && G[(size_t)b * (T2 + 1) + m] < half) b++;
        atomicAdd(&R[b], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < B; b += blockDim.x) im.ref[(size_t)k * B + b] = R[b];
}

DeviceOnce g_attrs_med;

// Threads (window centres) per CTA: the widest of 256, 128, 64, 32 whose
// histograms and count table fit; 0 when none does.
int med_nt_cap(int B, int r) {
    if (sizeof(uint32_t) * ((size_t)B * ((2 * r + 1) * (2 * r + 1) + 2)) > kMedSmemMax) return 0;
    for (int nt = 256; nt >= 32; nt >>= 1)
        if (med_smem(nt, B, r) <= kMedSmemMax) return nt;
    return 0;
}

}  // namespace

bool median_shape_ok(int B, int r) { return r >= 1 && med_nt_cap(B, r) > 0; }


size_t median_jobs_workspace_bytes(const MedianJob *jobs, int n, int d, int B) {
    size_t b = 0;
    for (int i = 0; i < n; i++) {
        const size_t T2 = (size_t)(2 * jobs[i].r + 1) * (2 * jobs[i].r + 1);
        b += align_up(sizeof(uint32_t) * d * B * (T2 + 1), 256);
    }
    return b;
}

cudaError_t launch_median_jobs(const MedianJob *jobs, int n, int d, int B, void *ws, cudaStream_t st) {
    int dev = 0;
    cudaGetDevice(&dev);
    int rmax = 0;
    for (int i = 0; i < n; i++) {
        if (jobs[i].H <= 2 * jobs[i].r || jobs[i].W <= 2 * jobs[i].r) return cudaErrorInvalidValue;
        rmax = std::max(rmax, jobs[i].r);
    }
    const int ntcap = med_nt_cap(B, rmax);
    if (ntcap == 0) return cudaErrorNotSupported;
    cudaError_t e = device_once(g_attrs_med, dev, [] {
        cudaError_t r = cudaFuncSetAttribute(k_median_ref, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMedSmemMax);
        if (r == cudaSuccess)
            r = cudaFuncSetAttribute(k_median_fin, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMedSmemMax);
        return r;
    });
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(ws, 0, median_jobs_workspace_bytes(jobs, n, d, B), st);
    if (e != cudaSuccess) return e;
    unsigned char *w = static_cast<unsigned char *>(ws);
    std::vector<uint32_t *> Dp(n);
    for (int i = 0; i < n; i++) {
        const size_t T2 = (size_t)(2 * jobs[i].r + 1) * (2 * jobs[i].r + 1);
        Dp[i] = reinterpret_cast<uint32_t *>(w);
        w += align_up(sizeof(uint32_t) * d * B * (T2 + 1), 256);
    }
    for (int i0 = 0; i0 < n; i0 += kMaxBatch) {
        const int m = std::min(kMaxBatch, n - i0);
        MedParams mp{};
        mp.n = m;
        mp.d = d;
        mp.B = B;
        int nt = 32;
        long ctas = 0;
        for (int i = 0; i < m; i++) {
            const MedianJob &j = jobs[i0 + i];
            MedImgP &q = mp.img[i];
            const int ncen = j.W - 2 * j.r, cap = ntcap;
            q.bins = j.bins;
            q.H = j.H;
            q.W = j.W;
            q.pitch = j.pitch;
            q.r = j.r;
            q.nstrip = (ncen + cap - 1) / cap;
            q.sw = (ncen + q.nstrip - 1) / q.nstrip;
            q.cta0 = ctas;
            q.D = Dp[i0 + i];
            q.ref = j.ref_out;
            nt = std::max(nt, (q.sw + 31) & ~31);
            ctas += (long)q.nstrip * d;
        }
        mp.nt = nt;
        const size_t smem = med_smem(nt, B, rmax);
        QFCA_LAUNCH("k_median_ref", st, (k_median_ref<<<(unsigned)ctas, nt, smem, st>>>(mp)));
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        const int T2max = (2 * rmax + 1) * (2 * rmax + 1);
        const size_t fsmem = sizeof(uint32_t) * ((size_t)B * (T2max + 1) + B);
        QFCA_LAUNCH("k_median_fin", st, (k_median_fin<<<(unsigned)(m * d), 256, fsmem, st>>>(mp)));
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace qfca
