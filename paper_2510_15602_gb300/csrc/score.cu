// score.cu -- per-pixel sliding-window histograms and the 1-D earth mover's
// distance to the reference histogram, averaged over components (arXiv
// 2510.15602, Sec. 3.1; W1 closed form of the supplement).
//
// For pixel p and component k with clipped window of N_loc pixels:
//     D_k(p) = sum_b |cumP_b * N_ref - cumR_b * N_loc|      (exact integers)
//     score(p) = sum_k D_k(p) / (d * N_loc * N_ref)
//
// k_window_emd: one CTA = a band of TH rows x a strip of SW columns x a group of
// components.  The bin tile with an r-pixel halo is staged in shared memory;
// each thread owns one output column and keeps its window histogram in shared
// memory (bin-major, thread-minor: conflict-free), sliding it down the band:
// one row of 2r+1 bins leaves and one enters per step (running window counts).
// The CDF walk is sequential per thread.  The per-pixel integer sum over the
// CTA's components goes to a u64 accumulator (atomic integer adds:
// order-independent and exact); k_finalize divides once per pixel.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "internal.cuh"

namespace qfca {
namespace {

constexpr int kSW = 128;  // output columns per CTA (one thread each)
constexpr int kTH = 16;   // output rows per CTA band

struct ScoreGeom {
    int TH, TR, TC, TCp, kg, n_kg;
    size_t smem;
};

ScoreGeom score_geom(int H, int W, int d, int B, int r, int nimg) {
    ScoreGeom g;
    g.TH = kTH;
    g.TR = g.TH + 2 * r;
    g.TC = kSW + 2 * r;
    g.TCp = (int)align_up(g.TC, 16);
    const long tiles = (long)((W + kSW - 1) / kSW) * ((H + g.TH - 1) / g.TH) * nimg;
    // enough CTAs for ~4 per SM over 152 SMs
    int n_kg = (int)((4 * 152 + tiles - 1) / tiles);
    if (n_kg < 1) n_kg = 1;
    if (n_kg > d) n_kg = d;
    g.kg = (d + n_kg - 1) / n_kg;
    g.n_kg = (d + g.kg - 1) / g.kg;
    g.smem = sizeof(uint32_t) * (size_t)B * kSW                 // histograms [B][kSW]
             + sizeof(unsigned long long) * (size_t)g.TH * kSW  // per-pixel sums
             + 2 * sizeof(uint32_t) * 256                       // cumR, cumR * N_loc(interior)
             + (size_t)g.TR * g.TCp;                            // bin tile
    return g;
}

// Window histograms + exact EMD numerators for a band of kTH rows x kSW columns
// and a group of components.  Thread t owns output column x0 + t: its window
// histogram lives in shared memory at hist[b * kSW + t] (conflict-free), and
// slides down the band (one row of 2r+1 bins leaves, one enters); increments
// are shared-memory atomics without return, so no thread waits on them.
// ACC is the type of the CDF walk: uint32_t when (B-1)(2r+1)^2 N_ref < 2^32
// (the numerator D and every term then fit), else unsigned long long.
template <typename ACC>
__global__ void __launch_bounds__(kSW) k_window_emd(const uint8_t *__restrict__ bins, int H, int W, int pitch, int d,
                                                     int B, int r, ScoreGeom g, const uint32_t *__restrict__ ref_hist,
                                                     uint32_t Nref, unsigned long long *__restrict__ acc,
                                                     uint64_t *__restrict__ numer) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *hist = reinterpret_cast<uint32_t *>(smem);
    unsigned long long *accS = reinterpret_cast<unsigned long long *>(hist + (size_t)B * kSW);
    uint32_t *cumR = reinterpret_cast<uint32_t *>(accS + (size_t)g.TH * kSW);
    uint32_t *cRi = cumR + 256;  // cumR[b] * N_loc for an interior window
    uint8_t *tile = reinterpret_cast<uint8_t *>(cRi + 256);

    const int t = threadIdx.x;
    const int x0 = blockIdx.x * kSW, y0 = blockIdx.y * g.TH;
    const long img = blockIdx.z / g.n_kg;
    const int k0 = (blockIdx.z % g.n_kg) * g.kg, k1 = min(d, k0 + g.kg);
    bins += img * d * H * (long)pitch;
    ref_hist += img * d * B;
    acc += img * H * (long)W;
    if (numer) numer += img * d * H * (long)W;
    const int x = x0 + t;
    const int ty0 = y0 - r, tx0 = x0 - r;  // image coordinates of the tile origin
    const uint32_t Nint = (uint32_t)((2 * r + 1) * (2 * r + 1));
    for (int i = 0; i < g.TH; i++) accS[i * kSW + t] = 0ull;

    const int xl = max(0, x - r), xr = min(W - 1, x + r);
    const int ncols = xr - xl + 1;
    for (int k = k0; k < k1; k++) {
        __syncthreads();
        const uint8_t *bk = bins + (long)k * H * pitch;
        for (int idx = t; idx < g.TR * g.TC; idx += kSW) {
            const int ty = idx / g.TC, tx = idx - ty * g.TC;
            const int gy = ty0 + ty, gx = tx0 + tx;
            int v = 0;
            if (gy >= 0 && gy < H && gx >= 0 && gx < W) v = bk[(long)gy * pitch + gx];
            tile[ty * g.TCp + tx] = (uint8_t)min(v, B - 1);  // out-of-range input bins clamp to B-1
        }
        if (t == 0) {
            uint32_t c = 0;
            for (int b = 0; b < B; b++) {
                c += ref_hist[(long)k * B + b];
                cumR[b] = c;
                cRi[b] = c * Nint;
            }
        }
        for (int b = 0; b < B; b++) hist[b * kSW + t] = 0;
        __syncthreads();
        if (x < W) {
            // window of the band's first row
            const int ya = max(0, y0 - r), yb = min(H - 1, y0 + r);
            for (int yy = ya; yy <= yb; yy++) {
                const uint8_t *row = tile + (yy - ty0) * g.TCp - tx0;
                for (int xx = xl; xx <= xr; xx++) atomicAdd(&hist[row[xx] * kSW + t], 1u);
            }
            for (int i = 0; i < g.TH; i++) {
                const int yy = y0 + i;
                if (yy >= H) break;
                if (i > 0) {
                    const int yo = yy - r - 1, yn = yy + r;
                    if (yo >= 0) {
                        const uint8_t *row = tile + (yo - ty0) * g.TCp - tx0;
                        for (int xx = xl; xx <= xr; xx++) atomicSub(&hist[row[xx] * kSW + t], 1u);
                    }
                    if (yn < H) {
                        const uint8_t *row = tile + (yn - ty0) * g.TCp - tx0;
                        for (int xx = xl; xx <= xr; xx++) atomicAdd(&hist[row[xx] * kSW + t], 1u);
                    }
                }
                const int nrows = min(H - 1, yy + r) - max(0, yy - r) + 1;
                const uint32_t Nloc = (uint32_t)(nrows * ncols);
                ACC D = 0, a = 0;
                if (Nloc == Nint) {
#pragma unroll 4
                    for (int b = 0; b < B; b++) {
                        a += (ACC)hist[b * kSW + t] * (ACC)Nref;
                        const ACC c = (ACC)cRi[b];
                        D += a > c ? a - c : c - a;
                    }
                } else {
#pragma unroll 4
                    for (int b = 0; b < B; b++) {
                        a += (ACC)hist[b * kSW + t] * (ACC)Nref;
                        const ACC c = (ACC)cumR[b] * (ACC)Nloc;
                        D += a > c ? a - c : c - a;
                    }
                }
                accS[i * kSW + t] += (unsigned long long)D;
                if (numer) numer[((long)k * H + yy) * W + x] = (uint64_t)D;
            }
        }
    }
    __syncthreads();
    if (x < W)
        for (int i = 0; i < g.TH; i++) {
            const int yy = y0 + i;
            if (yy >= H) break;
            if (g.n_kg == 1) acc[(long)yy * W + x] = accS[i * kSW + t];
            else atomicAdd(&acc[(long)yy * W + x], accS[i * kSW + t]);
        }
}

// Grid (pixels, images).
__global__ void k_finalize(const unsigned long long *__restrict__ acc, int H, int W, int r, int d, uint32_t Nref,
                           float *__restrict__ score) {
    const long p = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (long)H * W) return;
    acc += (long)blockIdx.y * H * W;
    score += (long)blockIdx.y * H * W;
    const int y = (int)(p / W), x = (int)(p - (long)y * W);
    const int nr = min(H - 1, y + r) - max(0, y - r) + 1;
    const int nc = min(W - 1, x + r) - max(0, x - r) + 1;
    const double den = (double)nr * (double)nc * (double)Nref * (double)d;
    score[p] = (float)((double)acc[p] / den);
}

}  // namespace

size_t score_workspace_bytes(int H, int W, int nimg) {
    return align_up(sizeof(unsigned long long) * (size_t)H * W * nimg, 256);
}

cudaError_t launch_score_ws(const uint8_t *bins, int H, int W, int pitch, int d, int nimg, int B, int r,
                            const uint32_t *ref_hist, uint32_t ref_total, float *score, uint64_t *numer,
                            void *ws, cudaStream_t st) {
    const ScoreGeom g = score_geom(H, W, d, B, r, nimg);
    if (g.smem > 200 * 1024) return cudaErrorNotSupported;  // nothing enqueued
    unsigned long long *acc = (unsigned long long *)ws;
    cudaError_t err = cudaSuccess;
    if (g.n_kg > 1) err = cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * (size_t)H * W * nimg, st);
    if (err != cudaSuccess) return err;
    // u32 walk when every partial and the numerator fit: (B-1) (2r+1)^2 N_ref < 2^32
    const double bound = (double)(B - 1) * (double)((2 * r + 1) * (2 * r + 1)) * (double)ref_total;
    const bool narrow = bound < 4294967295.0 && (double)(2 * r + 1) * (2 * r + 1) * ref_total < 4294967295.0;
    static int attr_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (attr_dev != dev) {
        err = cudaFuncSetAttribute(k_window_emd<uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (err == cudaSuccess)
            err = cudaFuncSetAttribute(k_window_emd<unsigned long long>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       200 * 1024);
        if (err != cudaSuccess) return err;
        attr_dev = dev;
    }
    dim3 grid((W + kSW - 1) / kSW, (H + g.TH - 1) / g.TH, g.n_kg * nimg);
    if (narrow)
        QFCA_LAUNCH("k_window_emd", st,
                    k_window_emd<uint32_t><<<grid, kSW, g.smem, st>>>(bins, H, W, pitch, d, B, r, g, ref_hist,
                                                                       ref_total, acc, numer));
    else
        QFCA_LAUNCH("k_window_emd", st,
                    k_window_emd<unsigned long long><<<grid, kSW, g.smem, st>>>(bins, H, W, pitch, d, B, r, g,
                                                                                 ref_hist, ref_total, acc, numer));
    const long N = (long)H * W;
    QFCA_LAUNCH("k_finalize", st,
                k_finalize<<<dim3((unsigned)((N + 255) / 256), nimg), 256, 0, st>>>(acc, H, W, r, d, ref_total, score));
    return cudaGetLastError();
}

// ---------------------------------------------------------------- allocation-free variant

// Scratch of qfca_score_noalloc: the per-pixel sums of the integer EMD
// numerators, u64 [H][W].  It lives in the module image, so every device that
// loads the library holds it (4 MiB) until the process exits; no call
// allocates anything.
namespace {
constexpr long kNoAllocMaxPixels = 1L << 19;
__device__ __align__(256) unsigned long long g_noalloc_acc[kNoAllocMaxPixels];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
unsigned long long *g_noalloc_ptr[kMaxDevices] = {};
}  // namespace

}  // namespace qfca

extern "C" qfca_status qfca_score_noalloc(const uint8_t *bins, int H, int W, int pitch, int d, int B, int r,
                                          const uint32_t *ref_hist, uint32_t ref_total, float *score,
                                          void *stream) {
    using namespace qfca;
    if (!bins || !ref_hist || !score) return QFCA_ERR_INVALID_ARG;
    if (H < 1 || W < 1 || pitch < W || pitch % 16 != 0) return QFCA_ERR_INVALID_ARG;
    if (d < 1 || d > kMaxD || B < 2 || B > kMaxB || r < 1 || 2 * r + 1 > 127 || ref_total < 1)
        return QFCA_ERR_INVALID_ARG;
    if ((long)H * W > kNoAllocMaxPixels) return QFCA_ERR_UNSUPPORTED;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return QFCA_ERR_CUDA;
    }
    unsigned long long *acc;
    {
        // once per device, with that device current: the device address of the
        // scratch array (in host code the symbol is only a stand-in)
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_acc) != cudaSuccess || !p) {
                cudaGetLastError();
                return QFCA_ERR_CUDA;
            }
            g_noalloc_ptr[dev] = (unsigned long long *)p;
        }
        acc = g_noalloc_ptr[dev];
    }
    const cudaError_t e = launch_score_ws(bins, H, W, pitch, d, 1, B, r, ref_hist, ref_total, score, nullptr, acc,
                                          (cudaStream_t)stream);
    if (e == cudaErrorNotSupported) return QFCA_ERR_UNSUPPORTED;
    if (e != cudaSuccess) {
        cudaGetLastError();
        return QFCA_ERR_CUDA;
    }
    return QFCA_OK;
}
