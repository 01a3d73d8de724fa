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
#include "tc.cuh"

namespace qfca {
namespace {

constexpr int kSW = 128;  // output columns per CTA (one thread each)
constexpr int kTH = 16;   // output rows per CTA band

struct ScoreGeom {
    int TH, TR, halo, TCp, kg, n_kg;  // TCp: TMA box width (bytes), halo: left margin (16-B aligned)
    size_t smem, tile_bytes;
};

constexpr uint32_t kTmaTries = 1u << 26;

// `slots`: CTAs resident at once on the whole GPU (0: geometry only).  The
// components are split into n_kg groups so that the waves of CTAs, each
// costing its number of components plus a fixed setup share, finish soonest.
ScoreGeom score_geom(int H, int W, int d, int B, int r, int nimg, long slots) {
    ScoreGeom g;
    g.TH = kTH;
    g.TR = g.TH + 2 * r;
    g.halo = (int)align_up(r, 16);
    g.TCp = kSW + 2 * g.halo;
    const long tiles = (long)((W + kSW - 1) / kSW) * ((H + g.TH - 1) / g.TH) * nimg;
    int n_kg = 1;
    if (slots > 0) {
        double best = 1e300;
        for (int n = 1; n <= d; n++) {
            const int kg = (d + n - 1) / n;
            if (n > 1 && (d + kg - 1) / kg != n) continue;  // same split as a smaller n
            const double waves = (double)((tiles * n + slots - 1) / slots);
            const double cost = waves * (kg + 0.5);
            if (cost < best * 0.999) best = cost, n_kg = n;
        }
    }
    g.kg = (d + n_kg - 1) / n_kg;
    g.n_kg = (d + g.kg - 1) / g.kg;
    g.tile_bytes = align_up((size_t)g.TR * g.TCp, 128);
    g.smem = 128                                                // alignment slack
             + 2 * g.tile_bytes                                 // bin tiles (double buffer, TMA)
             + sizeof(uint32_t) * (size_t)B * kSW                 // histograms [B][kSW]
             + sizeof(unsigned long long) * (size_t)g.TH * kSW  // per-pixel sums
             + 2 * sizeof(uint32_t) * 256                       // cumR, cumR * N_loc(interior)
             + 2 * sizeof(uint64_t);                            // mbarriers
    return g;
}

// Window histograms + exact EMD numerators for a band of kTH rows x kSW columns
// and a group of components.  Thread t owns output column x0 + t: its window
// histogram lives in shared memory at hist[b * kSW + t] (conflict-free), and
// slides down the band (one row of 2r+1 bins leaves, one enters); increments
// are shared-memory atomics without return, so no thread waits on them.
// ACC is the type of the CDF walk: uint32_t when (B-1)(2r+1)^2 N_ref < 2^32
// (the numerator D and every term then fit), else unsigned long long.
// The band's bin tile of each component (rows y0-r .. y0+TH-1+r, columns from
// x0 - halo, halo = r rounded up to 16 bytes) is one 3-D TMA box of the bins
// tensor [images*d][H][pitch]; boxes are double-buffered so the next
// component's tile arrives while the current one is processed.  Waits are
// bounded; a wait that runs out sets bit 0 of the status word and the CTA stops.
template <typename ACC>
__global__ void __launch_bounds__(kSW) k_window_emd(const __grid_constant__ CUtensorMap tmap, int H, int W, int d,
                                                     int B, int r, ScoreGeom g, const uint32_t *__restrict__ ref_hist,
                                                     uint32_t Nref, unsigned long long *__restrict__ acc,
                                                     uint64_t *__restrict__ numer, int *__restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    uint8_t *tiles = smem;
    uint32_t *hist = reinterpret_cast<uint32_t *>(smem + 2 * g.tile_bytes);
    unsigned long long *accS = reinterpret_cast<unsigned long long *>(hist + (size_t)B * kSW);
    uint32_t *cumR = reinterpret_cast<uint32_t *>(accS + (size_t)g.TH * kSW);
    uint32_t *cRi = cumR + 256;  // cumR[b] * N_loc for an interior window
    uint64_t *bar = reinterpret_cast<uint64_t *>(cRi + 256);

    const int t = threadIdx.x;
    const int x0 = blockIdx.x * kSW, y0 = blockIdx.y * g.TH;
    const long img = blockIdx.z / g.n_kg;
    const int k0 = (blockIdx.z % g.n_kg) * g.kg, k1 = min(d, k0 + g.kg);
    ref_hist += img * d * B;
    acc += img * H * (long)W;
    if (numer) numer += img * d * H * (long)W;
    const int x = x0 + t;
    const int ty0 = y0 - r, tx0 = x0 - g.halo;  // image coordinates of the tile origin
    const uint32_t Nint = (uint32_t)((2 * r + 1) * (2 * r + 1));
    const uint32_t box_bytes = (uint32_t)(g.TR * g.TCp);
    for (int i = 0; i < g.TH; i++) accS[i * kSW + t] = 0ull;
    if (t == 0) {
        tc::mbar_init(&bar[0], 1);
        tc::mbar_init(&bar[1], 1);
        tc::fence_mbar_init();
    }
    __syncthreads();
    if (t == 0 && k0 < k1) {
        tc::mbar_arrive_expect_tx(&bar[0], box_bytes);
        tc::tma_load_3d(tiles, &tmap, tx0, ty0, (int)(img * d + k0), &bar[0]);
    }
    bool failed = false;
    int issued = k0 < k1 ? 1 : 0, waited = 0;

    const int xl = max(0, x - r), xr = min(W - 1, x + r);
    const int ncols = xr - xl + 1;
    for (int k = k0; k < k1; k++) {
        __syncthreads();  // the buffer of component k-1 is free again
        const int buf = (k - k0) & 1;
        if (t == 0 && k + 1 < k1) {
            tc::mbar_arrive_expect_tx(&bar[buf ^ 1], box_bytes);
            tc::tma_load_3d(tiles + (size_t)(buf ^ 1) * g.tile_bytes, &tmap, tx0, ty0, (int)(img * d + k + 1),
                            &bar[buf ^ 1]);
        }
        if (k + 1 < k1) issued++;
        // warp 0: lane l loads reference bins [8l, 8l+8) of component k (independent loads, in flight during the wait)
        uint32_t rv[8];
        if (t < 32) {
#pragma unroll
            for (int j = 0; j < 8; j++) {
                const int b = 8 * t + j;
                rv[j] = b < B ? __ldg(&ref_hist[(long)k * B + b]) : 0u;
            }
        }
        const bool ok = tc::mbar_wait(&bar[buf], ((k - k0) >> 1) & 1, kTmaTries);
        waited++;
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        uint8_t *tile = tiles + (size_t)buf * g.tile_bytes;
        // clamp out-of-range input bins to B-1, four bytes at a time
        {
            uint32_t *tw = reinterpret_cast<uint32_t *>(tile);
            const uint32_t cap = 0x01010101u * (uint32_t)(B - 1);
            for (int i = t; i < (int)(box_bytes >> 2); i += kSW) tw[i] = __vminu4(tw[i], cap);
        }
        if (t < 32) {  // whole warp 0: prefix sums of the reference histogram
            uint32_t part = 0;
#pragma unroll
            for (int j = 0; j < 8; j++) part += rv[j];
            uint32_t incl = part;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t n = __shfl_up_sync(0xffffffffu, incl, o);
                if (t >= o) incl += n;
            }
            uint32_t c = incl - part;
#pragma unroll
            for (int j = 0; j < 8; j++) {
                const int b = 8 * t + j;
                c += rv[j];
                if (b < B) {
                    cumR[b] = c;
                    cRi[b] = c * Nint;
                }
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
        tc::fence_proxy_async_smem();  // the clamp's writes precede the next TMA write into this buffer
    }
    if (failed) {
        if (t == 0) atomicOr(status, kStatusMmaTimeout);
        // let every issued copy (including the one whose wait ran out) land before the CTA leaves (bounded)
        for (int w = waited - 1; w < issued; w++) tc::mbar_wait(&bar[w & 1], (w >> 1) & 1, kTmaTries);
        return;
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
                            void *ws, int *status, cudaStream_t st) {
    const ScoreGeom g0 = score_geom(H, W, d, B, r, nimg, 0);
    if (g0.smem > 200 * 1024 || g0.TCp > 256 || g0.TR > 256) return cudaErrorNotSupported;  // nothing enqueued
    alignas(64) CUtensorMap tmap;
    cudaError_t err = make_tmap_u8_3d(&tmap, bins, (uint64_t)pitch, (uint64_t)H, (uint64_t)nimg * d, (uint64_t)pitch,
                                      (uint64_t)H * pitch, (uint32_t)g0.TCp, (uint32_t)g0.TR);
    if (err != cudaSuccess) return err;
    // u32 walk when every partial and the numerator fit: (B-1) (2r+1)^2 N_ref < 2^32
    const double bound = (double)(B - 1) * (double)((2 * r + 1) * (2 * r + 1)) * (double)ref_total;
    const bool narrow = bound < 4294967295.0 && (double)(2 * r + 1) * (2 * r + 1) * ref_total < 4294967295.0;
    static int attr_dev = -1, n_sm = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (attr_dev != dev) {
        err = cudaFuncSetAttribute(k_window_emd<uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (err == cudaSuccess)
            err = cudaFuncSetAttribute(k_window_emd<unsigned long long>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       200 * 1024);
        if (err == cudaSuccess) err = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        if (err != cudaSuccess) return err;
        attr_dev = dev;
    }
    int per_sm = 0;
    err = narrow ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_window_emd<uint32_t>, kSW, g0.smem)
                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_window_emd<unsigned long long>, kSW,
                                                                 g0.smem);
    if (err != cudaSuccess) return err;
    const ScoreGeom g = score_geom(H, W, d, B, r, nimg, (long)max(per_sm, 1) * n_sm);
    unsigned long long *acc = (unsigned long long *)ws;
    if (g.n_kg > 1) err = cudaMemsetAsync(acc, 0, sizeof(unsigned long long) * (size_t)H * W * nimg, st);
    if (err != cudaSuccess) return err;
    dim3 grid((W + kSW - 1) / kSW, (H + g.TH - 1) / g.TH, g.n_kg * nimg);
    if (narrow)
        QFCA_LAUNCH("k_window_emd", st,
                    k_window_emd<uint32_t><<<grid, kSW, g.smem, st>>>(tmap, H, W, d, B, r, g, ref_hist, ref_total, acc,
                                                                       numer, status));
    else
        QFCA_LAUNCH("k_window_emd", st,
                    k_window_emd<unsigned long long><<<grid, kSW, g.smem, st>>>(tmap, H, W, d, B, r, g, ref_hist,
                                                                                 ref_total, acc, numer, status));
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
__device__ int g_noalloc_flag;  // bounded-wait status of the variant's kernels

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
unsigned long long *g_noalloc_ptr[kMaxDevices] = {};
int *g_noalloc_status[kMaxDevices] = {};
}  // namespace

}  // namespace qfca

extern "C" qfca_status qfca_score_noalloc(const uint8_t *bins, int H, int W, int pitch, int d, int B, int r,
                                          const uint32_t *ref_hist, uint32_t ref_total, float *score,
                                          void *stream) {
    using namespace qfca;
    if (!bins || !ref_hist || !score) return QFCA_ERR_INVALID_ARG;
    if (H < 1 || W < 1 || pitch < W || pitch % 16 != 0 || ((uintptr_t)bins & 15) != 0) return QFCA_ERR_INVALID_ARG;
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
            void *p = nullptr, *f = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_acc) != cudaSuccess || !p ||
                cudaGetSymbolAddress(&f, g_noalloc_flag) != cudaSuccess || !f) {
                cudaGetLastError();
                return QFCA_ERR_CUDA;
            }
            g_noalloc_ptr[dev] = (unsigned long long *)p;
            g_noalloc_status[dev] = (int *)f;
        }
        acc = g_noalloc_ptr[dev];
    }
    const cudaError_t e = launch_score_ws(bins, H, W, pitch, d, 1, B, r, ref_hist, ref_total, score, nullptr, acc,
                                          g_noalloc_status[dev], (cudaStream_t)stream);
    if (e == cudaErrorNotSupported) return QFCA_ERR_UNSUPPORTED;
    if (e != cudaSuccess) {
        cudaGetLastError();
        return QFCA_ERR_CUDA;
    }
    return QFCA_OK;
}
