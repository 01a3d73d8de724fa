// score.cu -- per-pixel sliding-window histograms and the 1-D earth mover's
// distance to the reference histogram, averaged over components (arXiv
// 2510.15602, Sec. 3.1; W1 closed form of the supplement).
//
// For pixel p and component k with clipped window of N_loc pixels:
//     D_k(p) = sum_b |cumP_b * N_ref - cumR_b * N_loc|      (exact integers)
//     score(p) = sum_k D_k(p) / (d * N_loc * N_ref)
//
// k_window_emd: one CTA = a band of TH rows x a strip of SW columns x a group of
// components.  Each component's bin tile (band plus an r-pixel halo) arrives
// in shared memory as one TMA box; the CTA rewrites it in place so that
// in-image pixels hold bin+1 and everything outside the image holds 0.  Each
// thread owns one output column and keeps its window histogram in shared
// memory (bin-major, thread-minor: conflict-free), row 0 counting the
// outside pixels, so every window update touches exactly 2r+1 entries with no
// clipping tests.  The histogram slides down the band (one row leaves, one
// enters: running window counts); the CDF walk is sequential per thread over
// the B bins.  Each numerator D_k(p) is written out (exact, u32 when it
// fits), and k_finalize sums them over k and divides once per pixel.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "internal.cuh"
#include "tc.cuh"

namespace qfca {
namespace {

constexpr int kMaxSW = 128;  // strip width limit (threads per CTA)
constexpr uint32_t kTmaTries = 1u << 26;

struct ScoreGeom {
    int SW, TH, TR, halo, TCp, kg, n_kg;  // TCp: TMA box width (bytes), halo: left margin (16-B aligned)
    size_t smem, tile_bytes;
};

ScoreGeom make_geom(int H, int W, int d, int B, int r, int nimg, int SW, int TH, int n_kg) {
    (void)H, (void)W, (void)nimg;
    ScoreGeom g;
    g.SW = SW;
    g.TH = TH;
    g.TR = TH + 2 * r;
    g.halo = (int)align_up(r, 16);
    g.TCp = SW + 2 * g.halo;
    n_kg = n_kg < 1 ? 1 : (n_kg > d ? d : n_kg);
    g.kg = (d + n_kg - 1) / n_kg;
    g.n_kg = (d + g.kg - 1) / g.kg;
    g.tile_bytes = align_up((size_t)g.TR * g.TCp, 128);
    g.smem = 128                                   // alignment slack
             + 2 * g.tile_bytes                    // bin tiles (double buffer, TMA)
             + sizeof(uint32_t) * (size_t)(B + 1) * SW  // histograms [B+1][SW], row 0 = outside
             + sizeof(uint32_t) * 256              // cumR
             + sizeof(uint64_t) * 256              // cumR * N_loc of an interior window
             + 2 * sizeof(uint64_t);               // mbarriers
    return g;
}

bool geom_ok(const ScoreGeom &g) { return g.smem <= 200 * 1024 && g.TCp <= 256 && g.TR <= 256; }

// Window histograms + exact EMD numerators for a band of TH rows x SW columns
// and a group of components.  Thread t owns output column x0 + t; its window
// histogram lives at hist[b * SW + t].  Increments are shared-memory atomics
// without return, so no thread waits on them.  ACC is the type of the CDF
// walk (u32 when (B-1)(2r+1)^2 N_ref < 2^32), OUT the type of the stored
// numerators; KB > 0 fixes B at compile time.
template <typename ACC, typename OUT, int KB>
__global__ void __launch_bounds__(kMaxSW) k_window_emd(const __grid_constant__ CUtensorMap tmap, int H, int W, int d,
                                                        int Bdyn, int r, ScoreGeom g,
                                                        const uint32_t *__restrict__ ref_hist, uint32_t Nref,
                                                        OUT *__restrict__ numer, unsigned long long *__restrict__ accum,
                                                        int *__restrict__ status) {
    const int B = KB > 0 ? KB : Bdyn;
    const int SW = g.SW;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *smem = tc::align_smem<128>(smem_raw);
    uint8_t *tiles = smem;
    uint32_t *hist = reinterpret_cast<uint32_t *>(smem + 2 * g.tile_bytes);
    uint32_t *cumR = hist + (size_t)(B + 1) * SW;
    ACC *cRi = reinterpret_cast<ACC *>(cumR + 256);  // cumR[b] * N_loc for an interior window
    uint64_t *bar = reinterpret_cast<uint64_t *>(reinterpret_cast<unsigned char *>(cumR + 256) + 256 * sizeof(uint64_t));

    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nwarps = SW >> 5;
    const int x0 = blockIdx.x * SW, y0 = blockIdx.y * g.TH;
    const int x = x0 + t;
    const long img = blockIdx.z / g.n_kg;
    const int k0 = (blockIdx.z % g.n_kg) * g.kg, k1 = min(d, k0 + g.kg);
    ref_hist += img * d * B;
    const long HW = (long)H * W;

    const int ty0 = y0 - r, tx0 = x0 - g.halo;  // image coordinates of the tile origin
    const int span = 2 * r + 1;
    const uint32_t Nint = (uint32_t)(span * span);
    const uint32_t box_bytes = (uint32_t)(g.TR * g.TCp);
    const int wpr = g.TCp >> 2;  // 32-bit words per tile row
    const bool inner = tx0 >= 0 && tx0 + g.TCp <= W && ty0 >= 0 && ty0 + g.TR <= H;
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

    const int ncols = min(W - 1, x + r) - max(0, x - r) + 1;
    const int c0 = t + g.halo - r;  // tile column of this thread's window's left edge
    uint32_t *hc = hist + t;
    for (int k = k0; k < k1; k++) {
        __syncthreads();  // the buffer of component k-1 is free again
        const int buf = (k - k0) & 1;
        if (t == 0 && k + 1 < k1) {
            tc::mbar_arrive_expect_tx(&bar[buf ^ 1], box_bytes);
            tc::tma_load_3d(tiles + (size_t)(buf ^ 1) * g.tile_bytes, &tmap, tx0, ty0, (int)(img * d + k + 1),
                            &bar[buf ^ 1]);
        }
        if (k + 1 < k1) issued++;
        // warp 0: lane l loads reference bins [8l, 8l+8) of component k (in flight during the wait)
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
        // in-image bytes -> min(bin, B-1) + 1, everything else -> 0; a warp per tile row
        {
            uint32_t *tw = reinterpret_cast<uint32_t *>(tile);
            const uint32_t cap = 0x01010101u * (uint32_t)(B - 1);
            for (int row = warp; row < g.TR; row += nwarps) {
                const int gy = ty0 + row;
                const bool rin = gy >= 0 && gy < H;
                for (int j = lane; j < wpr; j += 32) {
                    uint32_t w = __vadd4(__vminu4(tw[row * wpr + j], cap), 0x01010101u);
                    if (!inner) {
                        const int gx = tx0 + 4 * j;
                        const int lo = max(0, -gx), hi = min(4, W - gx);  // bytes [lo, hi) lie in the image
                        uint32_t m = 0;
                        if (rin && hi > lo) m = (hi >= 4 ? 0xFFFFFFFFu : ((1u << (8 * hi)) - 1u)) & (0xFFFFFFFFu << (8 * lo));
                        w &= m;
                    }
                    tw[row * wpr + j] = w;
                }
            }
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
                    cRi[b] = (ACC)c * (ACC)Nint;
                }
            }
        }
        if (KB > 0) {
#pragma unroll
            for (int b = 0; b <= KB; b++) hc[b * SW] = 0;
        } else {
            for (int b = 0; b <= B; b++) hc[b * SW] = 0;
        }
        __syncthreads();
        if (x < W) {
            // window of the band's first row: tile rows 0 .. 2r
            for (int ry = 0; ry < span; ry++) {
                const uint8_t *row = tile + ry * g.TCp + c0;
#pragma unroll 4
                for (int j = 0; j < span; j++) atomicAdd(hc + row[j] * SW, 1u);
            }
            for (int i = 0; i < g.TH; i++) {
                const int yy = y0 + i;
                if (yy >= H) break;
                if (i > 0) {
                    const uint8_t *ro = tile + (i - 1) * g.TCp + c0;       // image row yy - r - 1
                    const uint8_t *rn = tile + (i + 2 * r) * g.TCp + c0;   // image row yy + r
#pragma unroll 4
                    for (int j = 0; j < span; j++) {
                        atomicSub(hc + ro[j] * SW, 1u);
                        atomicAdd(hc + rn[j] * SW, 1u);
                    }
                }
                const int nrows = min(H - 1, yy + r) - max(0, yy - r) + 1;
                const uint32_t Nloc = (uint32_t)(nrows * ncols);
                ACC D = 0;
                uint32_t cnt = 0;
                const uint32_t *hb = hc + SW;  // bin 0
                // the last bin's term is 0 (both CDFs reach 1), so the walk stops at B-2
                if (Nloc == Nint) {
                    if (KB > 0) {
#pragma unroll
                        for (int b = 0; b < KB - 1; b++) {
                            cnt += hb[b * SW];
                            const ACC a = (ACC)cnt * (ACC)Nref, c = cRi[b];
                            D += max(a, c) - min(a, c);
                        }
                    } else {
#pragma unroll 4
                        for (int b = 0; b < B - 1; b++) {
                            cnt += hb[b * SW];
                            const ACC a = (ACC)cnt * (ACC)Nref, c = cRi[b];
                            D += max(a, c) - min(a, c);
                        }
                    }
                } else {
#pragma unroll 4
                    for (int b = 0; b < B - 1; b++) {
                        cnt += hb[b * SW];
                        const ACC a = (ACC)cnt * (ACC)Nref, c = (ACC)cumR[b] * (ACC)Nloc;
                        D += max(a, c) - min(a, c);
                    }
                }
                const long pix = (long)yy * W + x;
                if (accum) atomicAdd(&accum[img * HW + pix], (unsigned long long)D);
                else numer[(img * d + k) * HW + pix] = (OUT)D;
            }
        }
        tc::fence_proxy_async_smem();  // this iteration's writes to the tile precede the next TMA write into it
    }
    if (failed) {
        if (t == 0) atomicOr(status, kStatusMmaTimeout);
        // let every issued copy (including the one whose wait ran out) land before the CTA leaves (bounded)
        for (int w = waited - 1; w < issued; w++) tc::mbar_wait(&bar[w & 1], (w >> 1) & 1, kTmaTries);
    }
}

// Grid (pixels, images): s(p) = sum_k D_k(p) / (d * N_loc * N_ref), from the
// per-component numerators or from their running sums.
template <typename OUT>
__global__ void k_finalize(const OUT *__restrict__ numer, const unsigned long long *__restrict__ accum, int H, int W,
                           int r, int d, uint32_t Nref, float *__restrict__ score) {
    const long p = (long)blockIdx.x * blockDim.x + threadIdx.x;
    const long HW = (long)H * W;
    if (p >= HW) return;
    const long img = blockIdx.y;
    unsigned long long s = 0;
    if (accum) {
        s = accum[img * HW + p];
    } else {
        const OUT *nk = numer + img * d * HW + p;
        for (int k = 0; k < d; k++) s += (unsigned long long)__ldg(nk + (long)k * HW);
    }
    const int y = (int)(p / W), x = (int)(p - (long)y * W);
    const int nr = min(H - 1, y + r) - max(0, y - r) + 1;
    const int nc = min(W - 1, x + r) - max(0, x - r) + 1;
    const double den = (double)nr * (double)nc * (double)Nref * (double)d;
    score[img * HW + p] = (float)((double)s / den);
}

template <typename ACC, typename OUT>
cudaError_t launch_emd_kb(int KB, const ScoreGeom &g, dim3 grid, cudaStream_t st, const CUtensorMap &tmap, int H,
                          int W, int d, int B, int r, const uint32_t *ref_hist, uint32_t Nref, OUT *numer,
                          unsigned long long *accum, int *status) {
    if (KB == 32)
        QFCA_LAUNCH("k_window_emd", st,
                    (k_window_emd<ACC, OUT, 32><<<grid, g.SW, g.smem, st>>>(tmap, H, W, d, B, r, g, ref_hist, Nref,
                                                                             numer, accum, status)));
    else if (KB == 64)
        QFCA_LAUNCH("k_window_emd", st,
                    (k_window_emd<ACC, OUT, 64><<<grid, g.SW, g.smem, st>>>(tmap, H, W, d, B, r, g, ref_hist, Nref,
                                                                             numer, accum, status)));
    else
        QFCA_LAUNCH("k_window_emd", st,
                    (k_window_emd<ACC, OUT, 0><<<grid, g.SW, g.smem, st>>>(tmap, H, W, d, B, r, g, ref_hist, Nref,
                                                                            numer, accum, status)));
    return cudaSuccess;
}

template <typename ACC, typename OUT>
cudaError_t emd_occupancy(int KB, size_t smem, int SW, int *per_sm) {
    if (KB == 32) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_window_emd<ACC, OUT, 32>, SW, smem);
    if (KB == 64) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_window_emd<ACC, OUT, 64>, SW, smem);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_window_emd<ACC, OUT, 0>, SW, smem);
}

template <typename ACC, typename OUT>
cudaError_t emd_set_smem_attr() {
    cudaError_t e = cudaFuncSetAttribute(k_window_emd<ACC, OUT, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         200 * 1024);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_window_emd<ACC, OUT, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_window_emd<ACC, OUT, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    return e;
}

enum class EmdKind { U32_U32, U32_U64, U64_U64 };

cudaError_t emd_occupancy_kind(EmdKind kind, int KB, size_t smem, int SW, int *per_sm) {
    switch (kind) {
    case EmdKind::U32_U32: return emd_occupancy<uint32_t, uint32_t>(KB, smem, SW, per_sm);
    case EmdKind::U32_U64: return emd_occupancy<uint32_t, unsigned long long>(KB, smem, SW, per_sm);
    default: return emd_occupancy<unsigned long long, unsigned long long>(KB, smem, SW, per_sm);
    }
}

// Modelled cost (in lane-instructions) of one CTA and the choice of strip
// width, band height and component split that finishes the grid soonest.
double cta_cost(const ScoreGeom &g, int B, int r) {
    const int span = 2 * r + 1;
    const double row = 2.0 * span * 3.0 + 5.0 * (B - 1) + 12.0;
    const double setup = 3.0 * span * span + 6.0 * g.TR * g.TCp / (4.0 * g.SW) + 2.0 * B + 60.0;
    return g.kg * (g.TH * row + setup) + 200.0;
}

}  // namespace

size_t score_workspace_bytes(int H, int W, int d, int nimg) {
    return align_up(sizeof(unsigned long long) * (size_t)H * W * d * nimg, 256);
}

cudaError_t launch_score_ws(const uint8_t *bins, int H, int W, int pitch, int d, int nimg, int B, int r,
                            const uint32_t *ref_hist, uint32_t ref_total, float *score, uint64_t *numer_out,
                            void *ws, bool ws_accumulates, int *status, cudaStream_t st, const ScoreTiling *tiling) {
    // u32 walk when every partial and the numerator fit: (B-1) (2r+1)^2 N_ref < 2^32
    const double span2 = (double)(2 * r + 1) * (2 * r + 1);
    const bool narrow = (double)(B - 1) * span2 * (double)ref_total < 4294967295.0 && span2 * ref_total < 4294967295.0;
    const EmdKind kind = !narrow ? EmdKind::U64_U64
                         : (numer_out || ws_accumulates) ? EmdKind::U32_U64 : EmdKind::U32_U32;
    const int KB = (B == 32 || B == 64) ? B : 0;
    static int attr_dev = -1, n_sm = 0;
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    if (attr_dev != dev) {
        err = emd_set_smem_attr<uint32_t, uint32_t>();
        if (err == cudaSuccess) err = emd_set_smem_attr<uint32_t, unsigned long long>();
        if (err == cudaSuccess) err = emd_set_smem_attr<unsigned long long, unsigned long long>();
        if (err == cudaSuccess) err = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        if (err != cudaSuccess) return err;
        attr_dev = dev;
    }
    // geometry: the caller's tiling, else the modelled best over strip widths, band heights and splits
    ScoreGeom g{};
    bool have = false;
    if (tiling && tiling->SW > 0) {
        g = make_geom(H, W, d, B, r, nimg, tiling->SW, tiling->TH, tiling->n_kg);
        have = geom_ok(g) && (g.SW == 64 || g.SW == 128) && g.TH >= 1 && g.TH <= 64 && (long)g.n_kg * nimg <= 65535;
        if (!have) return cudaErrorNotSupported;
    } else {
        double best = 1e300;
        for (int SW : {128, 64})
            for (int TH : {16, 32, 8}) {
                const ScoreGeom g0 = make_geom(H, W, d, B, r, nimg, SW, TH, 1);
                if (!geom_ok(g0)) continue;
                int per_sm = 0;
                err = emd_occupancy_kind(kind, KB, g0.smem, SW, &per_sm);
                if (err != cudaSuccess) return err;
                if (per_sm < 1) continue;
                const long slots = (long)per_sm * n_sm;
                const long tiles = (long)((W + SW - 1) / SW) * ((H + TH - 1) / TH) * nimg;
                for (int n = 1; n <= d && (long)n * nimg <= 65535; n++) {
                    const ScoreGeom gn = make_geom(H, W, d, B, r, nimg, SW, TH, n);
                    if (gn.n_kg != n) continue;
                    const double waves = (double)((tiles * n + slots - 1) / slots);
                    const double cost = waves * cta_cost(gn, B, r);
                    if (cost < best * 0.999) best = cost, g = gn, have = true;
                }
            }
        if (!have) return cudaErrorNotSupported;  // nothing enqueued
    }
    alignas(64) CUtensorMap tmap;
    err = make_tmap_u8_3d(&tmap, bins, (uint64_t)pitch, (uint64_t)H, (uint64_t)nimg * d, (uint64_t)pitch,
                          (uint64_t)H * pitch, (uint32_t)g.TCp, (uint32_t)g.TR);
    if (err != cudaSuccess) return err;
    unsigned long long *accum = ws_accumulates ? (unsigned long long *)ws : nullptr;
    if (accum) err = cudaMemsetAsync(accum, 0, sizeof(unsigned long long) * (size_t)H * W * nimg, st);
    if (err != cudaSuccess) return err;
    const dim3 grid((W + g.SW - 1) / g.SW, (H + g.TH - 1) / g.TH, g.n_kg * nimg);
    const long N = (long)H * W;
    const dim3 fgrid((unsigned)((N + 255) / 256), nimg);
    switch (kind) {
    case EmdKind::U32_U32: {
        uint32_t *nm = (uint32_t *)ws;
        launch_emd_kb<uint32_t, uint32_t>(KB, g, grid, st, tmap, H, W, d, B, r, ref_hist, ref_total, nm, nullptr,
                                          status);
        QFCA_LAUNCH("k_finalize", st,
                    k_finalize<uint32_t><<<fgrid, 256, 0, st>>>(nm, nullptr, H, W, r, d, ref_total, score));
        break;
    }
    case EmdKind::U32_U64: {
        unsigned long long *nm = accum ? nullptr : (unsigned long long *)(numer_out ? (void *)numer_out : ws);
        launch_emd_kb<uint32_t, unsigned long long>(KB, g, grid, st, tmap, H, W, d, B, r, ref_hist, ref_total, nm,
                                                    accum, status);
        QFCA_LAUNCH("k_finalize", st,
                    k_finalize<unsigned long long><<<fgrid, 256, 0, st>>>(nm, accum, H, W, r, d, ref_total, score));
        break;
    }
    default: {
        unsigned long long *nm = accum ? nullptr : (unsigned long long *)(numer_out ? (void *)numer_out : ws);
        launch_emd_kb<unsigned long long, unsigned long long>(KB, g, grid, st, tmap, H, W, d, B, r, ref_hist,
                                                              ref_total, nm, accum, status);
        QFCA_LAUNCH("k_finalize", st,
                    k_finalize<unsigned long long><<<fgrid, 256, 0, st>>>(nm, accum, H, W, r, d, ref_total, score));
        break;
    }
    }
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
                                          true, g_noalloc_status[dev], (cudaStream_t)stream, nullptr);
    if (e == cudaErrorNotSupported) return QFCA_ERR_UNSUPPORTED;
    if (e != cudaSuccess) {
        cudaGetLastError();
        return QFCA_ERR_CUDA;
    }
    return QFCA_OK;
}
