// project_tma.cu -- BF16 principal-component projection Y = (X - mean) V
// (arXiv 2510.15602, Sec. 3.3) as a warp-specialised TMA / tcgen05 pipeline
// over a table of images of any size (one launch for up to 64 images).
//
// The projection reads each FP32 feature once and does 2d flops per byte, so
// it is bound by HBM bandwidth; the design keeps HBM busy.  One persistent CTA
// per SM owns a contiguous range of the table's 128-pixel tiles; a tile is
// processed in K-chunks of 64 channels.  Roles (14 warps), synchronised only
// through mbarriers:
//   - warp 0: TMA producer.  Keeps a ring of `stages` 32 KB boxes (64 channels
//     x 128 pixels of FP32, zero-filled beyond the image and beyond C) in
//     flight; a stage is refilled once the converters have read it.
//   - warp 1: MMA issuer.  For each converted chunk, 4 tcgen05.mma (M=128,
//     N=DT, K=16) into one of two tensor-memory accumulators (tiles
//     alternate), then tcgen05.commit to release the operand buffer; after a
//     tile's last chunk, a commit hands the accumulator to the epilogue.
//   - warps 2-9: converters.  Read a landed box, release the stage, centre by
//     the mean, convert to BF16 into the 128-byte swizzled K-major operand
//     layout (a ring of operand buffers), hand the chunk to the MMA warp.  At
//     an image change they wait for the MMAs in flight and reload V^T (BF16,
//     DT x Cp) and the FP32 mean into shared memory.
//   - warps 10-13: epilogue, one per accumulator lane quarter: read the
//     accumulator back (tcgen05.ld, 16 columns at a time), write Y [d][N]
//     coalesced, fold each 16-column group's min/max over the warp's 32
//     pixels with a halving shuffle reduction (lane L ends up owning column
//     (L >> 1) & 15 of the group), keep running values per lane and flush
//     them once per image as u32 keys, and release the accumulator; this
//     overlaps the next tile's conversion and MMAs.
// Every role keeps its warps converged (one lane issues) and every wait is
// bounded and watches a CTA-wide abort flag; a wait that runs out sets bit 0
// of the status word and the flag, every role leaves its loop (still passing
// its named barriers), the copies and MMAs in flight drain (bounded), tensor
// memory is freed and the CTA returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.cuh"
#include "tc.cuh"

namespace qfca {
namespace {

constexpr int kM = 128;        // pixels per tile (MMA M)
constexpr int kKc = 64;        // channels per K-chunk / TMA box (one 128-B swizzle row of BF16)
constexpr int kConv = 256;     // converter threads (warps 2-9)
constexpr int kEpi = 128;      // epilogue threads (warps 10-13)
constexpr int kThreads = 64 + kConv + kEpi;
constexpr int kMaxStages = 5;
constexpr int kMaxA = 4;       // operand buffers (chunks converted ahead of the MMAs)
constexpr uint32_t kStageBytes = kKc * kM * 4;  // 32 KB of FP32
constexpr uint32_t kAChunk = kM * 128;           // 16 KB of BF16
constexpr uint32_t kTries = 1u << 26;

struct ProjImgP {
    long N, tile0;
    const float *mean32;            // [Cp]
    const void *Vt;                 // BF16 [DT][Cp]; FP8: e4m3 hi [DT][Cp] then lo [DT][Cp]
    const float *scale;             // FP8: per-channel power-of-two scale s_c [Cp]
    const float *colscale;          // FP8: per-component power-of-two 1/t_j [DT]
    float *Y;                       // [d][N]
    uint32_t *mm;                   // [2 d kKeyStride]
    const float *qlo, *qhi;         // fixed range [d] when the epilogue quantises (bins != NULL)
    uint8_t *bins;                  // [d][N / W][pitch] or NULL
    int W, pitch, B;
};

struct ProjParams {
    int n, C, Cp, nk, d, stages, na;
    long total_tiles;
    ProjImgP img[kMaxBatch];
    CUtensorMap tmap[kMaxBatch];    // X of image i as [C][N] FP32, box {128 pixels, 64 channels}
};

__device__ __forceinline__ uint32_t swz_off(int row, int chunk16) {
    return (uint32_t)(row * 128 + ((chunk16 ^ (row & 7)) << 4));
}

// The image of tile w, searched forward from image `from` (a role walks its tiles in increasing
// order, so it passes each image boundary once: O(1) per tile instead of a scan of the table --
// the scan, up to 64 dependent parameter loads per box in the producer thread, had made the
// kernel's time grow with the number of images in the table).
__device__ __forceinline__ int find_img(const ProjParams &p, long w, int from) {
    int i = from < 0 ? 0 : from;
    while (i + 1 < p.n && p.img[i + 1].tile0 <= w) i++;
    return i;
}

// Bounded wait that also gives up when another role has aborted; a wait that
// runs out raises the abort flag itself.
__device__ __forceinline__ bool wait_or_abort(uint64_t *bar, uint32_t parity, volatile int *abort_flag) {
    for (uint32_t i = 0; i < kTries; i++) {
        if (tc::mbar_try_wait(bar, parity)) return true;
        if ((i & 255) == 255 && *abort_flag) return false;
    }
    *abort_flag = 1;
    return false;
}

// Warp-wide bounded wait: every lane probes (and so acquires the completed
// phase); the result is agreed across the warp.
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag) {
    return __all_sync(0xffffffffu, wait_or_abort(bar, parity, abort_flag));
}

// Min (or max) of 16 values per lane over the 32 lanes of a warp, halving
// the data at each exchange: on return v[0] of lane L holds the reduction of
// value (L >> 1) & 15 over all lanes.  NaN inputs are ignored (fminf/fmaxf).
template <bool kMin>
__device__ __forceinline__ void warp_reduce16(float (&v)[16]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16, h = 8; o >= 2; o >>= 1, h >>= 1) {
        const bool up = (lane & o) != 0;  // this lane keeps the upper half of its values
#pragma unroll
        for (int i = 0; i < h; i++) {
            const float send = up ? v[i] : v[i + h];
            const float keep = up ? v[i + h] : v[i];
            const float recv = __shfl_xor_sync(0xffffffffu, send, o);
            v[i] = kMin ? fminf(keep, recv) : fmaxf(keep, recv);
        }
    }
    const float recv = __shfl_xor_sync(0xffffffffu, v[0], 1);
    v[0] = kMin ? fminf(v[0], recv) : fmaxf(v[0], recv);
}

__device__ __forceinline__ void conv_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kConv) : "memory"); }
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 2, %0;" ::"n"(kEpi) : "memory"); }

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(bar)) : "memory");
}

struct SmemLayout {
    size_t stage, a, b, mean, bar, total;
};

__host__ __device__ inline SmemLayout smem_layout(int stages, int na, int Cp, int DT, bool f8) {
    SmemLayout L;
    size_t o = 0;
    L.stage = o;
    o += (size_t)stages * kStageBytes;
    L.a = o;
    o += (size_t)na * kAChunk;
    L.b = o;
    o += f8 ? 2 * (size_t)Cp * DT : (size_t)(Cp / kKc) * DT * 128;  // FP8: hi and lo, 128 channels per 128-B row
    L.mean = o;
    o += (f8 ? 2 : 1) * sizeof(float) * (size_t)Cp;                // mean (and FP8 scale)
    L.bar = o;
    o += 8 * (2 * kMaxStages + 2 * kMaxA + 4) + 16 + 2 * 4 * 64;  // barriers, tmem slot + abort flag, kmin/kmax
    L.total = o + 1024;                                // alignment slack
    return L;
}

// F8: A = e4m3((x - mean) s_c), B = e4m3 hi + lo of V^T / s_c scaled by t_j per
// component, kind::f8f6f4 MMAs (K = 32) over 128-channel K-chunks, each
// assembled from two 64-channel boxes; the epilogue multiplies by 1/t_j.
template <int DT, bool F8>
__global__ void __launch_bounds__(kThreads, 1) k_project_tma(const __grid_constant__ ProjParams p,
                                                            int *__restrict__ status) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = tc::align_smem<1024>(smem_raw);
    const SmemLayout L = smem_layout(p.stages, p.na, p.Cp, DT, F8);
    uint8_t *stage = smem + L.stage;
    uint8_t *As = smem + L.a;
    uint8_t *Bs = smem + L.b;
    float *mean_s = reinterpret_cast<float *>(smem + L.mean);
    float *scale_s = mean_s + p.Cp;  // FP8 only
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + L.bar);  // [kMaxStages] TMA landed
    uint64_t *empty = full + kMaxStages;                            // [kMaxStages] converters done with a stage
    uint64_t *a_full = empty + kMaxStages;                          // [kMaxA] operand chunk converted
    uint64_t *a_empty = a_full + kMaxA;                             // [kMaxA] MMAs of a chunk complete
    uint64_t *acc_full = a_empty + kMaxA;                           // [2] tile's MMAs complete
    uint64_t *acc_empty = acc_full + 2;                             // [2] accumulator read back
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acc_empty + 2);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    uint32_t *kmin = tmem_slot + 4;  // [64]
    uint32_t *kmax = kmin + 64;      // [64]
    constexpr uint32_t kCols = 2 * DT < 32 ? 32 : 2 * DT;  // two accumulators

    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int nk = p.nk, S = p.stages, NA = p.na, d = p.d;
    if (warp == 0) {
        tc::tmem_alloc(tmem_slot, kCols);
        tc::tmem_relinquish();
    }
    if (t == 32) {
        for (int s = 0; s < kMaxStages; s++) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], kConv / 32);
        }
        for (int b = 0; b < kMaxA; b++) {
            tc::mbar_init(&a_full[b], (F8 ? 2 : 1) * kConv / 32);  // FP8: two boxes per operand chunk
            tc::mbar_init(&a_empty[b], 1);
        }
        for (int b = 0; b < 2; b++) {
            tc::mbar_init(&acc_full[b], 1);
            tc::mbar_init(&acc_empty[b], kEpi / 32);
        }
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    if (t < 64) { kmin[t] = 0xffffffffu; kmax[t] = 0u; }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    // this CTA's contiguous range of tiles
    const long T = p.total_tiles, G = gridDim.x;
    const long w0 = T * blockIdx.x / G, w1 = T * (blockIdx.x + 1) / G;
    const long n_chunks = (w1 - w0) * nk;

    // Every role keeps its whole warp converged (one lane issues), and after an
    // abort the converters still pass every named barrier, so no thread can be
    // left waiting at a barrier or a .sync.aligned instruction.
    if (warp == 0) {
        // ---------------------------------------------------------------- TMA producer
        long q = 0;
        int pimg = -1;
        for (; q < n_chunks; q++) {
            const int s = (int)(q % S);
            const bool ok = q < S || warp_wait(&empty[s], (uint32_t)((q / S - 1) & 1), abort_flag);
            if (!ok) break;
            if (lane == 0) {
                const long w = w0 + q / nk;
                const int kc = (int)(q % nk);
                const int i = pimg = find_img(p, w, pimg);
                tc::mbar_arrive_expect_tx(&full[s], kStageBytes);
                tc::tma_load_2d(stage + (size_t)s * kStageBytes, &p.tmap[i], (int)((w - p.img[i].tile0) * kM),
                                kc * kKc, &full[s]);
            }
            __syncwarp();
        }
        if (*abort_flag && lane == 0) {
            // bounded drain of the copies that may still be landing
            for (long r = (q > S ? q - S : 0); r < q; r++) tc::mbar_wait(&full[r % S], (uint32_t)((r / S) & 1), kTries);
        }
    } else if (warp == 1) {
        // ---------------------------------------------------------------- MMA issuer
        const uint32_t idesc = F8 ? tc::idesc_e4m3_f32(kM, DT) : tc::idesc_bf16_f32(kM, DT);
        const uint32_t a_base = tc::smem_u32(As), b_base = tc::smem_u32(Bs);
        const int nq = F8 ? nk / 2 : nk;  // operand chunks per tile
        long q = 0, last_commit = -1;
        bool ok = true;
        for (long tile = 0; ok && tile < w1 - w0; tile++) {
            const int ac = (int)(tile & 1);
            if (tile >= 2) ok = warp_wait(&acc_empty[ac], (uint32_t)((tile / 2 - 1) & 1), abort_flag);
            for (int kc = 0; ok && kc < nq; kc++, q++) {
                const int ab = (int)(q % NA);
                ok = warp_wait(&a_full[ab], (uint32_t)((q / NA) & 1), abort_flag);
                if (!ok) break;
                tc::tc_fence_after();
                if (lane == 0) {
                    const uint32_t a0 = a_base + (uint32_t)ab * kAChunk, b0 = b_base + (uint32_t)kc * DT * 128;
                    if (F8) {
                        const uint32_t b1 = b0 + (uint32_t)(p.Cp * DT);  // lo part
#pragma unroll
                        for (int ks = 0; ks < 4; ks++) {
                            tc::mma_f8_ss(tmem + (uint32_t)(ac * DT), tc::sdesc_kmajor_sw128(a0 + ks * 32),
                                          tc::sdesc_kmajor_sw128(b0 + ks * 32), idesc, (kc > 0 || ks > 0) ? 1u : 0u);
                            tc::mma_f8_ss(tmem + (uint32_t)(ac * DT), tc::sdesc_kmajor_sw128(a0 + ks * 32),
                                          tc::sdesc_kmajor_sw128(b1 + ks * 32), idesc, 1u);
                        }
                    } else {
#pragma unroll
                        for (int ks = 0; ks < 4; ks++)
                            tc::mma_bf16_ss(tmem + (uint32_t)(ac * DT), tc::sdesc_kmajor_sw128(a0 + ks * 32),
                                            tc::sdesc_kmajor_sw128(b0 + ks * 32), idesc, (kc > 0 || ks > 0) ? 1u : 0u);
                    }
                    tc::mma_commit(&a_empty[ab]);
                    if (kc == nq - 1) tc::mma_commit(&acc_full[ac]);
                }
                __syncwarp();
                last_commit = q;
            }
        }
        if (*abort_flag && last_commit >= 0 && lane == 0)  // bounded drain of the MMAs in flight
            tc::mbar_wait(&a_empty[last_commit % NA], (uint32_t)((last_commit / NA) & 1), kTries);
    } else if (warp < 10) {
        // ---------------------------------------------------------------- converters
        const int ct = t - 64;
        const int m = ct & (kM - 1), h = ct >> 7;  // pixel row m, channels [32 h, 32 h + 32) of a chunk
        int cur = -1;
        long q = 0;
        bool ok = true;  // warp-uniform; once false the warp only keeps passing the named barriers
        for (long tile = 0; tile < w1 - w0; tile++) {
            const long w = w0 + tile;
            const int img = find_img(p, w, cur);
            if (img != cur) {
                // image change: wait for the MMAs in flight (they read the old V^T), then reload
                if (ok && q >= 1)
                    ok = warp_wait(&a_empty[(q - 1) % NA], (uint32_t)(((q - 1) / NA) & 1), abort_flag);
                conv_sync();
                const ProjImgP &im = p.img[img];
                for (int c = ct; c < p.Cp; c += kConv) mean_s[c] = im.mean32[c];
                if (F8) {
                    for (int c = ct; c < p.Cp; c += kConv) scale_s[c] = im.scale[c];
                    // hi then lo, each DT rows x Cp bytes: 16-B chunks of 16 channels, 128 channels per row
                    const uint8_t *src = reinterpret_cast<const uint8_t *>(im.Vt);
                    for (int e = ct; e < 2 * DT * (p.Cp / 16); e += kConv) {
                        const int part = e / (DT * (p.Cp / 16)), r = e % (DT * (p.Cp / 16));
                        const int j = r / (p.Cp / 16), c16 = r % (p.Cp / 16);
                        const uint4 v = *reinterpret_cast<const uint4 *>(src + ((size_t)part * DT + j) * p.Cp + c16 * 16);
                        *reinterpret_cast<uint4 *>(Bs + (size_t)part * p.Cp * DT + (size_t)(c16 >> 3) * DT * 128 +
                                                   swz_off(j, c16 & 7)) = v;
                    }
                } else {
                    const __nv_bfloat16 *vt = reinterpret_cast<const __nv_bfloat16 *>(im.Vt);
                    for (int e = ct; e < DT * (p.Cp / 8); e += kConv) {
                        const int j = e / (p.Cp / 8), c8 = e % (p.Cp / 8);
                        const uint4 v = *reinterpret_cast<const uint4 *>(vt + (long)j * p.Cp + c8 * 8);
                        *reinterpret_cast<uint4 *>(Bs + (size_t)(c8 >> 3) * DT * 128 + swz_off(j, c8 & 7)) = v;
                    }
                }
                tc::fence_proxy_async_smem();
                conv_sync();
                cur = img;
            }
            for (int kc = 0; kc < nk; kc++, q++) {
                // operand chunk of this box: one box each (BF16), two boxes each (FP8)
                const long qa = F8 ? q >> 1 : q;
                const int hf = F8 ? (int)(q & 1) : 0;
                const int s = (int)(q % S), ab = (int)(qa % NA);
                if (ok) ok = warp_wait(&full[s], (uint32_t)((q / S) & 1), abort_flag);
                if (!ok) continue;
                // read the 32 features first and release the stage, then wait for the operand buffer
                const float *xs = reinterpret_cast<const float *>(stage + (size_t)s * kStageBytes) + (32 * h) * kM + m;
                float xv[32];
#pragma unroll
                for (int i = 0; i < 32; i++) xv[i] = xs[i * kM];
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[s]);
                if (hf == 0 && qa >= NA) ok = warp_wait(&a_empty[ab], (uint32_t)((qa / NA - 1) & 1), abort_flag);
                if (!ok) continue;
                const float4 *mu4 = reinterpret_cast<const float4 *>(mean_s + kc * kKc + 32 * h);
                uint8_t *arow = As + (size_t)ab * kAChunk;
                if (F8) {
                    // 32 channels -> 32 bytes: 16-B chunks 4 hf + 2 h and 4 hf + 2 h + 1 of the 128-B row
                    const float4 *sc4 = reinterpret_cast<const float4 *>(scale_s + kc * kKc + 32 * h);
#pragma unroll
                    for (int g = 0; g < 2; g++) {
                        uint32_t w[4];
#pragma unroll
                        for (int u = 0; u < 4; u++) {
                            const int i = 16 * g + 4 * u;
                            const float4 mu = mu4[4 * g + u], sc = sc4[4 * g + u];
                            w[u] = tc::pack_e4m3x4((xv[i] - mu.x) * sc.x, (xv[i + 1] - mu.y) * sc.y,
                                                   (xv[i + 2] - mu.z) * sc.z, (xv[i + 3] - mu.w) * sc.w);
                        }
                        *reinterpret_cast<uint4 *>(arow + swz_off(m, 4 * hf + 2 * h + g)) = make_uint4(w[0], w[1], w[2], w[3]);
                    }
                } else {
#pragma unroll
                    for (int g = 0; g < 4; g++) {
                        const float4 ma = mu4[2 * g], mb = mu4[2 * g + 1];
                        const float *x8 = xv + 8 * g;
                        uint4 pk;
                        pk.x = tc::pack_bf16x2(x8[0] - ma.x, x8[1] - ma.y);
                        pk.y = tc::pack_bf16x2(x8[2] - ma.z, x8[3] - ma.w);
                        pk.z = tc::pack_bf16x2(x8[4] - mb.x, x8[5] - mb.y);
                        pk.w = tc::pack_bf16x2(x8[6] - mb.z, x8[7] - mb.w);
                        *reinterpret_cast<uint4 *>(arow + swz_off(m, 4 * h + g)) = pk;
                    }
                }
                tc::fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(&a_full[ab]);
            }
        }
    } else {
        // ---------------------------------------------------------------- epilogue
        const int et = t - 64 - kConv;
        const int quarter = warp & 3;  // TMEM lane quarter (warp id % 4)
        constexpr int NG = DT / 16;    // 16-column groups
        const int own = (lane >> 1) & 15;  // column of each group this lane accumulates
        float rmn[NG], rmx[NG];
#pragma unroll
        for (int g = 0; g < NG; g++) { rmn[g] = __int_as_float(0x7f800000); rmx[g] = -__int_as_float(0x7f800000); }
        auto flush = [&](int img) {  // all epilogue threads
#pragma unroll
            for (int g = 0; g < NG; g++) {
                const int j = 16 * g + own;
                if ((lane & 1) == 0 && j < d) {
                    atomicMin(&kmin[j], f2key(rmn[g]));
                    atomicMax(&kmax[j], f2key(rmx[g]));
                }
                rmn[g] = __int_as_float(0x7f800000);
                rmx[g] = -__int_as_float(0x7f800000);
            }
            epi_sync();
            if (et < d) {
                uint32_t *mm = p.img[img].mm;
                atomicMin(&mm[et * kKeyStride], kmin[et]);
                atomicMax(&mm[(d + et) * kKeyStride], kmax[et]);
                kmin[et] = 0xffffffffu;
                kmax[et] = 0u;
            }
            epi_sync();
        };
        int cur = -1;
        bool ok = true;
        for (long tile = 0; tile < w1 - w0; tile++) {
            const long w = w0 + tile;
            const int img = find_img(p, w, cur);
            if (img != cur) {
                if (cur >= 0) flush(cur);
                cur = img;
            }
            const ProjImgP &im = p.img[img];
            const int ac = (int)(tile & 1);
            if (ok) ok = warp_wait(&acc_full[ac], (uint32_t)((tile / 2) & 1), abort_flag);
            if (!ok) continue;
            tc::tc_fence_after();
            const long pe = (w - im.tile0) * kM + 32 * quarter + lane;
            const bool valid = pe < im.N;
            if (im.bins) {
                // fixed range: the bins straight from the accumulator (no Y, no range keys)
                const long py = valid ? pe / im.W : 0, px = valid ? pe - py * im.W : 0;
                const long H = im.N / im.W;
                const float fB = (float)im.B;
#pragma unroll
                for (int g = 0; g < NG; g++) {
                    uint32_t r[16];
                    tc::tmem_ld16(tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(ac * DT + 16 * g), r);
                    tc::tmem_wait_ld();
#pragma unroll
                    for (int i = 0; i < 16; i++) {
                        const int j = 16 * g + i;
                        if (j < d && valid) {
                            const float v = F8 ? __uint_as_float(r[i]) * __ldg(im.colscale + j) : __uint_as_float(r[i]);
                            const int q = quant_bin(v, __ldg(im.qlo + j), __ldg(im.qhi + j), fB, im.B);
                            im.bins[((long)j * H + py) * im.pitch + px] = (uint8_t)q;
                        }
                    }
                }
                tc::tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&acc_empty[ac]);
                continue;
            }
#pragma unroll
            for (int g = 0; g < NG; g++) {
                uint32_t r[16];
                tc::tmem_ld16(tmem + ((uint32_t)(32 * quarter) << 16) + (uint32_t)(ac * DT + 16 * g), r);
                tc::tmem_wait_ld();
                float vmn[16], vmx[16];
#pragma unroll
                for (int i = 0; i < 16; i++) {
                    const int j = 16 * g + i;
                    const float v = F8 ? __uint_as_float(r[i]) * __ldg(im.colscale + j) : __uint_as_float(r[i]);
                    if (j < d && valid) im.Y[(long)j * im.N + pe] = v;
                    vmn[i] = valid ? v : __int_as_float(0x7fc00000);  // NaN: ignored by the reduction
                    vmx[i] = vmn[i];
                }
                warp_reduce16<true>(vmn);
                warp_reduce16<false>(vmx);
                rmn[g] = fminf(rmn[g], vmn[0]);
                rmx[g] = fmaxf(rmx[g], vmx[0]);
            }
            tc::tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[ac]);
        }
        if (cur >= 0) flush(cur);  // unconditional: every epilogue thread passes the same barriers
    }
    if (t == 0 && *abort_flag) atomicOr(status, kStatusMmaTimeout);
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, kCols);
    }
}

template <int DT, bool F8>
cudaError_t launch_dt(const ProjParams &p, int *status, cudaStream_t st) {
    static DeviceOnce attrs;
    int dev = 0, n_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = device_once(attrs, dev, [] {
        return cudaFuncSetAttribute(k_project_tma<DT, F8>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    });
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const size_t smem = smem_layout(p.stages, p.na, p.Cp, DT, F8).total;
    const long grid = p.total_tiles < n_sm ? p.total_tiles : n_sm;
    QFCA_LAUNCH("k_project_tma", st, (k_project_tma<DT, F8><<<(unsigned)grid, kThreads, smem, st>>>(p, status)));
    return cudaGetLastError();
}

thread_local ProjTiling tl_last_proj{0, 0};

}  // namespace

thread_local const ProjTiling *tl_proj_tiling = nullptr;

ProjTiling project_last_tiling() { return tl_last_proj; }

int project_tilings(int C, int d, bool fp8, ProjTiling *out, int max_out) {
    const int DT = d <= 16 ? 16 : (d <= 32 ? 32 : 64);
    const int Cp = fp8 ? (C + 127) / 128 * 128 : (C + kKc - 1) / kKc * kKc;
    int n = 0;
    for (int sg = kMaxStages; sg >= 2; sg--)
        for (int a = kMaxA; a >= 2; a--)
            if (n < max_out && smem_layout(sg, a, Cp, DT, fp8).total <= 227 * 1024) out[n++] = ProjTiling{sg, a};
    return n;
}

bool project_tma_ok(const float *X, long N, int layout) {
    return layout == QFCA_NCHW && N % 4 == 0 && ((uintptr_t)X & 15) == 0;
}

cudaError_t launch_project_tma(const ProjJob *jobs, int n, int C, int d, bool fp8, int *status, cudaStream_t st) {
    const int DT = d <= 16 ? 16 : (d <= 32 ? 32 : 64);
    const int Cp = fp8 ? (C + 127) / 128 * 128 : (C + kKc - 1) / kKc * kKc;
    // deepest TMA ring first (bytes in flight), then the deepest operand ring
    int stages = 0, na = 0;
    for (int sg = kMaxStages; sg >= 3 && !stages; sg--)
        for (int a = kMaxA; a >= 2; a--)
            if (smem_layout(sg, a, Cp, DT, fp8).total <= 227 * 1024) { stages = sg, na = a; break; }
    if (!stages) {
        stages = 2, na = 2;
        if (smem_layout(stages, na, Cp, DT, fp8).total > 227 * 1024) return cudaErrorNotSupported;
    }
    if (tl_proj_tiling && tl_proj_tiling->stages >= 2 && tl_proj_tiling->stages <= kMaxStages &&
        tl_proj_tiling->na >= 2 && tl_proj_tiling->na <= kMaxA &&
        smem_layout(tl_proj_tiling->stages, tl_proj_tiling->na, Cp, DT, fp8).total <= 227 * 1024)
        stages = tl_proj_tiling->stages, na = tl_proj_tiling->na;
    tl_last_proj = ProjTiling{stages, na};
    for (int i0 = 0; i0 < n; i0 += kMaxBatch) {
        const int m = n - i0 < kMaxBatch ? n - i0 : kMaxBatch;
        ProjParams p;
        memset(&p, 0, sizeof(p));
        p.n = m, p.C = C, p.Cp = Cp, p.nk = Cp / kKc, p.d = d, p.stages = stages, p.na = na;
        long tiles = 0;
        for (int i = 0; i < m; i++) {
            const ProjJob &j = jobs[i0 + i];
            if (!project_tma_ok(j.X, j.N, QFCA_NCHW)) return cudaErrorNotSupported;
            if (fp8 && (!j.scale || !j.colscale)) return cudaErrorInvalidValue;
            ProjImgP &im = p.img[i];
            im.N = j.N, im.tile0 = tiles, im.mean32 = j.mean32, im.Vt = j.Vt, im.scale = j.scale;
            im.colscale = j.colscale, im.Y = j.Y, im.mm = j.mm;
            im.qlo = j.qlo, im.qhi = j.qhi, im.bins = j.bins, im.W = j.W, im.pitch = j.pitch, im.B = j.B;
            if (j.bins && (!j.qlo || !j.qhi || j.W < 1 || j.N % j.W != 0 || j.pitch < j.W || j.B < 2))
                return cudaErrorInvalidValue;
            tiles += (j.N + kM - 1) / kM;
            cudaError_t e = make_tmap_f32_2d(&p.tmap[i], j.X, (uint64_t)j.N, (uint64_t)C, (uint64_t)j.N * 4, kM, kKc);
            if (e != cudaSuccess) return e;
        }
        p.total_tiles = tiles;
        cudaError_t e;
        if (fp8) {
            switch (DT) {
                case 16: e = launch_dt<16, true>(p, status, st); break;
                case 32: e = launch_dt<32, true>(p, status, st); break;
                default: e = launch_dt<64, true>(p, status, st); break;
            }
        } else {
            switch (DT) {
                case 16: e = launch_dt<16, false>(p, status, st); break;
                case 32: e = launch_dt<32, false>(p, status, st); break;
                default: e = launch_dt<64, false>(p, status, st); break;
            }
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace qfca
