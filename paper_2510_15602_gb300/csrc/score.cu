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

#include <algorithm>
#include <cmath>
#include <atomic>
#include <mutex>

#include "internal.cuh"
#include "tc.cuh"

namespace qfca {
namespace {

constexpr uint32_t kTmaTries = 1u << 26;

// Per-image part of a window-EMD launch (kernel parameter block).
struct ScoreImgP {
    int H, W, r, nbx;        // nbx: strips
    long cta0;               // first CTA of this image
    const uint32_t *ref;     // [d][B]
    uint32_t Nref;
    void *numer;             // [d][H][W] of OUT, or NULL when accumulating
    unsigned long long *accum;  // [H][W] running sums, or NULL
    float *score;            // [H][W]: written by the kernel itself when it sums every component (fuse)
};

struct ScoreParams {
    int n, d, B, SW, TH, kg, n_kg;
    int BR;                     // bands per CTA: a run of consecutive bands of one strip and component group
    uint32_t tile_bytes;
    uint32_t first_wait_tries;  // probes of each CTA's first tile wait (kTmaTries; fewer only to test the timeout path)
    int fuse;                   // every CTA holds all d components: sum them per pixel in shared memory, write the score
    uint32_t acc_off;           // byte offset of the per-pixel sums [TH][SW] u64 in shared memory (fuse)
    ScoreImgP img[kMaxBatch];
    CUtensorMap tmap[kMaxBatch];  // bins of image i as [d][H][pitch] u8, box {TCp_i, TH + 2 r_i, 1}
};

struct FinImgP {
    int H, W, r;
    uint32_t Nref;
    long blk0;               // first pixel block of this image
    const void *numer;
    const unsigned long long *accum;
    float *score;
    const float *lo, *hi;    // value units: component ranges [d] (NULL: bin units)
};

struct FinParams {
    int n, d, B;
    FinImgP img[kMaxBatch];
};

constexpr int kFinMaxWeights = 512;  // components whose bin widths a value-unit finalisation keeps in shared memory

__host__ __device__ inline int halo_of(int r) { return (r + 15) & ~15; }
__host__ __device__ inline int tcp_of(int SW, int r) { return SW + 2 * halo_of(r); }
// Rows of a band's tile: the band's TH rows, r above and below, and one more above (the row that leaves
// the window when the band's first row continues the previous band's last window).
__host__ __device__ inline int tile_rows(int TH, int r) { return TH + 2 * r + 1; }

size_t score_smem_core(int SW, int TH, int B, int rmax) {
    const size_t tile = align_up((size_t)tile_rows(TH, rmax) * tcp_of(SW, rmax), 128);
    return 2 * tile + sizeof(uint32_t) * (size_t)(B + 1) * SW + sizeof(uint32_t) * 256 + sizeof(uint64_t) * 256 +
           2 * sizeof(uint64_t);
}
// fuse: plus the per-pixel u64 sums over the components of the CTA's TH x SW pixels
size_t score_smem(int SW, int TH, int B, int rmax, bool fuse = false) {
    return 128 + score_smem_core(SW, TH, B, rmax) + (fuse ? sizeof(uint64_t) * (size_t)TH * SW : 0);
}

// 32-bit shared-memory address of a pointer into shared memory, the
// fire-and-forget increment of a window count there, and the read of a count.
// Both are volatile asm with no memory clobber: the compiler keeps them in
// program order with respect to each other (a thread reads its own counts after
// its increments; the hardware orders one thread's accesses to one address), and
// the CTA and warp barriers order them against every other access, while the
// kernel's parameters and pointers stay in registers across them.
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void count_add(uint32_t addr, uint32_t v) {
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(v));
}
__device__ __forceinline__ uint32_t count_ld(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(smem_addr(p)));
    return v;
}

// The window counts of one thread, bin-major (count of code v at hbase + v * 4 SWT): the span bytes
// of a tile row from column c0 leave (rowo) or enter (rown) the window.  The row bytes come in as
// 32-bit words (five words for a 15-pixel span instead of fifteen byte loads), aligned to c0 by a
// funnel shift; each byte is extracted with one permute.  TWO = false: only rown, entering.
template <int SWT, bool TWO>
__device__ __forceinline__ void window_rows(const uint8_t *rowo, const uint8_t *rown, int c0, int span,
                                            uint32_t hbase) {
    constexpr int LOG = SWT == 128 ? 9 : 8;  // log2(4 SWT): bytes between consecutive codes' counts
    const uint32_t *wo = reinterpret_cast<const uint32_t *>(rowo) + (c0 >> 2);
    const uint32_t *wn = reinterpret_cast<const uint32_t *>(rown) + (c0 >> 2);
    const uint32_t sh = (uint32_t)(c0 & 3) * 8u;
    uint32_t lo_o = TWO ? wo[0] : 0u, lo_n = wn[0];
    int q = 0;
    for (; q + 4 <= span; q += 4) {
        const uint32_t hi_n = wn[(q >> 2) + 1];
        const uint32_t an = __funnelshift_r(lo_n, hi_n, sh);
        lo_n = hi_n;
        uint32_t ao = 0;
        if (TWO) {
            const uint32_t hi_o = wo[(q >> 2) + 1];
            ao = __funnelshift_r(lo_o, hi_o, sh);
            lo_o = hi_o;
        }
#pragma unroll
        for (int e = 0; e < 4; e++) {
            if (TWO) count_add(hbase + (__byte_perm(ao, 0u, 0x4440u + e) << LOG), 0xFFFFFFFFu);
            count_add(hbase + (__byte_perm(an, 0u, 0x4440u + e) << LOG), 1u);
        }
    }
    if (q < span) {  // 1..3 bytes left (span is odd)
        const uint32_t an = __funnelshift_r(lo_n, wn[(q >> 2) + 1], sh);
        uint32_t ao = 0;
        if (TWO) ao = __funnelshift_r(lo_o, wo[(q >> 2) + 1], sh);
#pragma unroll
        for (int e = 0; e < 3; e++)
            if (q + e < span) {
                if (TWO) count_add(hbase + (__byte_perm(ao, 0u, 0x4440u + e) << LOG), 0xFFFFFFFFu);
                count_add(hbase + (__byte_perm(an, 0u, 0x4440u + e) << LOG), 1u);
            }
    }
}

// Window histograms + exact EMD numerators for a band of TH rows x SWT columns
// and a group of kg components of one image of the table.  Thread t owns
// output column x0 + t; its window histogram lives at hist[b * SWT + t]
// (conflict-free for any bins the warp's threads touch).  Increments are
// shared-memory reductions without return, so no thread waits on them.  ACC
// is the type of the CDF walk (u32 when (B-1)(2r+1)^2 N_ref < 2^32 for every
// image), OUT the type of the stored numerators; KB > 0 fixes B at compile
// time; SWT is the strip width (64 or 128 threads), so every histogram address
// is a constant offset from the thread's column.  The band's bin tile of each
// component (rows y0-r .. y0+TH-1+r, columns from x0 - halo, halo = r rounded
// up to 16 bytes) is one 3-D TMA box; boxes are double-buffered so the next
// component's tile arrives while the current one is processed.  Waits are
// bounded; a wait that runs out sets bit 0 of the status word and the CTA
// stops.
//
// WALK selects the CDF walk of the interior pixels (the border pixels always
// take the per-thread walk):
//   0  per thread, sequential over the bins of its own pixel (with KB = 32 the
//      interior reference terms cumR_b N_loc are held in registers);
//   1  warp-shuffle segmented walk (KB = 32, u32 only): two lanes per pixel,
//      each walks 16 bins of it; the lower lane's count reaches the upper lane
//      by a shuffle as its CDF offset, the two partial sums are added by a
//      shuffle, and the owner lane of the pixel receives the result by a
//      third; 16 pixels per pass, two passes per row.
template <typename ACC, typename OUT, int KB, int SWT, int WALK>
__global__ void __launch_bounds__(SWT) k_window_emd(const __grid_constant__ ScoreParams p, int *__restrict__ status) {
    static_assert(WALK == 0 || (KB == 32 && sizeof(ACC) == 4), "the shuffle walk is built for 32 bins, u32");
    const int B = KB > 0 ? KB : p.B;
    const int TH = p.TH, d = p.d;
    constexpr int SW = SWT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *smem = tc::align_smem<128>(smem_raw);
    uint8_t *tiles = smem;
    uint32_t *hist = reinterpret_cast<uint32_t *>(smem + 2 * (size_t)p.tile_bytes);
    uint32_t *cumR = hist + (size_t)(B + 1) * SW;
    ACC *cRi = reinterpret_cast<ACC *>(cumR + 256);  // cumR[b] * N_loc for an interior window
    uint64_t *bar = reinterpret_cast<uint64_t *>(reinterpret_cast<unsigned char *>(cumR + 256) + 256 * sizeof(uint64_t));
    unsigned long long *acc = reinterpret_cast<unsigned long long *>(smem + p.acc_off);  // [TH][SW] (fuse only)

    // which image, component group, band and strip
    const long cta = blockIdx.x;
    const int ii = table_image(p.n, cta, [&](int i) { return p.img[i].cta0; });
    const ScoreImgP im = p.img[ii];  // in registers
    const CUtensorMap *tmap = &p.tmap[ii];
    const int H = im.H, W = im.W, r = im.r;
    long local = cta - im.cta0;
    const int kgi = (int)(local % p.n_kg);
    local /= p.n_kg;
    const int bx = (int)(local % im.nbx), brun = (int)(local / im.nbx);
    const int nby = (H + TH - 1) / TH;
    const int b_lo = brun * p.BR, nb = min(nby, b_lo + p.BR) - b_lo;  // this CTA's bands
    const int k0 = kgi * p.kg, k1 = min(d, k0 + p.kg);
    const int nitems = (k1 - k0) * nb;  // (component, band) pairs, component-major
    const uint32_t Nref = im.Nref;
    const uint32_t *ref_hist = im.ref;
    const long HW = (long)H * W;

    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    constexpr int nwarps = SW >> 5;
    const int x0 = bx * SW;
    const int x = x0 + t;
    const int halo = halo_of(r), TCp = SW + 2 * halo, TR = tile_rows(TH, r);
    const int tx0 = x0 - halo;  // image column of the tile origin; its row is band * TH - r - 1
    const int span = 2 * r + 1;
    const uint32_t Nint = (uint32_t)(span * span);
    const uint32_t box_bytes = (uint32_t)(TR * TCp);
    const int wpr = TCp >> 2;  // 32-bit words per tile row
    if (t == 0) {
        tc::mbar_init(&bar[0], 1);
        tc::mbar_init(&bar[1], 1);
        tc::fence_mbar_init();
    }
    __syncthreads();
    if (t == 0 && nitems > 0) {
        tc::mbar_arrive_expect_tx(&bar[0], box_bytes);
        tc::tma_load_3d(tiles, tmap, tx0, b_lo * TH - r - 1, k0, &bar[0]);
    }
    bool failed = false;
    int issued = nitems > 0 ? 1 : 0, waited = 0;

    const int ncols = min(W - 1, x + r) - max(0, x - r) + 1;
    const int c0 = t + halo - r;  // tile column of this thread's window's left edge
    uint32_t *hc = hist + t;
    const uint32_t hbase = smem_addr(hc);
    // the shuffle walk: this lane's pixel (column of the warp) in pass 0 / 1, and its half of the bins
    const int wp0 = lane >> 1, wg = lane & 1;
    // interior reference terms in registers (per-thread walk: all 31; shuffle walk: this lane's half)
    constexpr int NREG = (KB == 32 && sizeof(ACC) == 4) ? (WALK == 1 ? 16 : 31) : 1;
    uint32_t cr[NREG];
    for (int it = 0; it < nitems; it++) {
        const int k = k0 + it / nb, bi = it - (it / nb) * nb;
        const int y0 = (b_lo + bi) * TH, ty0 = y0 - r - 1;  // band origin; tile origin row
        const bool fresh = bi == 0;                       // first band of component k: a new window
        const bool inner = tx0 >= 0 && tx0 + TCp <= W && ty0 >= 0 && ty0 + TR <= H;
        __syncthreads();  // the buffer of item it-1 is free again
        const int buf = it & 1;
        if (t == 0 && it + 1 < nitems) {
            const int kn = k0 + (it + 1) / nb, bn = b_lo + (it + 1) % nb;
            tc::mbar_arrive_expect_tx(&bar[buf ^ 1], box_bytes);
            tc::tma_load_3d(tiles + (size_t)(buf ^ 1) * p.tile_bytes, tmap, tx0, bn * TH - r - 1, kn, &bar[buf ^ 1]);
        }
        if (it + 1 < nitems) issued++;
        // warp 0: lane l loads reference bins [8l, 8l+8) of component k (in flight during the wait)
        uint32_t rv[8];
        if (fresh && t < 32) {
#pragma unroll
            for (int j = 0; j < 8; j++) {
                const int b = 8 * t + j;
                rv[j] = b < B ? __ldg(&ref_hist[(long)k * B + b]) : 0u;
            }
        }
        // every thread waits for the tile itself; a wait that ran out is reported at the barrier after the
        // rewrite (one CTA barrier fewer per item), and the CTA then stops
        const bool ok = tc::mbar_wait(&bar[buf], (it >> 1) & 1, it == 0 ? p.first_wait_tries : kTmaTries);
        waited++;
        uint8_t *tile = tiles + (size_t)buf * p.tile_bytes;
        // in-image bytes -> min(bin, B-1) + 1, everything else -> 0; a warp per tile row
        {
            uint32_t *tw = reinterpret_cast<uint32_t *>(tile);
            const uint32_t cap = 0x01010101u * (uint32_t)(B - 1);
            for (int row = warp; row < TR; row += nwarps) {
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
        if (fresh && t < 32) {  // whole warp 0: prefix sums of the reference histogram
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
        if (fresh) {
            if (KB > 0) {
#pragma unroll
                for (int b = 0; b <= KB; b++) hc[b * SW] = 0;
            } else {
                for (int b = 0; b <= B; b++) hc[b * SW] = 0;
            }
        }
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        if (fresh && KB == 32 && sizeof(ACC) == 4) {
            const uint32_t *c32 = reinterpret_cast<const uint32_t *>(cRi);
#pragma unroll
            for (int j = 0; j < NREG; j++) {
                const int b = WALK == 1 ? 16 * wg + j : j;
                cr[j] = b < KB - 1 ? c32[b] : 0u;
            }
        }
        const bool xin = x < W;
        // this thread's column of the outputs
        OUT *numer_col = im.numer ? reinterpret_cast<OUT *>(im.numer) + (long)k * HW + x : nullptr;
        unsigned long long *accum_col = im.accum ? im.accum + x : nullptr;
        // window of the band's first row (tile rows 1 .. 2r+1), or the previous band's last window continued
        if (fresh && xin)
            for (int ry = 1; ry <= span; ry++) window_rows<SW, false>(tile + ry * TCp, tile + ry * TCp, c0, span, hbase);  // rowo unused
        for (int i = 0; i < TH; i++) {
            const int yy = y0 + i;
            if (yy >= H) break;
            if ((i > 0 || !fresh) && xin)  // image row yy - r - 1 (tile row i) leaves, row yy + r enters
                window_rows<SW, true>(tile + i * TCp, tile + (i + span) * TCp, c0, span, hbase);
            const int nrows = min(H - 1, yy + r) - max(0, yy - r) + 1;
            const uint32_t Nloc = (uint32_t)(nrows * ncols);
            ACC D = 0;
            const uint32_t *hb = hc + SW;  // bin 0
            bool walked = false;
            if (WALK == 1) {
                // every lane of the warp takes part (shuffles), so the test is warp-wide
                __syncwarp();
                if (__all_sync(0xffffffffu, !xin || Nloc == Nint)) {
                    uint32_t Dp[2];
#pragma unroll
                    for (int pass = 0; pass < 2; pass++) {
                        const uint32_t *h2 = hist + SW + (warp << 5) + 16 * pass + wp0 + 16 * wg * SW;
                        uint32_t hv[16], cnt = 0, s = 0;
#pragma unroll
                        for (int j = 0; j < 16; j++) {
                            hv[j] = count_ld(h2 + j * SW);
                            cnt += hv[j];  // this half's count
                        }
                        // the lower half's count is the upper half's CDF offset
                        const uint32_t below = __shfl_xor_sync(0xffffffffu, cnt, 1);
                        uint32_t a = wg ? below * Nref : 0u;
#pragma unroll
                        for (int j = 0; j < 16; j++) {
                            if (16 * wg + j < KB - 1) {  // the last bin's term is 0
                                a += hv[j] * Nref;
                                s = __usad(a, cr[j], s);
                            }
                        }
                        Dp[pass] = s + __shfl_xor_sync(0xffffffffu, s, 1);
                    }
                    __syncwarp();  // every lane's reads of the counts precede the next row's updates
                    // pixel `lane` was walked by lanes 2 lane, 2 lane + 1 (pass 0) or 2 (lane - 16) (pass 1)
                    const uint32_t d0 = __shfl_sync(0xffffffffu, Dp[0], (2 * lane) & 31);
                    const uint32_t d1 = __shfl_sync(0xffffffffu, Dp[1], (2 * lane) & 31);
                    D = (ACC)(lane < 16 ? d0 : d1);
                    walked = true;
                }
            }
            if (!xin) continue;
            // the last bin's term is 0 (both CDFs reach 1), so the walk stops at B-2
            if (walked) {
            } else if (Nloc == Nint) {
                if (KB == 32 && sizeof(ACC) == 4 && WALK == 0) {
                    // 32-bit walk: a = cumP_b N_ref accumulated directly, D += |a - c| in one
                    // sum-of-absolute-difference instruction, c from registers
                    uint32_t a = 0, D32 = 0;
#pragma unroll
                    for (int b = 0; b < KB - 1; b++) {
                        a += count_ld(hb + b * SW) * Nref;
                        D32 = __usad(a, cr[WALK == 0 ? b : 0], D32);
                    }
                    D = (ACC)D32;
                } else if (KB > 0 && sizeof(ACC) == 4) {
                    // the reference terms four at a time (16-byte broadcast loads)
                    const uint4 *c4 = reinterpret_cast<const uint4 *>(cRi);
                    uint32_t a = 0, D32 = 0;
#pragma unroll
                    for (int b4 = 0; b4 < KB / 4; b4++) {
                        const uint4 c = c4[b4];
                        const uint32_t cv[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
                        for (int e = 0; e < 4; e++) {
                            const int b = 4 * b4 + e;
                            if (b < KB - 1) {
                                a += count_ld(hb + b * SW) * Nref;
                                D32 = __usad(a, cv[e], D32);
                            }
                        }
                    }
                    D = (ACC)D32;
                } else if (KB > 0) {
                    uint32_t cnt = 0;
#pragma unroll
                    for (int b = 0; b < KB - 1; b++) {
                        cnt += count_ld(hb + b * SW);
                        const ACC a = (ACC)cnt * (ACC)Nref, c = cRi[b];
                        D += max(a, c) - min(a, c);
                    }
                } else {
                    uint32_t cnt = 0;
#pragma unroll 4
                    for (int b = 0; b < B - 1; b++) {
                        cnt += count_ld(hb + b * SW);
                        const ACC a = (ACC)cnt * (ACC)Nref, c = cRi[b];
                        D += max(a, c) - min(a, c);
                    }
                }
            } else {
                uint32_t cnt = 0;
#pragma unroll 4
                for (int b = 0; b < B - 1; b++) {
                    cnt += count_ld(hb + b * SW);
                    const ACC a = (ACC)cnt * (ACC)Nref, c = (ACC)cumR[b] * (ACC)Nloc;
                    D += max(a, c) - min(a, c);
                }
            }
            if (p.fuse) {  // one band per CTA: item it is component k0 + it
                unsigned long long &a = acc[i * SW + t];  // this thread's own column: no other thread touches it
                a = (it == 0 ? 0ull : a) + (unsigned long long)D;
            } else if (accum_col) {
                atomicAdd(accum_col + (long)yy * W, (unsigned long long)D);
            } else {
                numer_col[(long)yy * W] = (OUT)D;
            }
        }
        tc::fence_proxy_async_smem();  // this iteration's writes to the tile precede the next TMA write into it
    }
    if (failed) {
        if (t == 0) atomicOr(status, kStatusMmaTimeout);
        // let every issued copy (including the one whose wait ran out) land before the CTA leaves (bounded)
        for (int w = waited - 1; w < issued; w++) tc::mbar_wait(&bar[w & 1], (w >> 1) & 1, kTmaTries);
    } else if (p.fuse && x < W && nitems > 0) {
        // s(p) = sum_k D_k(p) / (d N_loc N_ref): one division per pixel, no numerators leave the SM
        const int y0 = b_lo * TH;
        for (int i = 0; i < TH; i++) {
            const int yy = y0 + i;
            if (yy >= H) break;
            const int nrows = min(H - 1, yy + r) - max(0, yy - r) + 1;
            const double den = (double)nrows * (double)ncols * (double)Nref * (double)d;
            im.score[(long)yy * W + x] = (float)((double)acc[i * SW + t] / den);
        }
    }
}

// s(p) = sum_k D_k(p) / (d * N_loc * N_ref), from the per-component numerators
// or from their running sums; blocks of 256 pixels over the table's images.
// In value units (ranges given) the distance between bins a and b of
// component k is |a - b| w_k with w_k = (hi_k - lo_k) / B, so
// s(p) = sum_k w_k D_k(p) / (d N_loc N_ref), summed in FP64 over k in order.
template <typename OUT>
__global__ void __launch_bounds__(256) k_finalize(const __grid_constant__ FinParams p) {
    __shared__ double wk[kFinMaxWeights];
    const long blk = blockIdx.x;
    const int ii = table_image(p.n, blk, [&](int i) { return p.img[i].blk0; });
    const FinImgP &im = p.img[ii];
    const int d = p.d;
    if (im.lo) {
        for (int k = threadIdx.x; k < d; k += 256) wk[k] = ((double)im.hi[k] - (double)im.lo[k]) / (double)p.B;
        __syncthreads();
    }
    const long HW = (long)im.H * im.W;
    const long q = (blk - im.blk0) * 256 + threadIdx.x;
    if (q >= HW) return;
    const int y = (int)(q / im.W), x = (int)(q - (long)y * im.W);
    const int r = im.r;
    const int nr = min(im.H - 1, y + r) - max(0, y - r) + 1;
    const int nc = min(im.W - 1, x + r) - max(0, x - r) + 1;
    const double den = (double)nr * (double)nc * (double)im.Nref * (double)d;
    if (im.lo) {
        const OUT *nk = reinterpret_cast<const OUT *>(im.numer) + q;
        double sv = 0.0;
        for (int k = 0; k < d; k++) sv = fma(wk[k], (double)__ldg(nk + (long)k * HW), sv);
        im.score[q] = (float)(sv / den);
        return;
    }
    unsigned long long s = 0;
    if (im.accum) {
        s = im.accum[q];
    } else {
        const OUT *nk = reinterpret_cast<const OUT *>(im.numer) + q;
        for (int k = 0; k < d; k++) s += (unsigned long long)__ldg(nk + (long)k * HW);
    }
    im.score[q] = (float)((double)s / den);
}

using EmdFn = void (*)(const ScoreParams, int *);

// The instantiation of k_window_emd for B (32, 64 or any), strip width and CDF walk.
template <typename ACC, typename OUT, int KB, int SWT>
EmdFn emd_fn_walk(int walk) {
    if constexpr (KB == 32 && sizeof(ACC) == 4) {
        if (walk == 1) return k_window_emd<ACC, OUT, KB, SWT, 1>;
    }
    return k_window_emd<ACC, OUT, KB, SWT, 0>;
}

template <typename ACC, typename OUT, int KB>
EmdFn emd_fn_sw(int SW, int walk) {
    return SW == 128 ? emd_fn_walk<ACC, OUT, KB, 128>(walk) : emd_fn_walk<ACC, OUT, KB, 64>(walk);
}

template <typename ACC, typename OUT>
EmdFn emd_fn(int KB, int SW, int walk) {
    if (KB == 32) return emd_fn_sw<ACC, OUT, 32>(SW, walk);
    if (KB == 64) return emd_fn_sw<ACC, OUT, 64>(SW, walk);
    return emd_fn_sw<ACC, OUT, 0>(SW, walk);
}

template <typename ACC, typename OUT>
void launch_emd_kb(int KB, int walk, long grid, size_t smem, int SW, cudaStream_t st, const ScoreParams &p,
                   int *status) {
    const EmdFn fn = emd_fn<ACC, OUT>(KB, SW, walk);
    QFCA_LAUNCH("k_window_emd", st, (fn<<<(unsigned)grid, SW, smem, st>>>(p, status)));
}

template <typename ACC, typename OUT>
cudaError_t emd_occupancy(int KB, int walk, size_t smem, int SW, int *per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, emd_fn<ACC, OUT>(KB, SW, walk), SW, smem);
}

template <typename ACC, typename OUT>
cudaError_t emd_set_smem_attr() {
    cudaError_t e = cudaSuccess;
    for (int KB : {32, 64, 0})
        for (int SW : {64, 128})
            for (int walk : {0, 1})
                if (e == cudaSuccess)
                    e = cudaFuncSetAttribute(emd_fn<ACC, OUT>(KB, SW, walk), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             200 * 1024);
    return e;
}

enum class EmdKind { U32_U32, U32_U64, U64_U64 };

cudaError_t emd_occupancy_kind(EmdKind kind, int KB, int walk, size_t smem, int SW, int *per_sm) {
    switch (kind) {
    case EmdKind::U32_U32: return emd_occupancy<uint32_t, uint32_t>(KB, walk, smem, SW, per_sm);
    case EmdKind::U32_U64: return emd_occupancy<uint32_t, unsigned long long>(KB, walk, smem, SW, per_sm);
    default: return emd_occupancy<unsigned long long, unsigned long long>(KB, walk, smem, SW, per_sm);
    }
}

// Modelled cost (lane-instructions) of the CTAs of one image at a given tiling: a band costs its rows
// and its tile's rewrite; the first band of each run and component also builds a window from scratch.
double image_cost(int H, int W, int d, int B, int r, int SW, int TH, int kg, int n_kg, int BR) {
    const int span = 2 * r + 1, TR = tile_rows(TH, r);
    const double row = 2.0 * span * 3.0 + 4.0 * (B - 1) + 12.0;
    const double band = 6.0 * TR * tcp_of(SW, r) / (4.0 * SW) + 40.0;
    const double fresh = 3.0 * span * span + 2.0 * B + 40.0;
    const int nby = (H + TH - 1) / TH, runs = (nby + BR - 1) / BR;
    const double ctas = (double)((W + SW - 1) / SW) * runs * n_kg;
    (void)d;
    return ctas * (kg * ((double)BR * (TH * row + band) + fresh) + 200.0);
}

DeviceOnce g_attrs_emd;

cudaError_t ensure_attrs(int *n_sm) {
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    err = device_once(g_attrs_emd, dev, [] {
        cudaError_t r = emd_set_smem_attr<uint32_t, uint32_t>();
        if (r == cudaSuccess) r = emd_set_smem_attr<uint32_t, unsigned long long>();
        if (r == cudaSuccess) r = emd_set_smem_attr<unsigned long long, unsigned long long>();
        return r;
    });
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(n_sm, cudaDevAttrMultiProcessorCount, dev);
    return err;
}

// One launch of at most kMaxBatch jobs.
cudaError_t score_chunk(const ScoreJob *jobs, int n, int d, int B, void *ws, bool ws_accumulates, int *status,
                        cudaStream_t st, const ScoreTiling *tiling, ScoreTiling *chosen, uint32_t first_wait_tries) {
    int rmax = 1;
    bool narrow = true, want_numer = false, value_units = false;
    for (int i = 0; i < n; i++) {
        value_units = value_units || jobs[i].lo;
        const double span2 = (double)(2 * jobs[i].r + 1) * (2 * jobs[i].r + 1);
        // u32 walk when every partial and the numerator fit: (B-1) (2r+1)^2 N_ref < 2^32
        narrow = narrow && (double)(B - 1) * span2 * (double)jobs[i].Nref < 4294967295.0 &&
                 span2 * jobs[i].Nref < 4294967295.0;
        want_numer = want_numer || jobs[i].numer_out;
        rmax = std::max(rmax, jobs[i].r);
    }
    const EmdKind kind = !narrow ? EmdKind::U64_U64
                         : (want_numer || ws_accumulates) ? EmdKind::U32_U64 : EmdKind::U32_U32;
    const size_t out_bytes = kind == EmdKind::U32_U32 ? 4 : 8;
    const int KB = (B == 32 || B == 64) ? B : 0;
    // a tiling with one component group sums the components inside the CTA (bin units, no numerators asked)
    const bool can_fuse = !want_numer && !ws_accumulates && !value_units;
    int n_sm = 0;
    cudaError_t err = ensure_attrs(&n_sm);
    if (err != cudaSuccess) return err;

    // tiling: the caller's, else the modelled best over strip widths, band heights, component splits and
    // band runs (a fused tiling, one component group, keeps one band per CTA: its per-pixel sums cover one band)
    auto fits = [&](int SW, int TH, bool fz) {
        return score_smem(SW, TH, B, rmax, fz) <= 200 * 1024 && tcp_of(SW, rmax) <= 256 && tile_rows(TH, rmax) <= 256;
    };
    int max_nby = 1;
    ScoreTiling best{0, 0, 0, 0, 0};
    if (tiling && tiling->SW > 0) {
        best = *tiling;
        if (!(best.SW == 64 || best.SW == 128) || best.TH < 1 || best.TH > 64 || best.n_kg < 1 || best.bands < 0)
            return cudaErrorNotSupported;
        if (best.walk < 0 || best.walk > 1) return cudaErrorNotSupported;
        if (!fits(best.SW, best.TH, can_fuse && best.n_kg == 1)) return cudaErrorNotSupported;
    } else {
        double best_cost = 1e300;
        for (int SW : {128, 64})
            for (int TH : {16, 32, 64, 8}) {
                if (!fits(SW, TH, false)) continue;
                long tiles = 0;
                int nby_max = 1;
                for (int i = 0; i < n; i++) {
                    tiles += (long)((jobs[i].W + SW - 1) / SW) * ((jobs[i].H + TH - 1) / TH);
                    nby_max = std::max(nby_max, (jobs[i].H + TH - 1) / TH);
                }
                for (int nk = 1; nk <= d; nk++) {
                    const int kg = (d + nk - 1) / nk;
                    if ((d + kg - 1) / kg != nk) continue;  // same split as a smaller count
                    const bool fz = can_fuse && nk == 1;
                    const size_t smem = score_smem(SW, TH, B, rmax, fz);
                    if (smem > 200 * 1024) continue;
                    int per_sm = 0;
                    err = emd_occupancy_kind(kind, KB, 0, smem, SW, &per_sm);
                    if (err != cudaSuccess) return err;
                    if (per_sm < 1) continue;
                    const long slots = (long)per_sm * n_sm;
                    for (int BR = 1; BR <= (fz ? 1 : nby_max); BR *= 2) {
                        double work = 0.0;
                        long ctas = 0;
                        for (int i = 0; i < n; i++) {
                            work += image_cost(jobs[i].H, jobs[i].W, d, B, jobs[i].r, SW, TH, kg, nk, BR);
                            const int nby = (jobs[i].H + TH - 1) / TH;
                            ctas += (long)((jobs[i].W + SW - 1) / SW) * ((nby + BR - 1) / BR) * nk;
                        }
                        (void)tiles;
                        const double waves = std::ceil((double)ctas / (double)slots);
                        // per-CTA average cost times the waves
                        const double cost = waves * (work / (double)ctas);
                        if (cost < best_cost * 0.999) best_cost = cost, best = ScoreTiling{SW, TH, nk, 0, BR};
                    }
                }
            }
        if (best.SW == 0) return cudaErrorNotSupported;  // nothing enqueued
        best.walk = tiling ? tiling->walk : 0;  // a walk asked for without a tiling (strip width 0)
    }
    // the shuffle walk exists for B = 32 with the u32 walk; elsewhere the per-thread walk runs
    if (best.walk == 1 && !(KB == 32 && kind != EmdKind::U64_U64)) best.walk = 0;
    const int SW = best.SW, TH = best.TH, walk = best.walk;
    const int kg = (d + best.n_kg - 1) / best.n_kg, n_kg = (d + kg - 1) / kg;
    const bool fuse = can_fuse && n_kg == 1;
    for (int i = 0; i < n; i++) max_nby = std::max(max_nby, (jobs[i].H + TH - 1) / TH);
    // bands per CTA: 0 asks for whole columns (every band of a strip); a fused tiling takes one
    int BR = best.bands <= 0 ? max_nby : std::min(best.bands, max_nby);
    if (fuse) BR = 1;
    best.bands = BR;
    if (chosen) *chosen = best;
    const size_t smem = score_smem(SW, TH, B, rmax, fuse);

    ScoreParams p;
    memset(&p, 0, sizeof(p));
    p.n = n, p.d = d, p.B = B, p.SW = SW, p.TH = TH, p.kg = kg, p.n_kg = n_kg, p.BR = BR;
    p.tile_bytes = (uint32_t)align_up((size_t)tile_rows(TH, rmax) * tcp_of(SW, rmax), 128);
    p.first_wait_tries = first_wait_tries;
    p.fuse = fuse ? 1 : 0;
    p.acc_off = (uint32_t)score_smem_core(SW, TH, B, rmax);
    FinParams f;
    memset(&f, 0, sizeof(f));
    f.n = n, f.d = d, f.B = B;
    long cta = 0, blk = 0;
    size_t off = 0;
    for (int i = 0; i < n; i++) {
        const ScoreJob &j = jobs[i];
        const long HW = (long)j.H * j.W;
        ScoreImgP &im = p.img[i];
        im.H = j.H, im.W = j.W, im.r = j.r, im.nbx = (j.W + SW - 1) / SW;
        im.cta0 = cta;
        const int nby = (j.H + TH - 1) / TH;
        cta += (long)im.nbx * ((nby + BR - 1) / BR) * n_kg;
        im.ref = j.ref, im.Nref = j.Nref;
        void *numer = nullptr;
        unsigned long long *accum = nullptr;
        if (ws_accumulates) {
            accum = (unsigned long long *)((char *)ws + off);
            off += align_up(sizeof(unsigned long long) * HW, 256);
        } else if (j.numer_out) {
            numer = j.numer_out;
        } else {
            numer = (char *)ws + off;
            off += align_up(out_bytes * (size_t)d * HW, 256);
        }
        im.numer = numer, im.accum = accum, im.score = j.score;
        err = make_tmap_u8_3d(&p.tmap[i], j.bins, (uint64_t)j.pitch, (uint64_t)j.H, (uint64_t)d, (uint64_t)j.pitch,
                              (uint64_t)j.H * j.pitch, (uint32_t)tcp_of(SW, j.r), (uint32_t)tile_rows(TH, j.r));
        if (err != cudaSuccess) return err;
        FinImgP &fi = f.img[i];
        fi.H = j.H, fi.W = j.W, fi.r = j.r, fi.Nref = j.Nref, fi.blk0 = blk;
        blk += (HW + 255) / 256;
        fi.numer = numer, fi.accum = accum, fi.score = j.score;
        fi.lo = j.lo, fi.hi = j.hi;
        if (j.lo && (accum || !j.hi || d > kFinMaxWeights)) return cudaErrorNotSupported;
    }
    for (int i = 0; i < n; i++)
        if (p.img[i].accum) {
            err = cudaMemsetAsync(p.img[i].accum, 0, sizeof(unsigned long long) * (size_t)jobs[i].H * jobs[i].W, st);
            if (err != cudaSuccess) return err;
        }
    switch (kind) {
    case EmdKind::U32_U32:
        launch_emd_kb<uint32_t, uint32_t>(KB, walk, cta, smem, SW, st, p, status);
        if (!fuse) QFCA_LAUNCH("k_finalize", st, k_finalize<uint32_t><<<(unsigned)blk, 256, 0, st>>>(f));
        break;
    case EmdKind::U32_U64:
        launch_emd_kb<uint32_t, unsigned long long>(KB, walk, cta, smem, SW, st, p, status);
        if (!fuse) QFCA_LAUNCH("k_finalize", st, k_finalize<unsigned long long><<<(unsigned)blk, 256, 0, st>>>(f));
        break;
    default:
        launch_emd_kb<unsigned long long, unsigned long long>(KB, walk, cta, smem, SW, st, p, status);
        if (!fuse) QFCA_LAUNCH("k_finalize", st, k_finalize<unsigned long long><<<(unsigned)blk, 256, 0, st>>>(f));
        break;
    }
    return cudaGetLastError();
}

}  // namespace

size_t score_jobs_workspace_bytes(const ScoreJob *jobs, int n, int d) {
    size_t b = 0;
    for (int i = 0; i < n; i++) b += align_up(sizeof(unsigned long long) * (size_t)jobs[i].H * jobs[i].W * d, 256);
    return b + 256;
}

bool score_shape_ok(int B, int r) {
    for (int SW : {128, 64})
        for (int TH : {16, 32, 8})
            if (score_smem(SW, TH, B, r) <= 200 * 1024 && tcp_of(SW, r) <= 256 && tile_rows(TH, r) <= 256) return true;
    return false;
}

cudaError_t launch_score_jobs(const ScoreJob *jobs, int n, int d, int B, void *ws, bool ws_accumulates, int *status,
                              cudaStream_t st, const ScoreTiling *tiling, ScoreTiling *chosen) {
    return launch_score_jobs_limited(jobs, n, d, B, ws, ws_accumulates, status, st, tiling, chosen, kTmaTries);
}

cudaError_t launch_score_jobs_limited(const ScoreJob *jobs, int n, int d, int B, void *ws, bool ws_accumulates,
                                      int *status, cudaStream_t st, const ScoreTiling *tiling, ScoreTiling *chosen,
                                      uint32_t first_wait_tries) {
    size_t off = 0;
    for (int i0 = 0; i0 < n; i0 += kMaxBatch) {
        const int m = std::min(kMaxBatch, n - i0);
        cudaError_t e = score_chunk(jobs + i0, m, d, B, (char *)ws + off, ws_accumulates, status, st, tiling, chosen,
                                    first_wait_tries);
        if (e != cudaSuccess) return e;
        for (int i = i0; i < i0 + m; i++)
            off += align_up((ws_accumulates ? 1 : (size_t)d) * sizeof(unsigned long long) * jobs[i].H * jobs[i].W, 256);
    }
    return cudaSuccess;
}

// ---------------------------------------------------------------- allocation-free variant

// Scratch of qfca_score_noalloc: the per-pixel sums of the integer EMD
// numerators, u64 [H][W], and the status word of its bounded waits.  Both live
// in the module image, so every device that loads the library holds them
// (4 MiB) until the process exits; no call allocates anything.
namespace {
constexpr long kNoAllocMaxPixels = 1L << 19;
__device__ __align__(256) unsigned long long g_noalloc_acc[kNoAllocMaxPixels];
__device__ __align__(256) int g_noalloc_flag;

// Probes of each CTA's first tile wait in the allocation-free path: the
// normal limit, or 0 (give up at once) while a test checks the timeout report.
std::atomic<uint32_t> g_noalloc_first_tries{kTmaTries};

// Device addresses of the two symbols for the current device.  In host code a
// __device__ symbol's name is only a host-side stand-in; the address is looked
// up on every call (a cheap table lookup that allocates nothing), so it stays
// valid if the application resets the device and the module is reloaded.
qfca_status noalloc_symbols(unsigned long long **acc, int **flag) {
    void *p = nullptr, *f = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_acc) != cudaSuccess || !p ||
        cudaGetSymbolAddress(&f, g_noalloc_flag) != cudaSuccess || !f) {
        cudaGetLastError();
        return QFCA_ERR_CUDA;
    }
    *acc = (unsigned long long *)p;
    *flag = (int *)f;
    return QFCA_OK;
}
}  // namespace

}  // namespace qfca

extern "C" qfca_status qfca_score_noalloc(const uint8_t *bins, int H, int W, int pitch, int d, int B, int r,
                                          const uint32_t *ref_hist, uint32_t ref_total, float *score,
                                          void *stream) {
    using namespace qfca;
    if (!bins || !ref_hist || !score) return QFCA_ERR_INVALID_ARG;
    if (H < 1 || W < 1 || pitch < W || pitch % 16 != 0 || ((uintptr_t)bins & 15) != 0) return QFCA_ERR_INVALID_ARG;
    if (d < 1 || d > kMaxPlanes || B < 2 || B > kMaxB || r < 1 || 2 * r + 1 > 127 || ref_total < 1)
        return QFCA_ERR_INVALID_ARG;
    if ((long)H * W > kNoAllocMaxPixels) return QFCA_ERR_UNSUPPORTED;
    unsigned long long *acc = nullptr;
    int *flag = nullptr;
    const qfca_status s = noalloc_symbols(&acc, &flag);
    if (s != QFCA_OK) return s;
    const ScoreJob job{bins, H, W, pitch, r, ref_hist, ref_total, score, nullptr};
    const cudaError_t e = launch_score_jobs_limited(&job, 1, d, B, acc, true, flag, (cudaStream_t)stream, nullptr,
                                                    nullptr, g_noalloc_first_tries.load());
    if (e == cudaErrorNotSupported) return QFCA_ERR_UNSUPPORTED;
    if (e != cudaSuccess) {
        cudaGetLastError();
        return QFCA_ERR_CUDA;
    }
    return QFCA_OK;
}

extern "C" qfca_status qfca_score_noalloc_status(int *out, void *stream) {
    using namespace qfca;
    if (!out) return QFCA_ERR_INVALID_ARG;
    unsigned long long *acc = nullptr;
    int *flag = nullptr;
    qfca_status s = noalloc_symbols(&acc, &flag);
    if (s != QFCA_OK) return s;
    int word = 0;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(&word, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return QFCA_ERR_CUDA;
    }
    *out = word;
    return word ? QFCA_ERR_TIMEOUT : QFCA_OK;
}

extern "C" qfca_status qfca_score_noalloc_test_wait_limit(int give_up_at_once) {
    qfca::g_noalloc_first_tries.store(give_up_at_once ? 0u : qfca::kTmaTries);
    return QFCA_OK;
}
