// gram.cu -- the covariance of the single-image PCA fit (arXiv 2510.15602,
// Sec. 3.3) with exact integer arithmetic on the BF16 tensor cores.
//
// GB300's FP64 pipe issues ~2 DFMA/clk/SM, so a plain FP64 Gram of a
// 256x256xC256 map costs ~5 ms.  Instead:
//   1. k_chan_absmax + k_chan_scale: per channel, the smallest e_c with |x_cp| < 2^e_c.
//   2. k_gram: y = x * 2^-e_c (exact, |y| < 1) is written as four signed 7-bit
//      digits, y ~= sum_i d_i 2^(-6-7i), d_i in [-64, 64] (round-to-nearest
//      splitting in FP32, each step exact); each digit is an integer, exact in
//      BF16.  For a 128x128 channel tile, tcgen05 accumulates in tensor memory
//      the level sums  A_L = sum_{i+j=L} sum_p d_i(c1,p) d_j(c2,p),  L = 0..3,
//      four FP32 accumulators of 128 columns.  Over a window of 512 pixels
//      every partial sum is an integer of magnitude <= 4 * 64 * 64 * 512 =
//      2^23, so the FP32 accumulation is exact; the window's sums are drained
//      into int64 registers, T += sum_L A_L << 7(4-L) (units of 2^-40), and
//      the CTA's totals are added into a global int64 Gram with integer
//      atomics (order-independent, so the result is deterministic).  Column
//      sums of the digits give the channel means.  On the diagonal the level-4
//      products sum_p (2 d1 d3 + d2^2) are added exactly as well (d2^2 >= 0
//      would otherwise bias every variance low); off the diagonal the dropped
//      level >= 4 products are zero-mean (<= 3 * 64^2 * 2^-40 each).  The
//      other rounding is the 27-bit fixed-point representation of y
//      (error <= 2^-28 2^e_c per element, round to nearest).
//   3. k_cov_finalize (FP64): mu_c = 2^e_c S_c / N,
//      Sigma_ij = 2^(e_i + e_j) T_ij 2^-40 / N - mu_i mu_j.
//
// One CTA (512 threads) = one 128x128 tile of the upper triangle x one range
// of pixels; per 32-pixel sub-chunk all threads convert both channel blocks
// into the 64-byte-swizzled K-major layout (channels are rows, pixels are K:
// NCHW is already K-major) of one of two operand buffers and arrive, one
// arrival per warp, on that buffer's `full` mbarrier; thread 0 waits for it,
// issues the sub-chunk's 12 MMAs (the 10 digit pairs stacked into 6 per K-step
// of 16) and commits to the buffer's `empty` mbarrier, which a warp waits for
// before converting into the buffer again.  No CTA-wide barrier in the loop:
// each warp runs ahead as far as the two buffers allow, and the features after
// next stream into shared memory with cp.async meanwhile.  At the end of a
// window thread 0 also commits to `acc_full`; every warp drains its TMEM
// quarter and arrives on `drained`, which thread 0 waits for before the next
// window's first MMA (it overwrites the accumulators).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.cuh"
#include "tc.cuh"

namespace qfca {
namespace {

constexpr int kTB = 128;         // channels per tile side
constexpr int kSub = 32;         // pixels per sub-chunk (one 64-B swizzle row of BF16)
constexpr int kSliceBytes = 128 * kSub * 2;  // one digit slice of a 128-channel block
constexpr int kBlockBytes = 4 * kSliceBytes; // the four slices of one block
constexpr int kStageRow = kSub + 4;           // floats per staged channel row (padded: rows start 4 banks apart)
constexpr int kStageBytes = 128 * kStageRow * 4;  // one block's FP32 features of a sub-chunk
constexpr int kWin = 512;        // pixels per exact accumulation window (level sums <= 4 * 64 * 64 * 512 = 2^23)
constexpr int kThreads = 512;
constexpr int kSlices = 4;
constexpr uint32_t kWaitTries = 1u << 26;
constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23: (v + kMagic) - kMagic rounds v to an integer

// Off-diagonal tile pair p (i < j, enumerated row by row) of nt channel tiles: returns i, sets j.
__device__ __forceinline__ int off_pair_idx(int p, int nt, int &j) {
    int i = 0;
    while (p >= nt - 1 - i) { p -= nt - 1 - i; i++; }
    j = i + 1 + p;
    return i;
}

// Per-image part of a table-driven fit launch.
struct FitImgP {
    const float *X;   // [C][N] (NCHW) or [N][C] (NHWC)
    long N;
    long chunk;       // pixels per Gram CTA (a multiple of the exact-accumulation window)
    int n_split;      // pixel ranges of this image
    long cta0;        // first Gram CTA of this image's off-diagonal tile pairs
    long cta0d;       // first Gram CTA of its diagonal tiles
};

struct FitParams {
    int n, C, layout, vec_ok, nt, n_pairs;
    long diag_start;  // the grid's off-diagonal CTAs (the longer ones) come first, then the diagonal
    FitImgP img[kMaxBatch];
};

// e_c = smallest exponent with max_p |x_cp| < 2^e_c  (stored as the max |x| bits first)
// Grid (x-chunks, C, images of the table).
__global__ void k_chan_absmax(const __grid_constant__ FitParams p, unsigned *__restrict__ amax) {
    const int c = blockIdx.y, C = p.C;
    const FitImgP &im = p.img[blockIdx.z];
    const float *X = im.X;
    const long N = im.N;
    amax += (long)blockIdx.z * C;
    unsigned m = 0;
    if (p.layout == QFCA_NCHW && p.vec_ok) {
        // 16-byte loads, four in flight per thread
        const float4 *row = reinterpret_cast<const float4 *>(X + (long)c * N);
        const long n4 = N / 4, stride = (long)gridDim.x * blockDim.x;
        long q = blockIdx.x * (long)blockDim.x + threadIdx.x;
        for (; q + 3 * stride < n4; q += 4 * stride) {
            float4 v[4];
#pragma unroll
            for (int u = 0; u < 4; u++) v[u] = __ldg(row + q + u * stride);
#pragma unroll
            for (int u = 0; u < 4; u++)
                m = max(max(m, max(__float_as_uint(v[u].x) & 0x7fffffffu, __float_as_uint(v[u].y) & 0x7fffffffu)),
                        max(__float_as_uint(v[u].z) & 0x7fffffffu, __float_as_uint(v[u].w) & 0x7fffffffu));
        }
        for (; q < n4; q += stride) {
            const float4 v = __ldg(row + q);
            m = max(max(m, max(__float_as_uint(v.x) & 0x7fffffffu, __float_as_uint(v.y) & 0x7fffffffu)),
                    max(__float_as_uint(v.z) & 0x7fffffffu, __float_as_uint(v.w) & 0x7fffffffu));
        }
    } else if (p.layout == QFCA_NCHW) {
        const float *row = X + (long)c * N;
        for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < N; q += (long)gridDim.x * blockDim.x)
            m = max(m, __float_as_uint(row[q]) & 0x7fffffffu);
    } else {
        for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < N; q += (long)gridDim.x * blockDim.x)
            m = max(m, __float_as_uint(X[q * C + c]) & 0x7fffffffu);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m) atomicMax(&amax[c], m);
}

// four 7-bit digits of y (|y| < 1): y ~= d0/2^6 + d1/2^13 + d2/2^20 + d3/2^27.
// Digit k rounds the remainder left by the digits above it, scaled by 2^(6+7k);
// the scaling is folded into the rounding add (a power-of-two product is exact,
// so the FMA rounds only once, to the integer) and each remainder r - d/2^m is
// exact (it is at most half a unit of the digit's place and keeps r's last
// bit), so the digits are those of the plain multiply / round / subtract chain.
__device__ __forceinline__ void digits4(float y, float &d0, float &d1, float &d2, float &d3) {
    d0 = __fsub_rn(__fmaf_rn(y, 64.0f, kMagic), kMagic);
    float r = __fmaf_rn(d0, -1.0f / 64.0f, y);
    d1 = __fsub_rn(__fmaf_rn(r, 8192.0f, kMagic), kMagic);
    r = __fmaf_rn(d1, -1.0f / 8192.0f, r);
    d2 = __fsub_rn(__fmaf_rn(r, 1048576.0f, kMagic), kMagic);
    r = __fmaf_rn(d2, -1.0f / 1048576.0f, r);
    d3 = __fsub_rn(__fmaf_rn(r, 134217728.0f, kMagic), kMagic);
}

// 64-byte swizzle (rows of 32 BF16 pixels): 16-B chunk c of row r lands at
// chunk c ^ ((r >> 1) & 3).
__device__ __forceinline__ uint32_t swz(int row, int chunk16) {
    return (uint32_t)(row * 64 + ((chunk16 ^ ((row >> 1) & 3)) << 4));
}

// Stage one operand block (128 channels starting at c0) of pixels [q0, q0+32)
// into shared memory as FP32 [128][32]: thread t copies channel row t >> 2,
// 8 consecutive pixels -- two asynchronous 16-byte copies when the row is
// 16-byte aligned and complete, else plain loads and stores (zero outside).
__device__ __forceinline__ void stage_block(const float *__restrict__ X, int layout, int vec_ok, int C, long N, int c0,
                                            long q0, long q1, float *stage) {
    const int row = threadIdx.x >> 2, g = threadIdx.x & 3;
    const int c = c0 + row;
    const long p = q0 + g * 8;
    float *dst = stage + row * kStageRow + g * 8;
    if (vec_ok && c < C && p + 8 <= q1) {
        const uint32_t d = tc::smem_u32(dst);
        tc::cp_async16(d, X + (long)c * N + p);
        tc::cp_async16(d + 16, X + (long)c * N + p + 4);
    } else {
#pragma unroll
        for (int e = 0; e < 8; e++) {
            const long pe = p + e;
            dst[e] = (c < C && pe < q1) ? (layout == QFCA_NCHW ? X[(long)c * N + pe] : X[pe * C + c]) : 0.0f;
        }
    }
}

// This thread's 8 values of a staged block (the ones it staged itself).
__device__ __forceinline__ void read_stage(const float *stage, float (&v)[8]) {
    const int row = threadIdx.x >> 2, g = threadIdx.x & 3;
    const float4 a = *reinterpret_cast<const float4 *>(stage + row * kStageRow + g * 8);
    const float4 b = *reinterpret_cast<const float4 *>(stage + row * kStageRow + g * 8 + 4);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

// Convert this thread's 8 values of a block into its 4 digit slices, packed as
// BF16 pairs in registers (pk[slice]); with `slot` (this thread's five counters, stride
// kThreads), also add its digit sums per slice and its level-4 diagonal terms
// 2 d1 d3 + d2^2 (exact in FP32: 8 digits of magnitude <= 64, and 8 terms <= 3 * 2^12; the
// integer conversion by the magic-number add is exact below 2^22).  The operand buffer is
// written afterwards (store_slice), so the conversion can run while the buffer is still
// being read.
__device__ __forceinline__ int small_int(float v) { return __float_as_int(__fadd_rn(v, kMagic)) - 0x4B400000; }
__device__ __forceinline__ void convert_block(const float (&v)[8], float s, uint4 (&pk)[kSlices],
                                              int *__restrict__ slot /* [5][kThreads] at this thread, or null */) {
    float dd[kSlices][8];
#pragma unroll
    for (int e = 0; e < 8; e++) digits4(__fmul_rn(v[e], s), dd[0][e], dd[1][e], dd[2][e], dd[3][e]);
#pragma unroll
    for (int sl = 0; sl < kSlices; sl++) {
        pk[sl].x = tc::pack_bf16x2(dd[sl][0], dd[sl][1]);
        pk[sl].y = tc::pack_bf16x2(dd[sl][2], dd[sl][3]);
        pk[sl].z = tc::pack_bf16x2(dd[sl][4], dd[sl][5]);
        pk[sl].w = tc::pack_bf16x2(dd[sl][6], dd[sl][7]);
        if (slot) {
            const float t = ((dd[sl][0] + dd[sl][1]) + (dd[sl][2] + dd[sl][3])) +
                            ((dd[sl][4] + dd[sl][5]) + (dd[sl][6] + dd[sl][7]));
            slot[sl * kThreads] += small_int(t);
        }
    }
    if (slot) {
        float t4 = 0.0f;
#pragma unroll
        for (int e = 0; e < 8; e++) t4 = fmaf(dd[2][e], dd[2][e], fmaf(2.0f * dd[1][e], dd[3][e], t4));
        slot[kSlices * kThreads] += small_int(t4);
    }
}

// Both BF16 halves of a packed pair divided by two: the exponent of each nonzero half
// lowered by one (the digits are integers of magnitude <= 64, so no half is subnormal and
// the halving is exact; a zero stays zero, and no borrow crosses the halves).
__device__ __forceinline__ uint32_t half_bf16x2(uint32_t w) {
    const uint32_t hi = (w & 0x7F800000u) ? 0x00800000u : 0u, lo = (w & 0x00007F80u) ? 0x00000080u : 0u;
    return w - (hi | lo);
}
__device__ __forceinline__ uint4 half_bf16x2(const uint4 &w) {
    return make_uint4(half_bf16x2(w.x), half_bf16x2(w.y), half_bf16x2(w.z), half_bf16x2(w.w));
}

// One packed slice into slot `sl` of an operand buffer (K-major, 64-byte swizzle).
__device__ __forceinline__ void store_slice(const uint4 &pk, uint8_t *slices, int sl) {
    const int row = threadIdx.x >> 2, g = threadIdx.x & 3;
    *reinterpret_cast<uint4 *>(slices + sl * kSliceBytes + swz(row, g)) = pk;
}

// The packed digits into the K-major, 64-byte-swizzled slices of an operand buffer.
__device__ __forceinline__ void store_block(const uint4 (&pk)[kSlices], uint8_t *slices) {
    const int row = threadIdx.x >> 2, g = threadIdx.x & 3;
#pragma unroll
    for (int sl = 0; sl < kSlices; sl++) *reinterpret_cast<uint4 *>(slices + sl * kSliceBytes + swz(row, g)) = pk[sl];
}

// The level sums of one 32-pixel sub-chunk: A_L += sum_{i+j=L} D_i E_j^T for
// L = 0..3 (D: the A block's digit slices, E: the B block's).  The B slices
// lie back to back in shared memory (128 rows each, the same 512-B row-group
// stride), so slices j..j+1 form one 256-row operand: A_i times slices
// j0..j0+1 fills the accumulators of levels i+j0 and i+j0+1 (TMEM columns
// 128 (i+j0) .. +256) in one N = 256 instruction.  Per K-step: A_0 x E_0..1
// and A_0 x E_2..3 (issued first: they start all four levels of a window),
// A_1 x E_0..1, A_1 x E_2, A_2 x E_0..1, A_3 x E_0 -- 6 MMAs instead of 10.
__device__ __forceinline__ void issue_level_mmas(uint32_t tmem, uint32_t a_addr, uint32_t b_addr, bool first) {
    const uint64_t ad0 = tc::sdesc_kmajor_sw64(a_addr), bd0 = tc::sdesc_kmajor_sw64(b_addr);
    constexpr uint32_t id256 = tc::idesc_bf16_f32(kTB, 256), id128 = tc::idesc_bf16_f32(kTB, 128);
    const uint32_t acc0 = first ? 0u : 1u;
#pragma unroll
    for (int ks = 0; ks < kSub / 16; ks++) {
        // descriptors differ only in the start-address field (bytes >> 4)
        auto A = [&](int i) { return ad0 + (uint64_t)((i * kSliceBytes + ks * 32) >> 4); };
        auto E = [&](int j) { return bd0 + (uint64_t)((j * kSliceBytes + ks * 32) >> 4); };
        const uint32_t a0 = ks == 0 ? acc0 : 1u;
        tc::mma_bf16_ss(tmem + 0 * kTB, A(0), E(0), id256, a0);  // levels 0, 1
        tc::mma_bf16_ss(tmem + 2 * kTB, A(0), E(2), id256, a0);  // levels 2, 3
        tc::mma_bf16_ss(tmem + 1 * kTB, A(1), E(0), id256, 1u);  // levels 1, 2
        tc::mma_bf16_ss(tmem + 3 * kTB, A(1), E(2), id128, 1u);  // level 3
        tc::mma_bf16_ss(tmem + 2 * kTB, A(2), E(0), id256, 1u);  // levels 2, 3
        tc::mma_bf16_ss(tmem + 3 * kTB, A(3), E(0), id128, 1u);  // level 3
    }
}

// A diagonal tile (A = B = the block's digits D_0..D_3) needs only the symmetric part
// of the level sums: with Y_L = sum over i <= j, i + j = L of c_ij D_i D_j^T, c_ij = 1 for
// i < j and 1/2 for i = j, T = Y + Y^T (the halves exact in BF16 and in the FP32
// accumulators).  Slots of the buffer: [D_0][D_0/2][D_1][D_1/2][D_2][D_3]; per K-step
// D_0 x [D_0/2 | D_1] (levels 0, 1), D_0 x [D_2 | D_3] and D_1 x [D_1/2 | D_2] (levels 2, 3):
// three N = 256 MMAs instead of six.
__device__ __forceinline__ void issue_level_mmas_sym(uint32_t tmem, uint32_t addr, bool first) {
    const uint64_t d0 = tc::sdesc_kmajor_sw64(addr);
    constexpr uint32_t id256 = tc::idesc_bf16_f32(kTB, 256);
    const uint32_t acc0 = first ? 0u : 1u;
#pragma unroll
    for (int ks = 0; ks < kSub / 16; ks++) {
        auto S = [&](int sl) { return d0 + (uint64_t)((sl * kSliceBytes + ks * 32) >> 4); };
        const uint32_t a0 = ks == 0 ? acc0 : 1u;
        tc::mma_bf16_ss(tmem + 0 * kTB, S(0), S(1), id256, a0);  // levels 0, 1
        tc::mma_bf16_ss(tmem + 2 * kTB, S(0), S(4), id256, a0);  // levels 2, 3
        tc::mma_bf16_ss(tmem + 2 * kTB, S(2), S(3), id256, 1u);  // levels 2, 3
    }
}

// Grid: images * n_pairs * n_split CTAs, off-diagonal tile pairs first.  Per image: Gint [C][C] int64 (upper
// tiles accumulated), Dsum [4][C] int64, scale [C].  Two operand buffers: the
// threads convert sub-chunk k into buffer k & 1 while the tensor cores work on
// sub-chunk k - 1 from the other buffer; a buffer is rewritten only after the
// MMAs that read it have completed (one mbarrier per buffer, bounded waits).
__global__ void __launch_bounds__(kThreads, 1) k_gram(const __grid_constant__ FitParams p,
                                                      const float *__restrict__ scale,
                                                      unsigned long long *__restrict__ Gint,
                                                      unsigned long long *__restrict__ Dsum,
                                                      int *__restrict__ status) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = tc::align_smem<1024>(smem_raw);
    // operand buffer b: A slices at smem + 2 b kBlockBytes, B slices right after (4 slices x 8 KB each)
    auto As = [&](int b) { return smem + 2 * b * kBlockBytes; };
    auto Bs = [&](int b) { return smem + (2 * b + 1) * kBlockBytes; };
    float *stg = (float *)(smem + 4 * kBlockBytes);                 // [2 stages][2 blocks][128][kStageRow] FP32
    uint64_t *bar = (uint64_t *)(smem + 4 * kBlockBytes + 4 * kStageBytes);  // [7] mbarriers + the abort flag
    uint32_t *tmem_slot = (uint32_t *)(bar + 8);
    int *slots = (int *)(tmem_slot + 4);  // [5][kThreads]: per-thread digit sums (4 slices) and level-4 terms

    const long cta = blockIdx.x;
    const bool diag = cta >= p.diag_start;
    const int img = diag ? table_image(p.n, cta, [&](int i) { return p.img[i].cta0d; })
                         : table_image(p.n, cta, [&](int i) { return p.img[i].cta0; });
    const FitImgP &im = p.img[img];
    const int C = p.C, layout = p.layout, vec_ok = p.vec_ok, nt = p.nt, n_off = p.n_pairs - p.nt;
    const long N = im.N, chunk = im.chunk;
    const float *X = im.X;
    const int rem = (int)(cta - (diag ? im.cta0d : im.cta0));
    int ti, tj, split;
    if (diag) {
        ti = tj = rem % nt;
        split = rem / nt;
    } else {
        ti = off_pair_idx(rem % n_off, nt, tj);
        split = rem / n_off;
    }
    scale += (long)img * C;
    Gint += (long)img * C * C;
    Dsum += (long)img * kSlices * C;
    const long p0 = (long)split * chunk, p1 = min(N, p0 + chunk);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (warp == 0) {
        tc::tmem_alloc(tmem_slot, 512);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(&bar[0], kThreads / 32);  // full[0], full[1]: one arrival per warp
        tc::mbar_init(&bar[1], kThreads / 32);
        tc::mbar_init(&bar[2], 1);              // empty[0], empty[1]: tcgen05.commit
        tc::mbar_init(&bar[3], 1);
        tc::mbar_init(&bar[4], 1);              // acc_full: tcgen05.commit
        tc::mbar_init(&bar[5], kThreads / 32);  // drained: one arrival per warp
        tc::mbar_init(&bar[6], 1);              // fin: the last commit after a failure
        *reinterpret_cast<volatile int *>(&bar[7]) = 0;
        tc::fence_mbar_init();
    }
    for (int sl = 0; sl <= kSlices; sl++) slots[sl * kThreads + tid] = 0;
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    long long tot[32];
#pragma unroll
    for (int j = 0; j < 32; j++) tot[j] = 0;
    const int q = warp & 3, cg4 = warp >> 2;  // TMEM lane quarter, 32-column group
    // the scales of this thread's channel row in both blocks, loaded once
    const int crow = tid >> 2;
    const float sA = ti * kTB + crow < C ? scale[ti * kTB + crow] : 0.0f;
    const float sB = tj * kTB + crow < C ? scale[tj * kTB + crow] : 0.0f;
    // full[b]: the 16 warps converted into buffer b; empty[b]: the MMAs reading buffer b
    // completed; acc_full: a window's MMAs completed; drained: the 16 warps read the window
    uint64_t *full = bar, *empty = bar + 2, *acc_full = bar + 4, *drained = bar + 5, *fin = bar + 6;
    volatile int *abort_flag = reinterpret_cast<volatile int *>(bar + 7);
    bool failed = false;
    // bounded wait that also gives up as soon as another warp has given up
    auto bwait = [&](uint64_t *b, uint32_t parity) -> bool {
        for (uint32_t n = 0; n < kWaitTries; n += 1u << 12) {
            if (tc::mbar_wait(b, parity, 1u << 12)) return true;
            if (*abort_flag) return false;
        }
        *abort_flag = 1;
        return false;
    };

    // features stream into two FP32 stages, two sub-chunks ahead of the conversion
    auto stage = [&](int s, long q0) {
        float *sa = stg + (size_t)s * 2 * kTB * kStageRow;
        if (q0 < p1) {
            stage_block(X, layout, vec_ok, C, N, ti * kTB, q0, p1, sa);
            if (!diag) stage_block(X, layout, vec_ok, C, N, tj * kTB, q0, p1, sa + kTB * kStageRow);
        }
        tc::cp_async_commit();  // one group per sub-chunk (possibly empty)
    };
    stage(0, p0);
    stage(1, p0 + kSub);
    int kk = 0, in_win = 0, win = 0, issued_windows = 0;
    bool pending = false;  // a window's MMAs are issued and its accumulators not drained yet
    // drain window `win`'s exact level sums into int64 (acc_full covers every MMA of the window)
    auto drain = [&]() -> bool {
        if (!bwait(acc_full, win & 1)) return false;
        tc::tc_fence_after();
#pragma unroll
        for (int L = 0; L < 4; L++) {
            uint32_t r0[16], r1[16];
            const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(L * kTB + 32 * cg4);
            tc::tmem_ld16(ta, r0);
            tc::tmem_ld16(ta + 16, r1);
            tc::tmem_wait_ld();
            // levels 0 and 2 of a diagonal tile hold half-integers: 2 A_L, one shift less.
            // Every level sum is an exact FP32 integer; all are within 2^22 (the exact range of
            // the magic-number conversion) except level 3 of an off-diagonal tile (four
            // products: up to 2^23), which takes the exact float-to-int instruction
            const bool hl = diag && (L == 0 || L == 2), wide = !diag && L == 3;
            const float m2 = hl ? 2.0f : 1.0f;
            const int sh = 7 * (4 - L) - (hl ? 1 : 0);
#pragma unroll
            for (int jj = 0; jj < 16; jj++) {
                const float f0 = __fmul_rn(__uint_as_float(r0[jj]), m2), f1 = __fmul_rn(__uint_as_float(r1[jj]), m2);
                const int v0 = wide ? __float2int_rn(f0) : small_int(f0);
                const int v1 = wide ? __float2int_rn(f1) : small_int(f1);
                tot[jj] += (long long)v0 << sh;
                tot[16 + jj] += (long long)v1 << sh;
            }
        }
        tc::tc_fence_before();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive_cta(drained);
        win++;
        return true;
    };
    for (long q0 = p0; q0 < p1; q0 += kSub, kk++) {
        const int bsel = kk & 1;
        if (*abort_flag) { failed = true; break; }
        tc::cp_async_wait<1>();  // this thread's copies of sub-chunk kk have landed (kk+1 may be in flight)
        // the A block is converted into registers while the MMAs of sub-chunk kk-2 may
        // still read the buffer (the registers of a second block would spill)
        const float *sa = stg + (size_t)bsel * 2 * kTB * kStageRow;
        uint4 pk[kSlices];
        {
            float v[8];
            read_stage(sa, v);
            convert_block(v, sA, pk, diag ? slots + tid : nullptr);
        }
        // the MMAs of sub-chunk kk-2 read this operand buffer
        if (kk >= 2 && !bwait(&empty[bsel], ((kk - 2) >> 1) & 1)) { failed = true; break; }
        if (diag) {
            uint8_t *buf = As(bsel);  // six slots across the A and B halves of the buffer
            store_slice(pk[0], buf, 0);
            store_slice(half_bf16x2(pk[0]), buf, 1);
            store_slice(pk[1], buf, 2);
            store_slice(half_bf16x2(pk[1]), buf, 3);
            store_slice(pk[2], buf, 4);
            store_slice(pk[3], buf, 5);
        } else {
            store_block(pk, As(bsel));
            float v[8];
            read_stage(sa + kTB * kStageRow, v);
            convert_block(v, sB, pk, nullptr);
            store_block(pk, Bs(bsel));
        }
        // each thread reads back only what it staged itself, so the stage can be
        // refilled (sub-chunk kk+2) right away
        stage(bsel, q0 + 2 * kSub);
        tc::fence_proxy_async_smem();  // this thread's operand writes, visible to the tensor cores
        __syncwarp();
        if (lane == 0) tc::mbar_arrive_cta(&full[bsel]);
        // the previous window is drained only now, so that its last MMAs complete behind this
        // sub-chunk's conversion; the first MMA of this window waits for `drained`
        if (pending) {
            if (!drain()) { failed = true; break; }
            pending = false;
        }
        const bool first = in_win == 0;
        in_win += kSub;
        const bool win_end = in_win >= kWin || q0 + kSub >= p1;
        if (tid == 0) {
            bool ok = bwait(&full[bsel], (kk >> 1) & 1);
            // the first MMA of a window overwrites the accumulators the warps drained
            if (ok && first && win > 0) ok = bwait(drained, (win - 1) & 1);
            if (ok) {
                tc::tc_fence_after();
                const uint32_t a_addr = tc::smem_u32(As(bsel));
                if (diag) issue_level_mmas_sym(tmem, a_addr, first);
                else issue_level_mmas(tmem, a_addr, tc::smem_u32(Bs(bsel)), first);
                tc::mma_commit(&empty[bsel]);
                if (win_end) {
                    tc::mma_commit(acc_full);
                    issued_windows++;
                }
            }
        }
        __syncwarp();
        if (win_end) {
            pending = true;
            in_win = 0;
        }
    }
    if (!failed && pending && !drain()) failed = true;
    __syncthreads();
    failed = failed || *abort_flag;
    if (failed) {
        if (tid == 0) {
            atomicOr(status, kStatusMmaTimeout);
            // every MMA issued so far completes (bounded) before the accumulators are freed
            tc::mma_commit(fin);
            tc::mbar_wait(fin, 0, kWaitTries);
        }
    } else {
        const int c1 = ti * kTB + 32 * q + lane;
        if (c1 < C) {
#pragma unroll
            for (int jj = 0; jj < 32; jj++) {
                const int c2 = tj * kTB + 32 * cg4 + jj;
                if (c2 >= C || tot[jj] == 0) continue;
                if (!diag) {
                    atomicAdd(&Gint[(long)c1 * C + c2], (unsigned long long)tot[jj]);
                } else if (c1 == c2) {  // T = Y + Y^T
                    atomicAdd(&Gint[(long)c1 * C + c2], (unsigned long long)(2 * tot[jj]));
                } else {
                    atomicAdd(&Gint[(long)c1 * C + c2], (unsigned long long)tot[jj]);
                    atomicAdd(&Gint[(long)c2 * C + c1], (unsigned long long)tot[jj]);
                }
            }
        }
        __syncthreads();  // every thread's counters complete
        if (diag && tid < kTB) {  // row tid: the counters of its four threads 4 tid .. 4 tid + 3
            const int c = ti * kTB + tid;
            if (c < C) {
                for (int sl = 0; sl <= kSlices; sl++) {
                    const int *t = slots + sl * kThreads + 4 * tid;
                    const long long v = (long long)t[0] + t[1] + t[2] + t[3];
                    if (v == 0) continue;
                    if (sl < kSlices) atomicAdd(&Dsum[(long)sl * C + c], (unsigned long long)v);
                    else atomicAdd(&Gint[(long)c * C + c], (unsigned long long)v);
                }
            }
        }
    }
    (void)issued_windows;
    tc::cp_async_wait<0>();  // no copy into this CTA's shared memory outlives it
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, 512);
    }
}

__global__ void k_chan_scale(const unsigned *__restrict__ amax, int C, float *__restrict__ scale, int *__restrict__ ex) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;  // over images * C
    if (c >= C) return;
    const unsigned b = amax[c];
    int e = 0;
    if (b != 0) {
        int eb = (int)(b >> 23);           // biased exponent of max |x|
        e = eb - 127 + 1;                  // max |x| < 2^(eb-127+1)
        if (eb == 0) e = -126;             // subnormal maximum
    }
    ex[c] = e;
    scale[c] = ldexpf(1.0f, -e);
}

// Sigma_ij = 2^(e_i+e_j) T_ij 2^-40 / N - mu_i mu_j ;  mu_c = 2^e_c S_c / N,
// S_c = sum_i D_i,c 2^(-6-7i).  Writes mean[C] and the full symmetric cov[C][C]
// of each image (grid.y = image).  One block = one 32 x 32 tile of the output
// (grid.x = tile): it forms the means and powers of two of its 32 rows and 32
// columns only, reads its tile of the upper triangle of T coalesced (rows
// a0.., columns b0.. with a0 <= b0) and, below the diagonal, writes it
// transposed through shared memory; every entry is formed from T[min][max]
// with the same operations in the same order as for the entry above the
// diagonal, so the matrix is exactly symmetric.
constexpr int kFinT = 32;
__global__ void __launch_bounds__(256) k_cov_finalize(const __grid_constant__ FitParams p,
                                                       const unsigned long long *__restrict__ Gint,
                                                       const unsigned long long *__restrict__ Dsum,
                                                       const int *__restrict__ ex, double *__restrict__ mean,
                                                       double *__restrict__ cov, float2 *__restrict__ cov_ff) {
    __shared__ long long Ts[kFinT][kFinT + 1];
    __shared__ double mu_s[2][kFinT], pw_s[2][kFinT];  // [0]: the tile's rows, [1]: its columns
    const long img = blockIdx.y;
    const int C = p.C, nt = (C + kFinT - 1) / kFinT;
    const int ti = (int)(blockIdx.x / nt), tj = (int)(blockIdx.x % nt);
    const double invN = 1.0 / (double)p.img[img].N;
    Gint += img * C * C;
    Dsum += img * kSlices * C;
    ex += img * C;
    mean += img * C;
    cov += img * C * C;
    if (cov_ff) cov_ff += img * C * C;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
    // 2^e_c and mu_c = 2^e_c S_c / N of the tile's rows and columns (powers of two: every scaling is exact)
    constexpr double kSl[kSlices] = {0x1p-6, 0x1p-13, 0x1p-20, 0x1p-27};
    if (threadIdx.x < 2 * kFinT) {
        const int side = threadIdx.x / kFinT, c = (side ? tj : ti) * kFinT + tx;
        double s = 0.0, pw = 1.0;
        if (c < C) {
            for (int sl = 0; sl < kSlices; sl++) s += (double)(long long)Dsum[(long)sl * C + c] * kSl[sl];
            pw = ldexp(1.0, ex[c]);
        }
        pw_s[side][tx] = pw;
        mu_s[side][tx] = s * pw * invN;
    }
    // the tile of the upper triangle that holds this tile's entries: rows a0.., columns b0..
    const int a0 = min(ti, tj) * kFinT, b0 = max(ti, tj) * kFinT;
    for (int y = ty; y < kFinT; y += 8) {
        const int a = a0 + y, b = b0 + tx;
        Ts[y][tx] = (a < C && b < C) ? (long long)Gint[(long)a * C + b] : 0;
    }
    __syncthreads();
    for (int y = ty; y < kFinT; y += 8) {
        const int i = ti * kFinT + y, j = tj * kFinT + tx;
        if (i >= C || j >= C) continue;
        // entry (i, j) from T[min(i, j)][max(i, j)]; (la, lb): its row and column within Ts
        const bool upper = ti < tj || (ti == tj && y <= tx);
        const int la = upper ? y : tx, lb = upper ? tx : y;
        // the row channel min(i, j) and the column channel max(i, j), as the upper entry takes them
        const int sa = ti <= tj ? 0 : 1, sb = 1 - sa;  // which side holds channel a (rows: 0, columns: 1)
        const int ca = ti == tj ? la : (sa == 0 ? y : tx), cb = ti == tj ? lb : (sb == 0 ? y : tx);
        const double mi = mu_s[ti == tj ? 0 : sa][ca], mj = mu_s[ti == tj ? 1 : sb][cb];
        const double pa = pw_s[ti == tj ? 0 : sa][ca], pb = pw_s[ti == tj ? 1 : sb][cb];
        const double g = (double)Ts[la][lb] * (pa * pb * 0x1p-40) * invN;
        const double v = g - mi * mj;
        cov[(long)i * C + j] = v;
        if (cov_ff) {
            const float h = (float)v;
            cov_ff[(long)i * C + j] = make_float2(h, (float)(v - (double)h));
        }
        if (i == j) mean[i] = mi;
    }
}

}  // namespace

struct GramPlan {
    int nt, n_pairs;
    size_t off_amax, off_scale, off_ex, off_G, off_D, total, smem;
};

static GramPlan gram_plan(int C, int nimg) {
    GramPlan g{};
    g.nt = (C + kTB - 1) / kTB;
    g.n_pairs = g.nt * (g.nt + 1) / 2;
    size_t o = 0;
    auto take = [&](size_t b) { size_t at = o; o = align_up(o + b, 256); return at; };
    g.off_amax = take(sizeof(unsigned) * (size_t)C * nimg);
    g.off_scale = take(sizeof(float) * (size_t)C * nimg);
    g.off_ex = take(sizeof(int) * (size_t)C * nimg);
    g.off_G = take(sizeof(unsigned long long) * (size_t)C * C * nimg);
    g.off_D = take(sizeof(unsigned long long) * (size_t)kSlices * C * nimg);
    g.total = o;
    g.smem = 1024 + 4 * (size_t)kBlockBytes + 4 * (size_t)kStageBytes + 128 + sizeof(int) * (kSlices + 1) * kThreads;
    return g;
}

size_t gram_workspace_bytes(int C, long N, int nimg) {
    (void)N;
    return gram_plan(C, nimg).total;
}

// mean[n][C] and cov[n][C][C] (FP64) of the n feature maps of `jobs` (one
// launch per stage for up to kMaxBatch images); ws: gram_workspace_bytes(C, *, n).
cudaError_t launch_gram_cov_jobs(const FitJob *jobs, int n, int layout, int C, double *mean, double *cov, void *cov_ff,
                                 void *ws, int *status, cudaStream_t st) {
    const GramPlan g = gram_plan(C, n);
    char *b = (char *)ws;
    unsigned *amax = (unsigned *)(b + g.off_amax);
    float *scale = (float *)(b + g.off_scale);
    int *ex = (int *)(b + g.off_ex);
    unsigned long long *G = (unsigned long long *)(b + g.off_G);
    unsigned long long *D = (unsigned long long *)(b + g.off_D);
    cudaError_t e = cudaMemsetAsync(amax, 0, sizeof(unsigned) * (size_t)C * n, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(G, 0, sizeof(unsigned long long) * (size_t)C * C * n, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(D, 0, sizeof(unsigned long long) * kSlices * (size_t)C * n, st);
    if (e != cudaSuccess) return e;
    static DeviceOnce attrs;
    int dev = 0;
    cudaGetDevice(&dev);
    e = device_once(attrs, dev, [&] {
        return cudaFuncSetAttribute(k_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem);
    });
    if (e != cudaSuccess) return e;
    int n_sm = 0;
    if ((e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    for (int i0 = 0; i0 < n; i0 += kMaxBatch) {
        const int m = n - i0 < kMaxBatch ? n - i0 : kMaxBatch;
        FitParams p;
        memset(&p, 0, sizeof(p));
        p.n = m, p.C = C, p.layout = layout, p.nt = g.nt, p.n_pairs = g.n_pairs;
        // float4 loads need 16-B aligned rows: NCHW, N % 4 == 0, X 16-B aligned (every image)
        int vec_ok = layout == QFCA_NCHW;
        long total_px = 0, max_n = 1;
        for (int i = 0; i < m; i++) {
            const FitJob &j = jobs[i0 + i];
            vec_ok = vec_ok && j.N % 4 == 0 && ((uintptr_t)j.X & 15) == 0;
            total_px += j.N;
            max_n = j.N > max_n ? j.N : max_n;
        }
        p.vec_ok = vec_ok;
        // about two waves of one CTA per SM (one for a single image), chunks a multiple of the window
        const long target = m == 1 ? n_sm : 2L * n_sm;
        long chunk = (total_px * g.n_pairs + target - 1) / target;
        chunk = (chunk + kWin - 1) / kWin * kWin;
        if (chunk < kWin) chunk = kWin;
        // a thread's int32 counters see chunk / 4 pixels: at most 2^16 x 3 * 2^12 level-4 terms
        if (chunk > (1L << 18)) chunk = 1L << 18;
        // all images' off-diagonal tile pairs first (each converts two channel blocks and
        // issues all ten digit products, the longest CTAs), then the diagonal tiles
        long cta = 0;
        for (int i = 0; i < m; i++) {
            const FitJob &j = jobs[i0 + i];
            FitImgP &im = p.img[i];
            im.X = j.X, im.N = j.N, im.chunk = chunk;
            im.n_split = (int)((j.N + chunk - 1) / chunk);
            im.cta0 = cta;
            cta += (long)im.n_split * (g.n_pairs - g.nt);
        }
        p.diag_start = cta;
        for (int i = 0; i < m; i++) {
            p.img[i].cta0d = cta;
            cta += (long)p.img[i].n_split * g.nt;
        }
        unsigned *am = amax + (size_t)i0 * C;
        float *sc = scale + (size_t)i0 * C;
        int *exi = ex + (size_t)i0 * C;
        unsigned long long *Gi = G + (size_t)i0 * C * C;
        unsigned long long *Di = D + (size_t)i0 * kSlices * C;
        const int xb = (int)((max_n + 256 * 64 - 1) / (256 * 64));
        QFCA_LAUNCH("k_chan_absmax", st, k_chan_absmax<<<dim3(xb < 1 ? 1 : xb, C, m), 256, 0, st>>>(p, am));
        QFCA_LAUNCH("k_chan_scale", st,
                    k_chan_scale<<<(unsigned)((C * m + 127) / 128), 128, 0, st>>>(am, C * m, sc, exi));
        QFCA_LAUNCH("k_gram", st, k_gram<<<(unsigned)cta, kThreads, g.smem, st>>>(p, sc, Gi, Di, status));
        const int nt32 = (C + kFinT - 1) / kFinT;
        QFCA_LAUNCH("k_cov_finalize", st,
                    k_cov_finalize<<<dim3((unsigned)(nt32 * nt32), m), 256, 0, st>>>(
                        p, Gi, Di, exi, mean + (size_t)i0 * C, cov + (size_t)i0 * C * C,
                        cov_ff ? (float2 *)cov_ff + (size_t)i0 * C * C : nullptr));
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_chan_absmax_jobs(const FitJob *jobs, int n, int layout, int C, unsigned *amax, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(amax, 0, sizeof(unsigned) * (size_t)C * n, st);
    for (int i0 = 0; i0 < n && e == cudaSuccess; i0 += kMaxBatch) {
        const int m = n - i0 < kMaxBatch ? n - i0 : kMaxBatch;
        FitParams p;
        memset(&p, 0, sizeof(p));
        p.n = m, p.C = C, p.layout = layout;
        long max_n = 1;
        int vec_ok = layout == QFCA_NCHW;
        for (int i = 0; i < m; i++) {
            p.img[i].X = jobs[i0 + i].X, p.img[i].N = jobs[i0 + i].N;
            max_n = jobs[i0 + i].N > max_n ? jobs[i0 + i].N : max_n;
            vec_ok = vec_ok && jobs[i0 + i].N % 4 == 0 && ((uintptr_t)jobs[i0 + i].X & 15) == 0;
        }
        p.vec_ok = vec_ok;
        const int xb = (int)((max_n + 256 * 64 - 1) / (256 * 64));
        QFCA_LAUNCH("k_chan_absmax", st,
                    k_chan_absmax<<<dim3(xb < 1 ? 1 : xb, C, m), 256, 0, st>>>(p, amax + (size_t)i0 * C));
        e = cudaGetLastError();
    }
    return e;
}

cudaError_t launch_gram_cov(const float *X, int layout, int C, long N, int nimg, double *mean, double *cov,
                            void *cov_ff, void *ws, int *status, cudaStream_t st) {
    // chunks of kMaxBatch images reuse the workspace in stream order
    FitJob jobs[kMaxBatch];
    for (int i0 = 0; i0 < nimg; i0 += kMaxBatch) {
        const int m = nimg - i0 < kMaxBatch ? nimg - i0 : kMaxBatch;
        for (int i = 0; i < m; i++) jobs[i] = FitJob{X + (long)(i0 + i) * C * N, N};
        cudaError_t e = launch_gram_cov_jobs(jobs, m, layout, C, mean + (size_t)i0 * C, cov + (size_t)i0 * C * C,
                                             cov_ff ? (float2 *)cov_ff + (size_t)i0 * C * C : nullptr, ws, status, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace qfca
