// assoc.cu -- the paper's own per-pixel scoring (arXiv 2510.15602, Sec. 3.1):
// Algorithm 1 per window and component, the error-to-pixel association, the
// mean over components and the final Gaussian smoothing.
//
// For component k and window centre p (clipped (2r+1)^2 window, N_loc
// pixels, histogram P), Algorithm 1 transports P onto the reference R at the
// common mass N_loc N_ref (P'_i = P_i N_ref, R'_j = R_j N_loc) with two
// pointers; the mass-weighted distance charged to bin i, Enum_i, is an exact
// integer and E_i = Enum_i / P'_i.  A pixel q of bin b takes E_{k,p}[b] from
// every window p that contains it and averages (sigma_p = infinity: a box
// average over the window centres within r of q):
//     raw(q) = (1/d) sum_k (1/n(q)) sum_{|p-q|_inf <= r} E_{k,p}[b_k(q)]
// and score = Gaussian(sigma_s) * raw, renormalised at the border.
//
// k_assoc: one CTA = one component of one image x a strip of output columns,
// all rows.  Thread c owns window column c (the strip plus r on each side);
// it slides two window histograms down the image, packed in one u32 per bin
// (low half: the leading window, centre row y + r; high half: the trailing
// window, centre row y - r - 1, the same window 2r+1 rows later), and forms
// Algorithm 1's per-bin integers for both in one pass over the bins (a closed
// form of the walk from prefix-sum tables of the reference for B <= 64, the
// two-pointer walk itself above).  The leading window adds its per-bin errors to a
// running column sum V[b][c] (fixed point, 2^s), the trailing one subtracts
// the identical values, so V holds the sum over the 2r+1 window rows around
// the output row exactly.  Output pixel x then sums V[b(x)][c] over the 2r+1
// window columns around it.  The per-component sums go to the workspace;
// k_assoc_fin adds them over components (exact, u64) and divides once;
// k_blur smooths.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.cuh"

namespace qfca {
namespace {

constexpr int kMaxTaps = 33;  // 2 ceil(4 sigma_s) + 1 for sigma_s <= 4

struct AssocImgP {
    const uint8_t *bins;   // [d][H][pitch]
    int H, W, pitch, r;
    int sw, nstrip;        // output columns per strip, strips
    int shift;             // fixed-point scale 2^shift of the per-bin errors
    long cta0;             // first CTA of this image
    const uint32_t *ref;   // [d][B]
    uint32_t Nref;
    uint32_t *F;           // [d][H][W] per-component sums of fixed-point errors
};

struct AssocParams {
    int n, d, B, nt;       // nt: threads per CTA (window columns)
    int p8;                // histogram bytes: 1 = 8-bit counts, two columns per word (r <= 7)
    AssocImgP img[kMaxBatch];
};

// Where window column c's packed counts live: 32-bit words per bin row
// (stride), the word of column c (col), the shift of its 16-bit pair (sh), and
// within the pair the leading count's mask (lm) and the trailing count's shift
// (ts).  Layout 16: one word per column, leading | trailing << 16.  Layout 8:
// two columns per word, each pair leading | trailing << 8 (counts <= 255).
struct HistView {
    int stride, col, sh, ts;
    uint32_t lm;
    __device__ __forceinline__ HistView(int nt, int c, bool p8)
        : stride(p8 ? nt / 2 : nt), col(p8 ? c >> 1 : c), sh(p8 ? 16 * (c & 1) : 0), ts(p8 ? 8 : 16),
          lm(p8 ? 0xffu : 0xffffu) {}
};

struct FinImg {
    int H, W, r, shift;
    long blk0;
    const uint32_t *F;
    float *raw, *comp;
    const float *lo, *hi;  // value units: component ranges [d] (NULL: bin units)
};

struct AssocFinParams {
    int n, d, B;
    FinImg img[kMaxBatch];
};

constexpr int kAssocMaxWeights = 512;

struct BlurImg {
    int H, W;
    long blk0;
    const float *in;
    float *out;
};

struct BlurParams {
    int n, R4, copy;
    float w[kMaxTaps];
    BlurImg img[kMaxBatch];
};

// Threads (window columns) per CTA for B bins: the histogram and the running
// sums take (2B + 1) words per column.
inline int max_cols(int B) { return B <= 32 ? 256 : (B <= 128 ? 128 : 64); }

__host__ __device__ inline int ring_rows(int r) { return 4 * r + 4; }

// Closed-form per-bin errors (tables of B (B+1) prefix sums) up to this many bins;
// above it the two-pointer walk itself runs.
constexpr int kClosedMaxB = 64;

// Boundary tables of the border window sizes N = (2r+1) k, k = r+1 .. 2r (a
// column-border window has all 2r+1 rows and k columns, a row-border one the
// reverse), packed one after another; not kept when they would take more than
// kColTabMax bytes (those windows then search the reference bins).
constexpr size_t kColTabMax = 8192;
__host__ __device__ inline int coltab_off(int r, int cols) {
    const int span = 2 * r + 1;
    return span * ((cols - 1) * cols / 2 - r * (r + 1) / 2) + (cols - r - 1);
}
__host__ __device__ inline size_t coltab_bytes(int r) {
    const size_t b = (size_t)coltab_off(r, 2 * r + 1);
    return b <= kColTabMax ? (b + 15) & ~(size_t)15 : 0;
}

size_t assoc_smem(int nt, int B, int r, bool wide) {
    const int span = 2 * r + 1;
    const int rw = (nt + 2 * r + 15) & ~15;
    size_t tab = sizeof(uint32_t) * (B + 1);  // reference (walk) or its exclusive prefix (closed form)
    size_t coltab = 0;  // images of a launch have radii <= r: the largest of their column tables
    for (int rr = 1; rr <= r; rr++) coltab = std::max(coltab, coltab_bytes(rr));
    if (B <= kClosedMaxB)
        tab += align_up((wide ? 8 : 4) * (size_t)B * (2 * B + 1), 16) + align_up((size_t)span * span + 1, 16) + coltab;
    const size_t hist_words = (size_t)(B + 1) * (r <= 7 && B <= kClosedMaxB ? nt / 2 : nt);
    return sizeof(uint32_t) * (hist_words + (size_t)B * nt) + align_up(tab, 16) +
           sizeof(float) * (span * span + 1) + (size_t)ring_rows(r) * rw + 64;
}

// Fixed-point scale: a window-column sum over 2r+1 rows and the output sum over
// (2r+1)^2 windows of errors <= B-1 must stay below 2^32.
int assoc_shift(int B, int r) {
    const double span2 = (double)(2 * r + 1) * (2 * r + 1);
    int s = (int)std::floor(std::log2(4294967295.0 / (span2 * (B - 1))));
    return std::min(20, std::max(0, s));
}

template <typename ACC>
__device__ __forceinline__ void alg1_column(const uint32_t *hist, int nt, int c, int B, int half, uint32_t Nloc,
                                            uint32_t Nref, const uint32_t *ref, const float *recip, uint32_t *V,
                                            bool add) {
    // Algorithm 1 with P'_i = P_i N_ref and R'_j = R_j N_loc; the bin-i errors are
    // flushed into V when bin i is used up (or empty).
    int i = 0, j = 0;
    uint32_t cnt = (hist[(size_t)1 * nt + c] >> half) & 0xffffu;
    ACC pr = (ACC)cnt * Nref, rr = (ACC)ref[0] * Nloc, en = 0;
    while (i < B && j < B) {
        const ACC m = pr < rr ? pr : rr;
        en += m * (ACC)(i > j ? i - j : j - i);
        pr -= m;
        rr -= m;
        if (pr == 0) {
            if (cnt) {
                float e;
                if (sizeof(ACC) == 4) e = __uint2float_rn((uint32_t)en) * recip[cnt];
                else e = __ull2float_rn((unsigned long long)en) * recip[cnt];
                const uint32_t fx = __float2uint_rn(e);
                uint32_t *v = V + (size_t)i * nt + c;
                *v = add ? *v + fx : *v - fx;
            }
            en = 0;
            if (++i < B) {
                cnt = (hist[(size_t)(i + 1) * nt + c] >> half) & 0xffffu;
                pr = (ACC)cnt * Nref;
            }
        } else {
            if (++j < B) rr = (ACC)ref[j] * Nloc;
        }
    }
}

// J(t) = max{x in [0, B-1] : N_loc cumRx[x] <= t}: the reference bin at
// position t of the common mass axis (any bin whose closed interval holds t
// serves, the transport integral being continuous).
template <typename ACC>
__device__ __forceinline__ int ref_bin_at(const uint32_t *cumRx, int B, uint32_t Nloc, ACC t) {
    int lo = 0, hi = B - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((ACC)Nloc * cumRx[mid] <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Algorithm 1's per-bin integers in closed form.  The mass of window bin i
// occupies [a, b) = [N_ref cumP_{i-1}, N_ref cumP_i) of the common mass axis;
// the walk moves each unit at t to reference bin J(t), so
//   Enum_i = F_i(b) - F_i(a),  F_i(t) = int_0^t |i - J(s)| ds
//          = N_loc T[i][J] + |i - J| (t - N_loc cumRx[J]),  J = J(t),
// with T[i][x] = sum_{j<x} |i - j| R_j and cumRx[x] = sum_{j<x} R_j: the same
// integers as the two-pointer walk.  Each boundary's J comes from Jtab (J at
// N_ref m for the interior window size) or a binary search; consecutive bins
// share a boundary.
// One window's running state in the closed form: cumulative count so far, the
// reference bin J(a) at the current boundary a = N_ref cumP, the window size
// and its boundary table (NULL: binary search).
template <typename ACC>
struct Walk {
    uint32_t cumP, Nloc;
    int Ja;
    ACC a;
    const uint8_t *Jtab;  // J at N_ref m for this window's size, or NULL (search)
    bool full;            // full-size window: the folded table U applies
};

// Fixed-point error of window bin i (count cnt): E_i = (F_i(b) - F_i(a)) /
// (cnt N_ref) with the closed form above.  For the full window size the two
// terms of F_i fold into one table, F_i(t) = U[i][J] + |i - J| t with
// U[i][J] = N T[i][J] - |i - J| N cumRx[J] (N = (2r+1)^2; taken modulo the
// word size: the difference is exact and non-negative).
template <typename ACC>
__device__ __forceinline__ uint32_t bin_error(Walk<ACC> &w, int i, uint32_t cnt, int B, uint32_t Nref,
                                              const uint32_t *cumRx, const ACC *Trow, const ACC *Urow,
                                              const float *recip) {
    w.cumP += cnt;
    const ACC b = (ACC)Nref * w.cumP;
    const int Ja = w.Ja;
    const int Jb = w.Jtab ? (int)w.Jtab[w.cumP] : ref_bin_at<ACC>(cumRx, B, w.Nloc, b);
    ACC en;
    if (w.full) {
        en = (Urow[Jb] + (ACC)(i > Jb ? i - Jb : Jb - i) * b) - (Urow[Ja] + (ACC)(i > Ja ? i - Ja : Ja - i) * w.a);
    } else {
        const ACC Fa = (ACC)w.Nloc * Trow[Ja] + (ACC)(i > Ja ? i - Ja : Ja - i) * (w.a - (ACC)w.Nloc * cumRx[Ja]);
        const ACC Fb = (ACC)w.Nloc * Trow[Jb] + (ACC)(i > Jb ? i - Jb : Jb - i) * (b - (ACC)w.Nloc * cumRx[Jb]);
        en = Fb - Fa;
    }
    w.Ja = Jb;
    w.a = b;
    float e;
    if (sizeof(ACC) == 4) e = __uint2float_rn((uint32_t)en) * recip[cnt];
    else e = __ull2float_rn((unsigned long long)en) * recip[cnt];
    return __float2uint_rn(e);
}

// Both windows of a window column in one pass over the bins (one load of the
// packed counts per bin): V[i] += E_lead,i - E_trail,i.
template <typename ACC>
__device__ __forceinline__ void alg1_pair(const uint32_t *hist, int nt, int c, bool p8, int B, bool lead_on, bool trail_on,
                                          uint32_t Nl, uint32_t Nt, uint32_t Nint, uint32_t Nref,
                                          const uint32_t *cumRx, const ACC *T, const ACC *U, const uint8_t *JtL,
                                          const uint8_t *JtT, const float *recip, uint32_t *V) {
    Walk<ACC> wl{0u, Nl, 0, (ACC)0, JtL, Nl == Nint};
    Walk<ACC> wt{0u, Nt, 0, (ACC)0, JtT, Nt == Nint};
    const uint32_t ml = lead_on ? 0xffffu : 0u, mt = trail_on ? 0xffffu : 0u;
    const HistView hv(nt, c, p8);
    const uint32_t *h = hist + hv.stride + hv.col;
    uint32_t *v = V + c;
    for (int i = 0; i < B; i++, h += hv.stride, v += nt) {
        const uint32_t word = *h >> hv.sh;
        const uint32_t cl = word & hv.lm & ml, ct = (word >> hv.ts) & hv.lm & mt;
        if (!(cl | ct)) continue;
        const ACC *Trow = T + (size_t)i * (B + 1);
        const ACC *Urow = U + (size_t)i * B;
        uint32_t delta = 0;
        if (cl) delta += bin_error<ACC>(wl, i, cl, B, Nref, cumRx, Trow, Urow, recip);
        if (ct) delta -= bin_error<ACC>(wt, i, ct, B, Nref, cumRx, Trow, Urow, recip);
        *v += delta;
    }
}

// The same pass when every window of the warp that is on is full-size: no
// branch per bin (an empty bin gives en = 0 and recip[0] = 0), so the bins'
// table lookups pipeline; J at each boundary comes from Jtab and F from U.
template <typename ACC>
__device__ __forceinline__ void alg1_pair_full(const uint32_t *hist, int nt, int c, bool p8, int B, bool lead_on,
                                               bool trail_on, uint32_t Nref, const ACC *U, const uint8_t *Jtab,
                                               const float *recip, uint32_t *V) {
    const uint32_t ml = lead_on ? 0xffffu : 0u, mt = trail_on ? 0xffffu : 0u;
    uint32_t cl_sum = 0, ct_sum = 0;
    int JaL = 0, JaT = 0;
    ACC aL = 0, aT = 0;
    const HistView hv(nt, c, p8);
    const uint32_t *h = hist + hv.stride + hv.col;
    uint32_t *v = V + c;
    const ACC *Urow = U;
#pragma unroll 4
    for (int i = 0; i < B; i++, h += hv.stride, v += nt, Urow += B) {
        const uint32_t word = *h >> hv.sh;
        const uint32_t cl = word & hv.lm & ml, ct = (word >> hv.ts) & hv.lm & mt;
        cl_sum += cl;
        ct_sum += ct;
        const ACC bL = (ACC)Nref * cl_sum, bT = (ACC)Nref * ct_sum;
        const int JbL = Jtab[cl_sum], JbT = Jtab[ct_sum];
        const ACC enL = (Urow[JbL] + (ACC)(i > JbL ? i - JbL : JbL - i) * bL) -
                        (Urow[JaL] + (ACC)(i > JaL ? i - JaL : JaL - i) * aL);
        const ACC enT = (Urow[JbT] + (ACC)(i > JbT ? i - JbT : JbT - i) * bT) -
                        (Urow[JaT] + (ACC)(i > JaT ? i - JaT : JaT - i) * aT);
        float eL, eT;
        if (sizeof(ACC) == 4) {
            eL = __uint2float_rn((uint32_t)enL) * recip[cl];
            eT = __uint2float_rn((uint32_t)enT) * recip[ct];
        } else {
            eL = __ull2float_rn((unsigned long long)enL) * recip[cl];
            eT = __ull2float_rn((unsigned long long)enT) * recip[ct];
        }
        const uint32_t delta = __float2uint_rn(eL) - __float2uint_rn(eT);
        if (delta) *v += delta;
        JaL = JbL;
        JaT = JbT;
        aL = bL;
        aT = bT;
    }
}

// The branch-free pass for warps whose windows all have a boundary table but are
// not all full-size (the column borders): F from T and cumRx for each window's
// own size N.  A window that is off passes N = 0 and any table (F stays 0).
template <typename ACC>
__device__ __forceinline__ void alg1_pair_tform(const uint32_t *hist, int nt, int c, bool p8, int B, bool lead_on,
                                                bool trail_on, uint32_t NL, uint32_t NT, const uint8_t *JtL,
                                                const uint8_t *JtT, uint32_t Nref, const uint32_t *cumRx,
                                                const ACC *T, const float *recip, uint32_t *V) {
    const uint32_t ml = lead_on ? 0xffffu : 0u, mt = trail_on ? 0xffffu : 0u;
    uint32_t cl_sum = 0, ct_sum = 0;
    int JaL = 0, JaT = 0;
    ACC aL = 0, aT = 0;
    const HistView hv(nt, c, p8);
    const uint32_t *h = hist + hv.stride + hv.col;
    uint32_t *v = V + c;
    const ACC *Trow = T;
    auto F = [&](int i, int J, ACC t, uint32_t N) -> ACC {
        return (ACC)N * Trow[J] + (ACC)(i > J ? i - J : J - i) * (t - (ACC)N * cumRx[J]);
    };
#pragma unroll 4
    for (int i = 0; i < B; i++, h += hv.stride, v += nt, Trow += B + 1) {
        const uint32_t word = *h >> hv.sh;
        const uint32_t cl = word & hv.lm & ml, ct = (word >> hv.ts) & hv.lm & mt;
        cl_sum += cl;
        ct_sum += ct;
        const ACC bL = (ACC)Nref * cl_sum, bT = (ACC)Nref * ct_sum;
        const int JbL = JtL[cl_sum], JbT = JtT[ct_sum];
        const ACC enL = F(i, JbL, bL, NL) - F(i, JaL, aL, NL);
        const ACC enT = F(i, JbT, bT, NT) - F(i, JaT, aT, NT);
        float eL, eT;
        if (sizeof(ACC) == 4) {
            eL = __uint2float_rn((uint32_t)enL) * recip[cl];
            eT = __uint2float_rn((uint32_t)enT) * recip[ct];
        } else {
            eL = __ull2float_rn((unsigned long long)enL) * recip[cl];
            eT = __ull2float_rn((unsigned long long)enT) * recip[ct];
        }
        const uint32_t delta = __float2uint_rn(eL) - __float2uint_rn(eT);
        if (delta) *v += delta;
        JaL = JbL;
        JaT = JbT;
        aL = bL;
        aT = bT;
    }
}

template <typename ACC, bool CLOSED>
__global__ void __launch_bounds__(256) k_assoc(const __grid_constant__ AssocParams p) {
    const int B = p.B, nt = p.nt;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const long cta = blockIdx.x;
    const int ii = table_image(p.n, cta, [&](int i) { return p.img[i].cta0; });
    const AssocImgP &im = p.img[ii];
    const int H = im.H, W = im.W, r = im.r, span = 2 * r + 1;
    long local = cta - im.cta0;
    const int strip = (int)(local % im.nstrip), k = (int)(local / im.nstrip);
    const int x0 = strip * im.sw;           // first output column
    const int c0 = x0 - r;                  // image column of window column 0
    const int px0 = x0 - 2 * r;             // image column of ring column 0
    const int rw = (nt + 2 * r + 15) & ~15; // ring row width
    const int RR = ring_rows(r);

    const bool p8 = CLOSED && p.p8;
    const int hstride = p8 ? nt / 2 : nt;
    uint32_t *hist = reinterpret_cast<uint32_t *>(smem_raw);  // [B+1][hstride], row 0: outside pixels (layout 16)
    uint32_t *V = hist + (size_t)(B + 1) * hstride;            // [B][nt]
    uint32_t *ref = V + (size_t)B * nt;                        // [B+1]: R_j (walk) or cumRx[x] (closed form)
    unsigned char *tp = reinterpret_cast<unsigned char *>(ref + B + 1);
    ACC *T = nullptr, *U = nullptr;
    uint8_t *Jtab = nullptr, *JC = nullptr;
    if (CLOSED) {
        tp = reinterpret_cast<unsigned char *>(((uintptr_t)tp + 15) & ~(uintptr_t)15);
        T = reinterpret_cast<ACC *>(tp);                       // [B][B+1]
        U = T + (size_t)B * (B + 1);                           // [B][B]
        Jtab = reinterpret_cast<uint8_t *>(U + (size_t)B * B);  // [span^2 + 1]
        JC = Jtab + ((span * span + 1 + 15) & ~15);             // column-border tables (coltab_bytes(r))
        tp = JC + coltab_bytes(r);
    }
    float *recip = reinterpret_cast<float *>(((uintptr_t)tp + 15) & ~(uintptr_t)15);  // [span^2 + 1]: 2^s / (n N_ref)
    uint8_t *ring = reinterpret_cast<uint8_t *>(recip + span * span + 1);  // [RR][rw]: bin+1, 0 outside

    const int t = threadIdx.x;
    const uint8_t *plane = im.bins + (size_t)k * H * im.pitch;
    const uint32_t Nref = im.Nref;
    const uint32_t *Rk = im.ref + (size_t)k * B;
    for (int e = t; e < (B + 1) * hstride + B * nt; e += nt) hist[e] = 0;  // hist and V
    if (CLOSED) {
        if (t == 0) {
            uint32_t acc = 0;
            for (int x = 0; x <= B; x++) {
                ref[x] = acc;
                if (x < B) acc += Rk[x];
            }
        }
        for (int i = t; i < B; i += nt) {
            ACC acc = 0;
            for (int x = 0; x <= B; x++) {
                T[i * (B + 1) + x] = acc;
                if (x < B) acc += (ACC)(i > x ? i - x : x - i) * Rk[x];
            }
        }
        __syncthreads();
        const uint32_t Nint = (uint32_t)(span * span);
        for (int m = t; m <= span * span; m += nt) Jtab[m] = (uint8_t)ref_bin_at<ACC>(ref, B, Nint, (ACC)Nref * (uint32_t)m);
        for (int e = t; e < B * B; e += nt) {
            const int i = e / B, J = e % B;
            U[e] = (ACC)Nint * T[i * (B + 1) + J] - (ACC)(i > J ? i - J : J - i) * ((ACC)Nint * ref[J]);
        }
        if (coltab_bytes(r)) {
            const int ncol_tab = coltab_off(r, 2 * r + 1);
            for (int e = t; e < ncol_tab; e += nt) {
                int cols = r + 1;
                while (coltab_off(r, cols + 1) <= e) cols++;
                const int m = e - coltab_off(r, cols);
                JC[e] = (uint8_t)ref_bin_at<ACC>(ref, B, (uint32_t)(span * cols), (ACC)Nref * (uint32_t)m);
            }
        }
    } else {
        for (int b = t; b < B; b += nt) ref[b] = Rk[b];
    }
    const float scale = ldexpf(1.0f, im.shift);
    for (int n = t; n <= span * span; n += nt) recip[n] = n ? scale / ((float)n * (float)Nref) : 0.0f;
    auto load_row = [&](int yy) {
        uint8_t *dst = ring + (size_t)(((yy % RR) + RR) % RR) * rw;
        for (int col = t; col < rw; col += nt) {
            const int x = px0 + col;
            uint8_t v = 0;
            if (yy >= 0 && yy < H && x >= 0 && x < W) v = (uint8_t)(min((int)plane[(size_t)yy * im.pitch + x], B - 1) + 1);
            dst[col] = v;
        }
    };
    // rows needed by the first step: y0 - 2r - 2 .. y0 + 2r with y0 = -2r
    const int ys = -2 * r;
    for (int yy = ys - 2 * r - 2; yy <= ys + 2 * r; yy++) load_row(yy);
    __syncthreads();

    const int c = c0 + t;                   // this thread's window column (image coordinates)
    const bool col_ok = c >= 0 && c < W;
    const int wx0 = max(0, c - r), wx1 = min(W - 1, c + r);
    const uint32_t wcols = col_ok ? (uint32_t)(wx1 - wx0 + 1) : 0u;
    const int sw_here = min(im.sw, W - x0);
    uint32_t *Fk = im.F + (size_t)k * H * W;

    for (int y = ys; y < H; y++) {
        // ---- the bins of row y+2r+1 (needed next step) are fetched now and stored
        // after the window work, so their latency hides behind it
        const int yn = y + 1 + 2 * r;
        uint8_t pf[3];
#pragma unroll
        for (int q = 0; q < 3; q++) {
            const int col = t + q * nt, x = px0 + col;
            pf[q] = 0;
            if (col < rw && yn < H && x >= 0 && x < W) pf[q] = (uint8_t)(min((int)plane[(size_t)yn * im.pitch + x], B - 1) + 1);
        }
        // ---- slide the two histograms: row y+2r enters the leading window,
        // row y-1 leaves it and enters the trailing one, row y-2r-2 leaves the trailing one
        {
            const uint8_t *ra = ring + (size_t)((((y + 2 * r) % RR) + RR) % RR) * rw + t;
            const uint8_t *rb = ring + (size_t)((((y - 1) % RR) + RR) % RR) * rw + t;
            const uint8_t *rc = ring + (size_t)((((y - 2 * r - 2) % RR) + RR) % RR) * rw + t;
            if (p8) {
                // 8-bit counts: outside pixels are not counted (no carry can reach the
                // neighbouring column); (2r+2)(2r+1) <= 240 keeps every count below 256
                uint32_t *hc = hist + (t >> 1);
                const int sh = 16 * (t & 1);
#pragma unroll 4
                for (int u = 0; u < span; u++) {
                    if (ra[u]) atomicAdd(&hc[(size_t)ra[u] * hstride], 1u << sh);
                    if (rb[u]) atomicAdd(&hc[(size_t)rb[u] * hstride], 0xffu << sh);  // leading -1, trailing +1
                    if (rc[u]) atomicAdd(&hc[(size_t)rc[u] * hstride], 0xffffff00u << sh);  // trailing -1
                }
            } else {
#pragma unroll 4
                for (int u = 0; u < span; u++) {
                    atomicAdd(&hist[(size_t)ra[u] * nt + t], 1u);
                    atomicAdd(&hist[(size_t)rb[u] * nt + t], 0xffffu);  // -1 low half, +1 high half
                    atomicAdd(&hist[(size_t)rc[u] * nt + t], 0xffff0000u);  // -1 high half
                }
            }
        }
        // ---- Algorithm 1 on the leading window (centre y+r) and the trailing one (centre y-r-1)
        if (CLOSED) {
            const int a = y + r, bq = y - r - 1;
            const bool lead_on = col_ok && a >= 0 && a < H, trail_on = col_ok && bq >= 0;
            const uint32_t Nint = (uint32_t)(span * span);
            const uint32_t Nl = lead_on ? (uint32_t)(min(H - 1, a + r) - max(0, a - r) + 1) * wcols : 0u;
            const uint32_t Ntr = trail_on ? (uint32_t)(min(H - 1, bq + r) - max(0, bq - r) + 1) * wcols : 0u;
            const bool full = (!lead_on || Nl == Nint) && (!trail_on || Ntr == Nint);
            // boundary table of each window: full size, or (2r+1) x k with r < k < 2r+1 -- a
            // column-border window (all rows) or a row-border one (all columns): the table
            // depends only on N = (2r+1) k -- or none (the corners search)
            auto table = [&](uint32_t N, int rows) -> const uint8_t * {
                if (N == Nint) return Jtab;
                const int cols = (int)wcols;
                if (!coltab_bytes(r)) return nullptr;
                if (rows == span && cols > r && cols < span) return JC + coltab_off(r, cols);
                if (cols == span && rows > r && rows < span) return JC + coltab_off(r, rows);
                return nullptr;
            };
            const int rows_l = lead_on ? min(H - 1, a + r) - max(0, a - r) + 1 : 0;
            const int rows_t = trail_on ? min(H - 1, bq + r) - max(0, bq - r) + 1 : 0;
            const uint8_t *jl = lead_on ? table(Nl, rows_l) : Jtab;
            const uint8_t *jt = trail_on ? table(Ntr, rows_t) : Jtab;
            const bool warp_full = __all_sync(0xffffffffu, full);
            const bool warp_tab = __all_sync(0xffffffffu, jl != nullptr && jt != nullptr);
            if (lead_on || trail_on) {
                if (warp_full)
                    alg1_pair_full<ACC>(hist, nt, t, p8, B, lead_on, trail_on, Nref, U, Jtab, recip, V);
                else if (warp_tab)
                    alg1_pair_tform<ACC>(hist, nt, t, p8, B, lead_on, trail_on, Nl, Ntr, jl, jt, Nref, ref, T, recip, V);
                else
                    alg1_pair<ACC>(hist, nt, t, p8, B, lead_on, trail_on, Nl, Ntr, Nint, Nref, ref, T, U, jl, jt, recip, V);
            }
        } else if (col_ok) {
            const int a = y + r, bq = y - r - 1;
            if (a >= 0 && a < H) {
                const uint32_t Nloc = (uint32_t)(min(H - 1, a + r) - max(0, a - r) + 1) * wcols;
                alg1_column<ACC>(hist, nt, t, B, 0, Nloc, Nref, ref, recip, V, true);
            }
            if (bq >= 0) {
                const uint32_t Nloc = (uint32_t)(min(H - 1, bq + r) - max(0, bq - r) + 1) * wcols;
                alg1_column<ACC>(hist, nt, t, B, 16, Nloc, Nref, ref, recip, V, false);
            }
        }
        {
            uint8_t *dst = ring + (size_t)(yn % RR) * rw;  // the slot of row y-2r-3, read by no one this step
#pragma unroll
            for (int q = 0; q < 3; q++)
                if (t + q * nt < rw) dst[t + q * nt] = pf[q];
        }
        __syncthreads();
        // ---- output row y: each pixel sums its own bin over the 2r+1 window columns around it
        if (y >= 0 && t < sw_here) {
            const int x = x0 + t;
            const int b = (int)ring[(size_t)(y % RR) * rw + (x - px0)] - 1;
            const uint32_t *vb = V + (size_t)b * nt + t;  // window columns x-r .. x+r are t .. t+2r
            uint32_t s = 0;
            for (int u = 0; u < span; u++) s += vb[u];
            Fk[(size_t)y * W + x] = s;
        }
        __syncthreads();
    }
}

// raw(q) = sum_k F_k(q) / (d n(q) 2^s); comp_k(q) = F_k(q) / (n(q) 2^s) when asked.
// Value units: F_k weighs w_k = (hi_k - lo_k) / B (the bin width: Algorithm 1's
// cost is the distance of the quantized values), summed in FP64 over k in order.
__global__ void __launch_bounds__(256) k_assoc_fin(const __grid_constant__ AssocFinParams p) {
    __shared__ double wk[kAssocMaxWeights];
    const long blk = blockIdx.x;
    const int ii = table_image(p.n, blk, [&](int i) { return p.img[i].blk0; });
    const FinImg &im = p.img[ii];
    if (im.lo) {
        for (int k = threadIdx.x; k < p.d; k += 256) wk[k] = ((double)im.hi[k] - (double)im.lo[k]) / (double)p.B;
        __syncthreads();
    }
    const long HW = (long)im.H * im.W;
    const long q = (blk - im.blk0) * 256 + threadIdx.x;
    if (q >= HW) return;
    const int y = (int)(q / im.W), x = (int)(q % im.W);
    const int r = im.r;
    const double n = (double)(min(im.H - 1, y + r) - max(0, y - r) + 1) * (double)(min(im.W - 1, x + r) - max(0, x - r) + 1);
    const double unit = n * ldexp(1.0, im.shift);
    if (im.lo) {
        double sv = 0.0;
        for (int k = 0; k < p.d; k++) {
            const double f = wk[k] * (double)im.F[(size_t)k * HW + q];
            sv += f;
            if (im.comp) im.comp[(size_t)k * HW + q] = (float)(f / unit);
        }
        im.raw[q] = (float)(sv / (unit * p.d));
        return;
    }
    unsigned long long s = 0;
    for (int k = 0; k < p.d; k++) {
        const uint32_t f = im.F[(size_t)k * HW + q];
        s += f;
        if (im.comp) im.comp[(size_t)k * HW + q] = (float)((double)f / unit);
    }
    im.raw[q] = (float)((double)s / (unit * p.d));
}

// Separable Gaussian on a 32 x 32 tile with a halo of R4, weights renormalised
// over the taps inside the image.
__global__ void __launch_bounds__(256) k_blur(const __grid_constant__ BlurParams p) {
    __shared__ float tile[32 + 2 * 16][32 + 2 * 16 + 1];
    __shared__ float mid[32 + 2 * 16][33];
    const long blk = blockIdx.x;
    const int ii = table_image(p.n, blk, [&](int i) { return p.img[i].blk0; });
    const BlurImg &im = p.img[ii];
    const int H = im.H, W = im.W, R4 = p.R4;
    const int nbx = (W + 31) / 32;
    const long local = blk - im.blk0;
    const int tx0 = (int)(local % nbx) * 32, ty0 = (int)(local / nbx) * 32;
    const int TW = 32 + 2 * R4;
    for (int e = threadIdx.x; e < TW * TW; e += 256) {
        const int yy = e / TW, xx = e % TW;
        const int gy = ty0 - R4 + yy, gx = tx0 - R4 + xx;
        tile[yy][xx] = (gy >= 0 && gy < H && gx >= 0 && gx < W) ? im.in[(size_t)gy * W + gx] : 0.0f;
    }
    __syncthreads();
    if (p.copy) {
        for (int e = threadIdx.x; e < 32 * 32; e += 256) {
            const int gy = ty0 + e / 32, gx = tx0 + e % 32;
            if (gy < H && gx < W) im.out[(size_t)gy * W + gx] = tile[e / 32 + R4][e % 32 + R4];
        }
        return;
    }
    // horizontal pass over all tile rows (the halo rows too)
    for (int e = threadIdx.x; e < TW * 32; e += 256) {
        const int yy = e / 32, xo = e % 32;
        const int gx = tx0 + xo;
        float s = 0.0f, w = 0.0f;
        for (int u = -R4; u <= R4; u++) {
            if (gx + u < 0 || gx + u >= W) continue;
            s = fmaf(p.w[u + R4], tile[yy][xo + R4 + u], s);
            w += p.w[u + R4];
        }
        mid[yy][xo] = s / w;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < 32 * 32; e += 256) {
        const int yo = e / 32, xo = e % 32;
        const int gy = ty0 + yo, gx = tx0 + xo;
        if (gy >= H || gx >= W) continue;
        float s = 0.0f, w = 0.0f;
        for (int u = -R4; u <= R4; u++) {
            if (gy + u < 0 || gy + u >= H) continue;
            s = fmaf(p.w[u + R4], mid[yo + R4 + u][xo], s);
            w += p.w[u + R4];
        }
        im.out[(size_t)gy * W + gx] = s / w;
    }
}

DeviceOnce g_attrs_assoc;

}  // namespace

bool assoc_shape_ok(int B, int r) {
    const int nt = max_cols(B);
    if (nt - 2 * r < 8) return false;
    return assoc_smem(nt, B, r, true) <= 200 * 1024;
}

size_t assoc_jobs_workspace_bytes(const AssocJob *jobs, int n, int d) {
    size_t b = 0;
    for (int i = 0; i < n; i++) {
        const size_t HW = (size_t)jobs[i].H * jobs[i].W;
        b += align_up(sizeof(uint32_t) * HW * d, 256);
        if (jobs[i].sigma_s > 0.0f || !jobs[i].raw) b += align_up(sizeof(float) * HW, 256);
    }
    return b;
}

cudaError_t launch_assoc_jobs(const AssocJob *jobs, int n, int d, int B, void *ws, cudaStream_t st) {
    int dev = 0;
    cudaGetDevice(&dev);
    int rmax = 0;
    bool wide = false;
    for (int i = 0; i < n; i++) {
        rmax = std::max(rmax, jobs[i].r);
        const double span2 = (double)(2 * jobs[i].r + 1) * (2 * jobs[i].r + 1);
        if ((double)(B - 1) * span2 * jobs[i].Nref >= 4294967296.0) wide = true;
        if (!(jobs[i].sigma_s <= 4.0f)) return cudaErrorInvalidValue;
    }
    if (!assoc_shape_ok(B, rmax)) return cudaErrorNotSupported;
    const int ntmax = max_cols(B);
    // threads per CTA: the widest strip any image needs, rounded to warps
    int nt = 32;
    std::vector<int> sw(n), ns(n);
    for (int i = 0; i < n; i++) {
        const int r = jobs[i].r, W = jobs[i].W;
        const int cap = ntmax - 2 * r;
        ns[i] = (W + cap - 1) / cap;
        sw[i] = (W + ns[i] - 1) / ns[i];
        nt = std::max(nt, (sw[i] + 2 * r + 31) & ~31);
    }
    nt = std::min(nt, ntmax);
    const size_t smem = assoc_smem(nt, B, rmax, wide);
    const bool closed = B <= kClosedMaxB;
    cudaError_t ea = device_once(g_attrs_assoc, dev, [] {
        const int lim = 200 * 1024;
        cudaError_t r = cudaFuncSetAttribute(k_assoc<uint32_t, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        if (r == cudaSuccess)
            r = cudaFuncSetAttribute(k_assoc<unsigned long long, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        if (r == cudaSuccess)
            r = cudaFuncSetAttribute(k_assoc<uint32_t, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        if (r == cudaSuccess)
            r = cudaFuncSetAttribute(k_assoc<unsigned long long, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        return r;
    });
    if (ea != cudaSuccess) return ea;
    // workspace carve: F per image, then the unblurred map where the caller gave none (or a blur follows)
    std::vector<uint32_t *> F(n);
    std::vector<float *> rawp(n);
    unsigned char *w = static_cast<unsigned char *>(ws);
    for (int i = 0; i < n; i++) {
        const size_t HW = (size_t)jobs[i].H * jobs[i].W;
        F[i] = reinterpret_cast<uint32_t *>(w);
        w += align_up(sizeof(uint32_t) * HW * d, 256);
    }
    for (int i = 0; i < n; i++) {
        const size_t HW = (size_t)jobs[i].H * jobs[i].W;
        if (jobs[i].sigma_s > 0.0f || !jobs[i].raw) {
            rawp[i] = reinterpret_cast<float *>(w);
            w += align_up(sizeof(float) * HW, 256);
        } else {
            rawp[i] = jobs[i].raw;
        }
    }
    for (int i0 = 0; i0 < n; i0 += kMaxBatch) {
        const int m = std::min(kMaxBatch, n - i0);
        AssocParams ap{};
        ap.n = m;
        ap.d = d;
        ap.B = B;
        ap.nt = nt;
        ap.p8 = (closed && rmax <= 7) ? 1 : 0;
        long ctas = 0;
        for (int i = 0; i < m; i++) {
            const AssocJob &j = jobs[i0 + i];
            AssocImgP &q = ap.img[i];
            q.bins = j.bins;
            q.H = j.H;
            q.W = j.W;
            q.pitch = j.pitch;
            q.r = j.r;
            q.sw = sw[i0 + i];
            q.nstrip = ns[i0 + i];
            q.shift = assoc_shift(B, j.r);
            q.cta0 = ctas;
            q.ref = j.ref;
            q.Nref = j.Nref;
            q.F = F[i0 + i];
            ctas += (long)q.nstrip * d;
        }
        if (wide && closed) QFCA_LAUNCH("k_assoc", st, (k_assoc<unsigned long long, true><<<(unsigned)ctas, nt, smem, st>>>(ap)));
        else if (closed) QFCA_LAUNCH("k_assoc", st, (k_assoc<uint32_t, true><<<(unsigned)ctas, nt, smem, st>>>(ap)));
        else if (wide) QFCA_LAUNCH("k_assoc", st, (k_assoc<unsigned long long, false><<<(unsigned)ctas, nt, smem, st>>>(ap)));
        else QFCA_LAUNCH("k_assoc", st, (k_assoc<uint32_t, false><<<(unsigned)ctas, nt, smem, st>>>(ap)));
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;

        AssocFinParams fp{};
        fp.n = m;
        fp.d = d;
        fp.B = B;
        long blks = 0;
        for (int i = 0; i < m; i++) {
            const AssocJob &j = jobs[i0 + i];
            FinImg &q = fp.img[i];
            q.H = j.H;
            q.W = j.W;
            q.r = j.r;
            q.shift = ap.img[i].shift;
            q.blk0 = blks;
            q.F = F[i0 + i];
            q.raw = rawp[i0 + i];
            q.comp = j.comp;
            q.lo = j.lo;
            q.hi = j.hi;
            blks += ((long)j.H * j.W + 255) / 256;
        }
        QFCA_LAUNCH("k_assoc_fin", st, (k_assoc_fin<<<(unsigned)blks, 256, 0, st>>>(fp)));
        if ((e = cudaGetLastError()) != cudaSuccess) return e;

        // smoothing (or a copy into the caller's raw map / the score); images of one launch share sigma_s
        for (int i = 0; i < m;) {
            const float sg = jobs[i0 + i].sigma_s;
            int i1 = i + 1;
            while (i1 < m && jobs[i0 + i1].sigma_s == sg) i1++;
            BlurParams bp{};
            bp.n = i1 - i;
            bp.copy = sg > 0.0f ? 0 : 1;
            bp.R4 = sg > 0.0f ? (int)std::ceil(4.0 * sg) : 0;
            for (int u = -bp.R4; u <= bp.R4; u++) bp.w[u + bp.R4] = (float)std::exp(-(double)u * u / (2.0 * sg * sg));
            long bb = 0;
            for (int q = i; q < i1; q++) {
                const AssocJob &j = jobs[i0 + q];
                BlurImg &b = bp.img[q - i];
                b.H = j.H;
                b.W = j.W;
                b.blk0 = bb;
                b.in = rawp[i0 + q];
                b.out = j.score;
                bb += (long)((j.W + 31) / 32) * ((j.H + 31) / 32);
            }
            QFCA_LAUNCH("k_blur", st, (k_blur<<<(unsigned)bb, 256, 0, st>>>(bp)));
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            if (sg > 0.0f)
                for (int q = i; q < i1; q++)
                    if (jobs[i0 + q].raw)
                        if ((e = cudaMemcpyAsync(jobs[i0 + q].raw, rawp[i0 + q],
                                                 sizeof(float) * jobs[i0 + q].H * jobs[i0 + q].W,
                                                 cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
                            return e;
            i = i1;
        }
    }
    return cudaSuccess;
}

}  // namespace qfca
