// eig32.cu -- top-d eigenpairs of a symmetric n x n covariance (the
// eigendecomposition of the single-image PCA fit, arXiv 2510.15602, Sec. 3.3)
// to FP64-level accuracy from FP32 work plus one Newton correction whose
// residuals are formed in float-float; one CTA per matrix, nothing but CTA
// barriers (n <= 256, d <= 32).
//
//   1. Householder tridiagonalisation A = Q T Q^T in FP32 on the lower
//      triangle packed by columns in shared memory (column j contiguous).  One
//      pass over the trailing block per step, warp per column: the rank-2
//      update of reflector k and, on the updated entries, the symmetric product
//      with reflector k+1 (formed first, in place, from column k+1, updated
//      alone); each lane keeps the next reflector and the row sums of its rows
//      in registers, and the row and column partial sums are added in a fixed
//      order.  Three CTA barriers per step.  Reflector k stays in column k
//      (contiguous) for the later passes.
//   2. The top d eigenvalues sigma_j of T by warp multisection on the FP32
//      Sturm count; eigenvectors z_j of T by two steps of inverse iteration
//      (Gaussian elimination with partial pivoting, one lane per eigenvector);
//      back-transformation x_j = Q z_j (warp per column).
//   3. Newton correction per column (x, sigma approximate; A x = lambda x):
//      r = A x - sigma x with A in float-float (exact FP32 products, compensated
//      sums), u = Q^T r, u -= (z.u) z, solve (T - sigma I) y = u (the same
//      pivoted elimination), y -= (z.y) z, x' = x - Q y carried as an unevaluated
//      pair.  One step squares the FP32 start's error: about 1e-12 of lambda_1/gap.
//   4. A x' = A x - A (Q y): A x in float-float from the residual, A (Q y) in
//      FP32 (the correction is small, so its rounding is far below the
//      tolerance); lambda_j = x'^T A x' / x'^T x' (float-float), the residual
//      |A x' - lambda x'| / |x'| of every column; a matrix whose residual
//      exceeds tol * |lambda_max| is flagged for the float-float solver (eig.cu)
//      instead.  Normalisation, sign (largest-magnitude entry positive, first on
//      ties), descending order, FP64 output.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "ff.cuh"
#include "internal.cuh"

namespace qfca {
namespace {

using ffa::ff;
constexpr int kT = 1024;
constexpr int kNW = kT / 32;
template <bool B>
struct BoolC {
    static constexpr bool value = B;
};
constexpr BoolC<true> kTrue{};
constexpr BoolC<false> kFalse{};
constexpr int kQ = 8;    // rows per lane in a tridiagonalisation pass (n <= 256)
constexpr int kXS = 33;  // row stride of the n x d panels (conflict-free by rows and by columns)

struct Eig32Args {
    const float2 *cov;  // [mats][n][n] float-float (hi, lo) covariance, full symmetric storage
    int n, d;
    float *scr;         // [mats][3][n][32] U factor of the pivoted elimination (one column per lane)
    float *Z;           // [mats][n][32] eigenvectors of T
    float2 *W;          // [mats][n][32] A x in float-float (hi, lo), from the Newton residual pass
    double *V;          // [mats][n][d]
    double *eig;        // [mats][d]
    int *flag;          // [mats] 1: residual check failed, the float-float solver redoes the matrix
    int *redo_count;    // matrices flagged (added to; read and cleared by the host)
    float tol;
};

__host__ __device__ inline int poff(int i) { return i * (i + 1) / 2; }
// Lower triangle packed by columns: entry (i, j), i >= j, at coff(j, n) + i - j.
__host__ __device__ inline int coff(int j, int n) { return j * n - j * (j - 1) / 2; }

// Shared-memory plan in floats (every region starts on a 16-byte boundary):
// packed triangle (later the float-float W' panel), the X and U panels, seven
// n-vectors, block-reduction slots, per-warp column partial sums, eigenvalues, order.
struct Smem32 {
    int ap, x, u, vec, red, pacc, pden, lam, ord, total;
};
__host__ __device__ inline int up4(int v) { return (v + 3) & ~3; }
__host__ __device__ inline Smem32 smem32_plan(int n) {
    Smem32 s;
    const int apsz = up4(poff(n) > 2 * n * kXS ? poff(n) : 2 * n * kXS);
    s.ap = 0;
    s.x = apsz;
    s.u = s.x + up4(n * kXS);
    s.vec = s.u + up4(n * kXS);
    s.red = s.vec + 7 * up4(n);
    s.pacc = s.red + 64;
    s.pden = s.pacc + 2 * kNW * 32;
    s.lam = s.pden + 2 * kNW * 32;
    s.ord = s.lam + 32;
    s.total = s.ord + 32;
    return s;
}

__device__ __forceinline__ float warp_sum_f(float s) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// Column c of an [n][kXS] panel in the registers of one warp: lane l holds rows l + 32 q.
__device__ __forceinline__ void col_load(const float *p, int n, int lane, float (&r)[kQ]) {
#pragma unroll
    for (int q = 0; q < kQ; q++) {
        const int i = lane + 32 * q;
        r[q] = i < n ? p[(size_t)i * kXS] : 0.0f;
    }
}
__device__ __forceinline__ void col_store(float *p, int n, int lane, const float (&r)[kQ]) {
#pragma unroll
    for (int q = 0; q < kQ; q++) {
        const int i = lane + 32 * q;
        if (i < n) p[(size_t)i * kXS] = r[q];
    }
}
// r0, r1 <- (I - tau v v^T) r0, r1 for the reflector v stored in rows m0..n-1 of vk (vk[i],
// i >= m0): two columns at once, so each entry of v is loaded once for both.
__device__ __forceinline__ void reflect2(float (&r0)[kQ], float (&r1)[kQ], const float *vk, float tau, int m0, int n,
                                         int lane) {
    float v[kQ], s0 = 0.0f, s1 = 0.0f;
#pragma unroll
    for (int q = 0; q < kQ; q++) {
        const int i = lane + 32 * q;
        v[q] = 0.0f;
        if (32 * q + 31 >= m0 && i >= m0 && i < n) v[q] = vk[i];
        s0 = fmaf(v[q], r0[q], s0);
        s1 = fmaf(v[q], r1[q], s1);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    }
    s0 *= tau;
    s1 *= tau;
#pragma unroll
    for (int q = 0; q < kQ; q++) {
        r0[q] = fmaf(-s0, v[q], r0[q]);
        r1[q] = fmaf(-s1, v[q], r1[q]);
    }
}

// r -= (z_j . r) z_j for column j of the [n][32] eigenvectors of T.
__device__ __forceinline__ void project_out_z(float (&r)[kQ], const float *Zg, int j, int n, int lane) {
    float z[kQ], s = 0.0f;
#pragma unroll
    for (int q = 0; q < kQ; q++) {
        const int i = lane + 32 * q;
        z[q] = i < n ? Zg[(size_t)i * 32 + j] : 0.0f;
        s = fmaf(z[q], r[q], s);
    }
    s = warp_sum_f(s);
#pragma unroll
    for (int q = 0; q < kQ; q++) r[q] = fmaf(-s, z[q], r[q]);
}
// Number of eigenvalues of T below x (the signs of the LDL^T pivots of T - x I).
// The approximate division (2 ulp) only perturbs pivots that are not near zero, and
// a count off by one near an eigenvalue moves that bisection by one FP32 step.
__device__ int sturm32(const float *dg, const float *e2, int n, float x) {
    int cnt = 0;
    float q = dg[0] - x;
    if (fabsf(q) < 1e-30f) q = -1e-30f;
    cnt += q < 0.0f;
    for (int i = 1; i < n; i++) {
        q = (dg[i] - x) - __fdividef(e2[i - 1], q);
        if (fabsf(q) < 1e-30f) q = -1e-30f;
        cnt += q < 0.0f;
    }
    return cnt;
}

// Solve (T - sigma I) y = b in place (b: column j of a panel, stride kXS) by
// Gaussian elimination with partial pivoting; the U factor's three diagonals
// go to scr [3][n][32] (lane j's column).  Pivots below `tiny` in magnitude are
// replaced by +-tiny.  Run by one lane per column.
__device__ void tri_solve_piv(const float *dg, const float *ed, int n, float sigma, float tiny, float *b,
                              float *scr, int j) {
    float *u0 = scr, *u1 = scr + (size_t)n * 32, *u2 = scr + (size_t)2 * n * 32;
    // forward elimination: row i holds (r0, r1, r2) on columns (i, i+1, i+2) and rhs rb
    float r0 = dg[0] - sigma, r1 = n > 1 ? ed[0] : 0.0f, r2 = 0.0f, rb = b[0];
    for (int i = 0; i < n - 1; i++) {
        const float s0 = ed[i], s1 = dg[i + 1] - sigma, s2 = (i + 1 < n - 1) ? ed[i + 1] : 0.0f;
        const float sb = b[(size_t)(i + 1) * kXS];
        float p0, p1, p2, pb, q0, q1, q2, qb;  // pivot row p, other row q
        if (fabsf(r0) >= fabsf(s0)) {
            p0 = r0, p1 = r1, p2 = r2, pb = rb, q0 = s0, q1 = s1, q2 = s2, qb = sb;
        } else {
            p0 = s0, p1 = s1, p2 = s2, pb = sb, q0 = r0, q1 = r1, q2 = r2, qb = rb;
        }
        if (fabsf(p0) < tiny) p0 = p0 < 0.0f ? -tiny : tiny;
        const float rp = __fdividef(1.0f, p0);
        const float l = q0 * rp;  // |l| <= 1 except at replaced pivots
        u0[(size_t)i * 32 + j] = rp;  // the pivot's reciprocal: back substitution multiplies
        u1[(size_t)i * 32 + j] = p1;
        u2[(size_t)i * 32 + j] = p2;
        b[(size_t)i * kXS] = pb;
        // eliminated row becomes the next row (columns i+1, i+2, i+3: the last is 0)
        r0 = fmaf(-l, p1, q1);
        r1 = fmaf(-l, p2, q2);
        r2 = 0.0f;
        rb = fmaf(-l, pb, qb);
    }
    if (fabsf(r0) < tiny) r0 = r0 < 0.0f ? -tiny : tiny;
    // back substitution (u0 holds the pivots' reciprocals)
    float y2 = 0.0f, y1 = rb / r0;
    b[(size_t)(n - 1) * kXS] = y1;
    for (int i = n - 2; i >= 0; i--) {
        const float y0 = (b[(size_t)i * kXS] - u1[(size_t)i * 32 + j] * y1 - u2[(size_t)i * 32 + j] * y2) *
                         u0[(size_t)i * 32 + j];
        b[(size_t)i * kXS] = y0;
        y2 = y1;
        y1 = y0;
    }
}

__global__ void __launch_bounds__(kT, 1) k_eig32(Eig32Args a) {
    const int n = a.n, d = a.d, mat = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    extern __shared__ __align__(16) float sm[];
    const Smem32 L = smem32_plan(n);
    const int n4 = up4(n);
    float *Ap = sm + L.ap;                                   // packed lower triangle, then W' (float-float)
    float *X = sm + L.x;                                     // [n][kXS] x (then x'.hi)
    float *U = sm + L.u;                                     // [n][kXS] residuals, corrections (then x'.lo)
    float *vs = sm + L.vec;                                  // [n] current reflector
    float *ps = vs + n4;                                     // [n] p = tau A v
    float *dT = ps + n4, *eT = dT + n4, *e2 = eT + n4;       // T
    float *tauv = e2 + n4, *v1s = tauv + n4;                 // reflector scalars: tau_k, first entry v_k[k+1]
    float *red = sm + L.red;                                 // [64]
    ffa::acc *pacc = reinterpret_cast<ffa::acc *>(sm + L.pacc);  // [kNW][32] x'.w' per warp and column
    ffa::acc *pden = reinterpret_cast<ffa::acc *>(sm + L.pden);  // [kNW][32] x'.x' per warp and column
    float *lamv = sm + L.lam;                                    // [32] eigenvalues (FP32)
    int *ord = reinterpret_cast<int *>(sm + L.ord);              // [32] output position of each column

    const float2 *A = a.cov + (size_t)mat * n * n;
    float *scr = a.scr + (size_t)mat * 3 * n * 32;
    float *Zg = a.Z + (size_t)mat * n * 32;
    float2 *Wg = a.W + (size_t)mat * n * 32;

    // ---------------------------------------------------------------- 0. load hi parts (column j = row j)
    for (int jc = warp; jc < n; jc += kNW) {
        float *col = Ap + coff(jc, n) - jc;  // col[i] = A(i, jc), i >= jc
        for (int i = jc + lane; i < n; i += 32) col[i] = A[(size_t)jc * n + i].x;
    }
    __syncthreads();

    // ---------------------------------------------------------------- 1. tridiagonalisation (FP32)
    // Reflector k is formed in place in column k of the packed triangle (rows k+1..n-1; its
    // first entry v1 replaces the sub-diagonal entry, which goes to eT as alpha) and stays
    // there for the later passes.  pv: the product of the trailing block with the current
    // reflector (unscaled); red: partial sums of p.v (K = tau^2/2 p.v); nv: column k+1 after
    // the update by reflector k; pw: per-warp row partials [kNW][n+1]; dp: per-lane column
    // partials [n][32].  Two CTA barriers per step.
    float *pv = ps;
    float *bc = vs;               // reflector k+1 for all warps: v1, tau, the stored first entry x1
    float *nv = X, *dp = X + n4;  // the X panel is free until the eigenvectors
    float *pw = U;                // the U panel likewise
    const int pws = n + 1;        // row stride of pw (the four threads of a row hit four banks)
    auto colp = [&](int c) { return Ap + coff(c, n) - c; };  // colp(c)[i] = A(i, c), i >= c
    // alpha, tau and first entry v1 of the reflector that maps (x1, rest) to (alpha, 0),
    // sig = |rest|^2
    auto reflector = [](float x1, float sig, float &alpha, float &v1) -> float {
        alpha = x1;
        v1 = 0.0f;
        if (!(sig > 0.0f)) return 0.0f;
        const float nn = fmaf(x1, x1, sig);
        const float nrm = sqrtf(nn);
        alpha = x1 >= 0.0f ? -nrm : nrm;
        v1 = x1 - alpha;
        return 1.0f / (nn - alpha * x1);
    };
    // Step k's pass over columns j0 = k+2 .. n-1 of the trailing block, warp per column
    // (columns j0 + warp + 32 s).  With UPD, the rank-2 update A -= v w^T + w v^T of
    // reflector k (v = column k, w = tau p - K v formed where needed: every thread knows K
    // and tau); with ACC, the product of the updated entries with column k+1 updated by
    // reflector k (the next reflector as stored: its first entry is corrected in
    // reduce_pass).  Lane l of a warp meets only rows i_q = j0 + warp + l + 32 q (q >= s in
    // column s), so v, w and the updated column k+1 at those rows, and their row sums, stay
    // in registers; the row sums go to pw[warp], each lane's column dot to dp.
    // (m0 = k+1; vjm, wjm: v and w at row m0.)
    auto fused_pass = [&](auto upd_c, auto acc_c, int j0, const float *vc, const float *cm, float tau, float K,
                          float vjm, float wjm) {
        constexpr bool UPD = decltype(upd_c)::value, ACC = decltype(acc_c)::value;
        const int rb = j0 + warp + lane;
        const int S = n - j0 - warp > 0 ? (n - j0 - warp + 31) >> 5 : 0;  // columns of this warp
        if (S == 0) return;  // no column: nothing of this warp is read
        // row groups q >= S lie below row n - 1 in every lane (rb + 32 S >= j0 + warp + 32 S >= n)
        float vq[kQ], pr[kQ], vcq[kQ], wq[kQ];
#pragma unroll
        for (int q = 0; q < kQ; q++) {
            const int i = rb + 32 * q;
            vcq[q] = 0.0f, wq[q] = 0.0f, vq[q] = 0.0f, pr[q] = 0.0f;
            if (q < S && i < n) {
                if (UPD) {
                    vcq[q] = vc[i];
                    wq[q] = fmaf(-K, vcq[q], tau * pv[i]);
                }
                if (ACC) vq[q] = UPD ? fmaf(-vcq[q], wjm, fmaf(-wq[q], vjm, cm[i])) : cm[i];
            }
        }
#pragma unroll
        for (int s = 0; s < kQ; s++) {
            if (s < S) {
                const int jc = j0 + warp + 32 * s;
                float *col = colp(jc);
                float vj = 0.0f, wj = 0.0f, vnj = 0.0f;
                if (UPD) {
                    vj = vc[jc];
                    wj = fmaf(-K, vj, tau * pv[jc]);
                }
                if (ACC) vnj = UPD ? fmaf(-vj, wjm, fmaf(-wj, vjm, cm[jc])) : cm[jc];
                float dot = 0.0f;
#pragma unroll
                for (int q = s; q < kQ; q++) {
                    const int i = rb + 32 * q;
                    if (q < S && i < n) {
                        float a = col[i];
                        if (UPD) {
                            a = fmaf(-vcq[q], wj, fmaf(-wq[q], vj, a));
                            col[i] = a;
                        }
                        if (ACC) {
                            dot = fmaf(a, vq[q], dot);
                            if (q > s || lane > 0) pr[q] = fmaf(a, vnj, pr[q]);  // below the diagonal
                        }
                    }
                }
                if (ACC) dp[(jc - j0) * 32 + lane] = dot;
            }
        }
        if (ACC) {
#pragma unroll
            for (int q = 0; q < kQ; q++) {
                const int i = rb + 32 * q;
                if (q < S && i < n) pw[warp * pws + i] = pr[q];
            }
        }
    };
    // Column m0 = k+1 updated by reflector k (rows m0..n-1, the same operations as the
    // pass's) into nv, and reflector k+1 from it: one warp, while the others run the pass
    auto next_column = [&](bool upd, const float *vc, const float *cm, int m0, float tau, float K, float vjm,
                           float wjm, bool has_next) {
        float sq = 0.0f, x1 = 0.0f;
#pragma unroll
        for (int q = 0; q < kQ; q++) {
            const int i = m0 + lane + 32 * q;
            if (i < n) {
                float c = cm[i];
                if (upd) {
                    const float vi = vc[i], wi = fmaf(-K, vi, tau * pv[i]);
                    c = fmaf(-vi, wjm, fmaf(-wi, vjm, c));
                }
                nv[i] = c;
                if (i >= m0 + 2) sq = fmaf(c, c, sq);
                if (i == m0 + 1) x1 = c;
            }
        }
        sq = warp_sum_f(sq);
        x1 = __shfl_sync(0xffffffffu, x1, 1);  // row m0 + 1: lane 1, q = 0
        if (has_next && lane == 0) {
            float alpha, v1;
            const float t = reflector(x1, sq, alpha, v1);
            eT[m0] = alpha, tauv[m0] = t, v1s[m0] = v1;
            bc[0] = v1, bc[1] = t, bc[2] = x1;
        }
    };
    // pv[i] (i >= j0): the row partials of warps 0..i-j0 (the only warps that reach row i)
    // plus the 32 lane partials of column i, four threads per row, fixed order, plus
    // dv A(i, j0) (dv = v1 - x1: the reflector's first entry in place of the stored one);
    // the products pv_i vn_i summed per warp into red (the next step's K)
    auto reduce_pass = [&](int j0, const float *vnp, float v1n, float dv) {
        if (j0 + (warp << 3) >= n) {  // no row of this warp
            if (lane == 0) red[warp] = 0.0f;
            return;
        }
        const int i = j0 + (tid >> 2), part = tid & 3;
        float t = 0.0f, kp = 0.0f;
        if (i < n) {
            const int wmax = min(kNW - 1, i - j0);
#pragma unroll
            for (int m = 0; m < kNW / 4; m++) {
                const int w = (kNW / 4) * part + m;  // contiguous warp ranges: the four parts hit four bank groups
                if (w <= wmax) t += pw[w * pws + i];
            }
            const float4 *c = reinterpret_cast<const float4 *>(dp + (i - j0) * 32 + part * 8);
            const float4 c0 = c[0], c1 = c[1];
            t += ((c0.x + c0.y) + (c0.z + c0.w)) + ((c1.x + c1.y) + (c1.z + c1.w));
        }
        t += __shfl_xor_sync(0xffffffffu, t, 1);
        t += __shfl_xor_sync(0xffffffffu, t, 2);
        if (i < n && part == 0) {
            t = fmaf(dv, colp(j0)[i], t);
            pv[i] = t;
            kp = t * (i == j0 ? v1n : vnp[i]);
        }
        kp = warp_sum_f(kp);
        if (lane == 0) red[warp] = kp;
    };
    if (tid == 0) {
        for (int i = n - 2 < 0 ? 0 : n - 2; i < n; i++) eT[i] = 0.0f, tauv[i] = 0.0f;
    }
    // reflector 0 and its product with the untouched trailing block
    float tau_cur = 0.0f;
    if (n >= 3) {
        const float *c0 = colp(0);
        if (warp == kNW - 1) next_column(false, nullptr, c0, 0, 0.0f, 0.0f, 0.0f, 0.0f, true);
        __syncthreads();
        tau_cur = bc[1];
        if (tau_cur != 0.0f) fused_pass(kFalse, kTrue, 1, nullptr, c0, 0.0f, 0.0f, 0.0f, 0.0f);
        __syncthreads();
        if (tau_cur != 0.0f) reduce_pass(1, c0, bc[0], bc[0] - bc[2]);
        if (tid == 0) Ap[1] = bc[0];  // column 0 now holds reflector 0
        __syncthreads();
    }
    for (int k = 0; k + 2 < n; k++) {
        const int m0 = k + 1;
        const float *vc = colp(k);  // reflector k
        float *cm = colp(m0);
        const bool has_next = k + 3 < n;
        const bool upd = tau_cur != 0.0f;
        // K = tau^2/2 p.v from the previous reduction; v and w at row m0 (every thread)
        float K = 0.0f, vjm = 0.0f, wjm = 0.0f;
        if (upd) {
            K = 0.5f * tau_cur * tau_cur * warp_sum_f(red[lane]);
            vjm = vc[m0];
            wjm = fmaf(-K, vjm, tau_cur * pv[m0]);
        }
        if (warp == kNW - 1) next_column(upd, vc, cm, m0, tau_cur, K, vjm, wjm, has_next);
        if (tid == 0) dT[k] = vc[k];
        if (upd && has_next) fused_pass(kTrue, kTrue, k + 2, vc, cm, tau_cur, K, vjm, wjm);
        else if (upd) fused_pass(kTrue, kFalse, k + 2, vc, cm, tau_cur, K, vjm, wjm);
        else if (has_next) fused_pass(kFalse, kTrue, k + 2, vc, cm, tau_cur, K, vjm, wjm);
        __syncthreads();
        const float tau_next = has_next ? bc[1] : 0.0f;
        if (tau_next != 0.0f) reduce_pass(k + 2, nv, bc[0], bc[0] - bc[2]);
        // store the updated column k+1 (reflector k+1 in its rows below the diagonal)
        for (int i = m0 + tid; i < n; i += kT) cm[i] = (has_next && i == m0 + 1) ? bc[0] : nv[i];
        tau_cur = tau_next;
        __syncthreads();
    }
    if (tid == 0) {
        if (n >= 2) {
            dT[n - 2] = Ap[coff(n - 2, n)];
            eT[n - 2] = Ap[coff(n - 2, n) + 1];
            tauv[n - 2] = 0.0f;
        }
        dT[n - 1] = Ap[coff(n - 1, n)];
        eT[n - 1] = 0.0f;
        tauv[n - 1] = 0.0f;
    }
    __syncthreads();
    for (int i = tid; i < n; i += kT) e2[i] = eT[i] * eT[i];
    // Gershgorin bounds (block min / max)
    float glo = 3e38f, ghi = -3e38f;
    for (int i = tid; i < n; i += kT) {
        const float rr = (i > 0 ? fabsf(eT[i - 1]) : 0.0f) + (i < n - 1 ? fabsf(eT[i]) : 0.0f);
        glo = fminf(glo, dT[i] - rr);
        ghi = fmaxf(ghi, dT[i] + rr);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        glo = fminf(glo, __shfl_xor_sync(0xffffffffu, glo, o));
        ghi = fmaxf(ghi, __shfl_xor_sync(0xffffffffu, ghi, o));
    }
    __syncthreads();
    if (lane == 0) red[warp] = glo, red[32 + warp] = ghi;
    __syncthreads();
    glo = red[0];
    ghi = red[32];
    for (int w = 1; w < kNW; w++) glo = fminf(glo, red[w]), ghi = fmaxf(ghi, red[32 + w]);
    const float tnorm = fmaxf(fabsf(glo), fabsf(ghi)) + 1e-30f;
    const float tiny = tnorm * 0x1p-40f;

    // ---------------------------------------------------------------- 2. eigenvalues, eigenvectors of T
    // a first round over the whole CTA: the Sturm count at np points of the Gershgorin interval
    // (in the U panel, free until the inverse iteration: np = kT, fewer when the panel is
    // smaller), so that every warp starts its own multisection from a bracket of 1/(np+1)
    const float span = ghi - glo;
    const float lo0 = glo - 1e-3f * span - 1e-30f, hi0 = ghi + 1e-3f * span + 1e-30f;
    const int np = n * kXS < kT ? n * kXS : kT;
    auto grid_x = [&](int m) { return lo0 + (hi0 - lo0) * (float)(m + 1) / (float)(np + 1); };
    int *cnt0 = reinterpret_cast<int *>(U);
    if (tid < np) cnt0[tid] = sturm32(dT, e2, n, grid_x(tid));
    __syncthreads();
    if (warp < d) {  // warp t: the eigenvalue of ascending index n-1-t (multisection, 32 points per round)
        const int t = warp, target = n - 1 - t;
        // the first grid point whose count exceeds the target (lane l scans points 32 l .. 32 l + 31)
        int first = np;
        for (int m = 32 * lane; m < 32 * lane + 32 && m < np; m++) {
            if (cnt0[m] > target) {
                first = m;
                break;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) first = min(first, __shfl_xor_sync(0xffffffffu, first, o));
        float lo = first > 0 ? grid_x(first - 1) : lo0, hi = first < np ? grid_x(first) : hi0;
        for (int round = 0; round < 16; round++) {
            const float x = lo + (hi - lo) * (float)(lane + 1) / 33.0f;
            const int c = sturm32(dT, e2, n, x);
            const unsigned mask = __ballot_sync(0xffffffffu, c > target);
            const float x31 = __shfl_sync(0xffffffffu, x, 31);
            if (mask == 0u) {
                lo = x31;
            } else {
                const int f = __ffs(mask) - 1;
                const float xf = __shfl_sync(0xffffffffu, x, f);
                const float xp = __shfl_sync(0xffffffffu, x, f > 0 ? f - 1 : 0);
                hi = xf;
                if (f > 0) lo = xp;
            }
            if (hi - lo <= 2.4e-7f * fmaxf(fabsf(lo), fabsf(hi)) + 1e-30f) break;
        }
        if (lane == 0) lamv[t] = 0.5f * lo + 0.5f * hi;
    }
    __syncthreads();
    if (warp == 0 && lane < d) {  // inverse iteration, lane j = eigenvector j (in the U panel)
        const int j = lane;
        const float sg = lamv[j];
        float *z = U + j;
        for (int i = 0; i < n; i++) {
            unsigned h = (unsigned)(i + 1) * 2654435761u ^ (unsigned)(j + 1) * 40503u;
            h ^= h >> 15;
            h *= 2246822519u;
            h ^= h >> 13;
            z[(size_t)i * kXS] = 1.0f + 0.5f * ((float)(h & 0xffffu) / 65536.0f - 0.5f);
        }
        for (int it = 0; it < 2; it++) {
            tri_solve_piv(dT, eT, n, sg, tiny, z, scr, j);
            float mx = 0.0f;
            for (int i = 0; i < n; i++) mx = fmaxf(mx, fabsf(z[(size_t)i * kXS]));
            const float sc = mx > 0.0f ? 1.0f / mx : 1.0f;
            float nn = 0.0f;
            for (int i = 0; i < n; i++) {
                const float v = z[(size_t)i * kXS] * sc;
                z[(size_t)i * kXS] = v;
                nn = fmaf(v, v, nn);
            }
            const float inv = rsqrtf(nn);
            for (int i = 0; i < n; i++) z[(size_t)i * kXS] *= inv;
        }
        for (int i = 0; i < n; i++) {
            const float v = z[(size_t)i * kXS];
            X[(size_t)i * kXS + j] = v;
            Zg[(size_t)i * 32 + j] = v;
        }
    }
    __syncthreads();
    // back-transformation x_j = H_0 ... H_{n-3} z_j, columns 2w and 2w+1 in the registers of
    // warp w (a missing second column is carried as zeros)
    if (2 * warp < d) {
        const int j0 = 2 * warp, j1 = j0 + 1 < d ? j0 + 1 : j0;
        float xr0[kQ], xr1[kQ];
        col_load(X + j0, n, lane, xr0);
        col_load(X + j1, n, lane, xr1);
        for (int k = n - 3; k >= 0; k--) {
            const float tau = tauv[k];
            if (tau != 0.0f) reflect2(xr0, xr1, Ap + coff(k, n) - k, tau, k + 1, n, lane);  // rows k+1..n-1
        }
        col_store(X + j0, n, lane, xr0);
        if (j1 != j0) col_store(X + j1, n, lane, xr1);
    }
    __syncthreads();

    // ---------------------------------------------------------------- 3. Newton correction
    // r = A x - sigma x (float-float; A's hi and lo parts, exact FP32 products), rounded into U;
    // rows i and i + 32 of a warp together, two columns of A per 16-byte load when n is even
    // (the terms of each row are added in the same order either way)
    const bool pairs = (n & 1) == 0;  // float2 rows start on 16-byte boundaries
    auto acc_term = [](float &S, float &Cc, float a_hi, float a_lo, float xv) {
        const float p = __fmul_rn(a_hi, xv);
        float e = __fmaf_rn(a_hi, xv, -p);
        e = __fmaf_rn(a_lo, xv, e);
        const ff t = ffa::two_sum(S, p);
        S = t.hi;
        Cc = __fadd_rn(Cc, __fadd_rn(t.lo, e));
    };
    for (int i0 = warp; i0 < n; i0 += 2 * kNW) {
        const int i1 = i0 + kNW < n ? i0 + kNW : i0;
        if (lane < d) {
            const float2 *A0 = A + (size_t)i0 * n, *A1 = A + (size_t)i1 * n;
            float S0 = 0.0f, C0 = 0.0f, S1 = 0.0f, C1 = 0.0f;
            int l = 0;
            if (pairs) {
                for (; l < n; l += 2) {
                    const float4 a0 = *reinterpret_cast<const float4 *>(A0 + l);
                    const float4 a1 = *reinterpret_cast<const float4 *>(A1 + l);
                    const float x0 = X[(size_t)l * kXS + lane], x1 = X[(size_t)(l + 1) * kXS + lane];
                    acc_term(S0, C0, a0.x, a0.y, x0);
                    acc_term(S1, C1, a1.x, a1.y, x0);
                    acc_term(S0, C0, a0.z, a0.w, x1);
                    acc_term(S1, C1, a1.z, a1.w, x1);
                }
            }
            for (; l < n; l++) {
                const float xv = X[(size_t)l * kXS + lane];
                acc_term(S0, C0, A0[l].x, A0[l].y, xv);
                acc_term(S1, C1, A1[l].x, A1[l].y, xv);
            }
            for (int h = 0; h < 2; h++) {
                const int i = h ? i1 : i0;
                if (h && i1 == i0) break;
                const float S = h ? S1 : S0, Cc = h ? C1 : C0;
                const ff w = ffa::two_sum(S, Cc);  // A x, kept for the Rayleigh quotient
                Wg[(size_t)i * 32 + lane] = make_float2(w.hi, w.lo);
                // minus sigma x (the product exact as a pair)
                const float xi = X[(size_t)i * kXS + lane], sg = lamv[lane];
                const float p = __fmul_rn(sg, xi);
                const float e = __fmaf_rn(sg, xi, -p);
                const ff t = ffa::two_sum(S, -p);
                U[(size_t)i * kXS + lane] = __fadd_rn(t.hi, __fadd_rn(Cc, __fsub_rn(t.lo, e)));
            }
        }
    }
    __syncthreads();
    // u = Q^T r = H_{n-3} ... H_0 r, then u -= (z.u) z; warp per column
    if (2 * warp < d) {
        const int j0 = 2 * warp, j1 = j0 + 1 < d ? j0 + 1 : j0;
        float ur0[kQ], ur1[kQ];
        col_load(U + j0, n, lane, ur0);
        col_load(U + j1, n, lane, ur1);
        for (int k = 0; k + 2 < n; k++) {
            const float tau = tauv[k];
            if (tau != 0.0f) reflect2(ur0, ur1, Ap + coff(k, n) - k, tau, k + 1, n, lane);
        }
        project_out_z(ur0, Zg, j0, n, lane);
        col_store(U + j0, n, lane, ur0);
        if (j1 != j0) {
            project_out_z(ur1, Zg, j1, n, lane);
            col_store(U + j1, n, lane, ur1);
        }
    }
    __syncthreads();
    if (warp == 0 && lane < d) tri_solve_piv(dT, eT, n, lamv[lane], tiny, U + lane, scr, lane);
    __syncthreads();
    // y -= (z.y) z, then delta = Q y = H_0 ... H_{n-3} y into U
    if (2 * warp < d) {
        const int j0 = 2 * warp, j1 = j0 + 1 < d ? j0 + 1 : j0;
        float ur0[kQ], ur1[kQ];
        col_load(U + j0, n, lane, ur0);
        col_load(U + j1, n, lane, ur1);
        project_out_z(ur0, Zg, j0, n, lane);
        project_out_z(ur1, Zg, j1, n, lane);
        for (int k = n - 3; k >= 0; k--) {
            const float tau = tauv[k];
            if (tau != 0.0f) reflect2(ur0, ur1, Ap + coff(k, n) - k, tau, k + 1, n, lane);
        }
        col_store(U + j0, n, lane, ur0);
        if (j1 != j0) col_store(U + j1, n, lane, ur1);
    }
    __syncthreads();

    // ---------------------------------------------------------------- 4. Rayleigh quotients, residuals, output
    // x' = x - delta, and A x' = A x - A delta: A x in float-float from the residual pass,
    // A delta in FP32 (delta is the Newton correction, so the rounding of its product lies
    // far below the residual tolerance); the reflectors are no longer needed, so A delta
    // goes where the packed triangle was
    float *G = Ap;  // [n][kXS]
    for (int i0 = warp; i0 < n; i0 += 2 * kNW) {
        const int i1 = i0 + kNW < n ? i0 + kNW : i0;
        if (lane < d) {
            const float2 *A0 = A + (size_t)i0 * n, *A1 = A + (size_t)i1 * n;
            float g0 = 0.0f, g1 = 0.0f;
            int l = 0;
            if (pairs) {
                for (; l < n; l += 2) {
                    const float4 a0 = *reinterpret_cast<const float4 *>(A0 + l);
                    const float4 a1 = *reinterpret_cast<const float4 *>(A1 + l);
                    const float u0 = U[(size_t)l * kXS + lane], u1 = U[(size_t)(l + 1) * kXS + lane];
                    g0 = fmaf(a0.z, u1, fmaf(a0.x, u0, g0));
                    g1 = fmaf(a1.z, u1, fmaf(a1.x, u0, g1));
                }
            }
            for (; l < n; l++) {
                const float u = U[(size_t)l * kXS + lane];
                g0 = fmaf(A0[l].x, u, g0);
                g1 = fmaf(A1[l].x, u, g1);
            }
            G[(size_t)i0 * kXS + lane] = g0;
            if (i1 != i0) G[(size_t)i1 * kXS + lane] = g1;
        }
    }
    __syncthreads();
    // x' as the pair (X, U) = two_sum(x, -delta); per warp and column, over the warp's rows
    // i = warp, warp + 32, ...: partial x'^T A x' = x^T w - 2 w^T delta + delta^T (A delta)
    // (A symmetric, so x^T A delta = w^T delta: only the second-order term carries the
    // rounding of the FP32 product) and x'^T x'
    auto wprime = [&](int i, int j) {
        const float2 w = Wg[(size_t)i * 32 + j];
        return ffa::sub(ffa::make(w.x, w.y), ffa::make(G[(size_t)i * kXS + j], 0.0f));
    };
    if (lane < d) {
        ffa::acc P = ffa::acc_zero(), Q = ffa::acc_zero();
        for (int i = warp; i < n; i += kNW) {
            const float xi = X[(size_t)i * kXS + lane], di = U[(size_t)i * kXS + lane];
            const float2 w2 = Wg[(size_t)i * 32 + lane];
            const ff w = ffa::make(w2.x, w2.y);
            ffa::acc_fma(P, ffa::make(xi, 0.0f), w);
            ffa::acc_fma(P, ffa::make(-2.0f * di, 0.0f), w);
            ffa::acc_fma(P, ffa::make(di, 0.0f), ffa::make(G[(size_t)i * kXS + lane], 0.0f));
            const ff xv = ffa::two_sum(xi, -di);
            X[(size_t)i * kXS + lane] = xv.hi;
            U[(size_t)i * kXS + lane] = xv.lo;
            ffa::acc_fma(Q, xv, xv);
        }
        pacc[warp * 32 + lane] = P;
        pden[warp * 32 + lane] = Q;
    }
    __syncthreads();
    // warp j: lambda_j, residual, norm, sign; lane 0 keeps the results in registers of warp j
    float res_rel = 0.0f;
    ff lam = ffa::zero(), nrm2 = ffa::zero();
    if (warp < d) {
        const int j = warp;
        ffa::acc P = pacc[lane * 32 + j], Q = pden[lane * 32 + j];
        P = ffa::warp_sum(P);
        Q = ffa::warp_sum(Q);
        nrm2 = ffa::acc_value(Q);
        lam = ffa::div(ffa::acc_value(P), nrm2);
        float rr = 0.0f;
        for (int i = lane; i < n; i += 32) {
            const ff xv = ffa::make(X[(size_t)i * kXS + j], U[(size_t)i * kXS + j]);
            const ff r = ffa::sub(wprime(i, j), ffa::mul(lam, xv));
            rr = fmaf(r.hi, r.hi, rr);
        }
        rr = warp_sum_f(rr);
        res_rel = sqrtf(rr) / sqrtf(nrm2.hi);
        if (lane == 0) {
            lamv[j] = lam.hi;   // for the order and the bound (FP32 is enough to rank)
            red[j] = res_rel;
        }
    }
    __syncthreads();
    if (tid == 0) {
        float lmax = 0.0f, rmax = 0.0f;
        for (int j = 0; j < d; j++) lmax = fmaxf(lmax, fabsf(lamv[j])), rmax = fmaxf(rmax, red[j]);
        // descending order of the eigenvalues, the lower column first on ties
        for (int j = 0; j < d; j++) {
            int pos = 0;
            for (int k = 0; k < d; k++) pos += lamv[k] > lamv[j] || (lamv[k] == lamv[j] && k < j);
            ord[j] = pos;
        }
        const int redo = !(rmax <= a.tol * lmax) ? 1 : 0;
        a.flag[mat] = redo;
        if (redo && a.redo_count) atomicAdd(a.redo_count, 1);
    }
    __syncthreads();
    if (warp < d) {
        const int j = warp, pos = ord[j];
        float best = -1.0f;
        int bi = 0x7fffffff;
        for (int i = lane; i < n; i += 32) {
            const float v = fabsf(X[(size_t)i * kXS + j]);
            if (v > best) best = v, bi = i;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) best = ob, bi = oi;
        }
        const double sgn = X[(size_t)bi * kXS + j] < 0.0f ? -1.0 : 1.0;
        const double inv = sgn / sqrt(ffa::to_double(nrm2));
        double *V = a.V + (size_t)mat * n * d;
        for (int i = lane; i < n; i += 32)
            V[(size_t)i * d + pos] = inv * ((double)X[(size_t)i * kXS + j] + (double)U[(size_t)i * kXS + j]);
        if (lane == 0) a.eig[(size_t)mat * d + pos] = ffa::to_double(lam);
    }
}

DeviceOnce g_attrs32;

}  // namespace

bool eig32_ok(int n, int d) { return n >= 2 && n <= 256 && d >= 1 && d <= 32 && d <= n; }

size_t eig32_workspace_bytes(int n, int mats) { return align_up(sizeof(float) * (size_t)mats * 6 * n * 32, 256); }

cudaError_t launch_eig32(const void *cov_ff, int n, int d, int mats, double *V, double *eigvals, void *ws,
                         int *flag_out, int *redo_count, float tol, cudaStream_t st) {
    if (!eig32_ok(n, d)) return cudaErrorNotSupported;
    const size_t smem = sizeof(float) * (size_t)smem32_plan(n).total;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = device_once(g_attrs32, dev, [] {
        return cudaFuncSetAttribute(k_eig32, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    });
    if (e != cudaSuccess) return e;
    if (smem > 227 * 1024) return cudaErrorNotSupported;
    Eig32Args a;
    a.cov = (const float2 *)cov_ff;
    a.n = n;
    a.d = d;
    a.scr = (float *)ws;
    a.Z = (float *)ws + (size_t)mats * 3 * n * 32;
    a.W = (float2 *)((float *)ws + (size_t)mats * 4 * n * 32);
    a.V = V;
    a.eig = eigvals;
    a.flag = flag_out;
    a.redo_count = redo_count;
    a.tol = tol;
    QFCA_LAUNCH("k_eig32", st, k_eig32<<<mats, kT, smem, st>>>(a));
    return cudaGetLastError();
}

}  // namespace qfca
