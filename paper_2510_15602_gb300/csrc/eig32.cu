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
//      with reflector k+1 (formed first from column k+1, updated alone); the
//      row contributions go to per-warp partial vectors, summed in a fixed
//      order.  Reflector k stays in column k (contiguous) for the later passes.
//   2. The top d eigenvalues sigma_j of T by warp multisection on the FP32
//      Sturm count; eigenvectors z_j of T by two steps of inverse iteration
//      (Gaussian elimination with partial pivoting, one lane per eigenvector);
//      back-transformation x_j = Q z_j (warp per column).
//   3. Newton correction per column (x, sigma approximate; A x = lambda x):
//      r = A x - sigma x with A in float-float (exact FP32 products, compensated
//      sums), u = Q^T r, u -= (z.u) z, solve (T - sigma I) y = u (the same
//      pivoted elimination), y -= (z.y) z, x' = x - Q y carried as (x, -Q y).
//      One step squares the FP32 start's error: about 1e-12 of lambda_1/gap.
//   4. lambda_j = x'^T A x' / x'^T x' (float-float), the residual
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
constexpr int kXS = 33;  // row stride of the n x d panels (conflict-free by rows and by columns)

struct Eig32Args {
    const float2 *cov;  // [mats][n][n] float-float (hi, lo) covariance, full symmetric storage
    int n, d;
    float *scr;         // [mats][3][n][32] U factor of the pivoted elimination (one column per lane)
    float *Z;           // [mats][n][32] eigenvectors of T
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
    const int apsz = up4(poff(n)) > 2 * n * kXS ? up4(poff(n)) : 2 * n * kXS;
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

// Sum over the block, the same value in every thread (fixed order).
__device__ __forceinline__ float block_sum_f(float s, float *red) {
    s = warp_sum_f(s);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    float t = 0.0f;
#pragma unroll
    for (int w = 0; w < kNW; w++) t += red[w];
    return t;
}

__device__ int sturm32(const float *dg, const float *e2, int n, float x) {
    int cnt = 0;
    float q = dg[0] - x;
    if (fabsf(q) < 1e-30f) q = -1e-30f;
    cnt += q < 0.0f;
    for (int i = 1; i < n; i++) {
        q = (dg[i] - x) - e2[i - 1] / q;
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
        const float l = q0 / p0;
        u0[(size_t)i * 32 + j] = p0;
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
    // back substitution
    float y2 = 0.0f, y1 = rb / r0;
    b[(size_t)(n - 1) * kXS] = y1;
    for (int i = n - 2; i >= 0; i--) {
        const float y0 = (b[(size_t)i * kXS] - u1[(size_t)i * 32 + j] * y1 - u2[(size_t)i * 32 + j] * y2) /
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

    // ---------------------------------------------------------------- 0. load hi parts (column j = row j)
    for (int jc = warp; jc < n; jc += kNW) {
        float *col = Ap + coff(jc, n) - jc;  // col[i] = A(i, jc), i >= jc
        for (int i = jc + lane; i < n; i += 32) col[i] = A[(size_t)jc * n + i].x;
    }
    __syncthreads();

    // ---------------------------------------------------------------- 1. tridiagonalisation (FP32)
    // vcur: the current reflector v_k, vn: the next one (the two swap every step), pv: the
    // product of the trailing block with v_k (unscaled), wv: w_k
    float *vcur = vs, *pv = ps;
    float *wv = X, *vn = X + n4;  // the X panel is free until the eigenvectors
    float *pw = U;                // [kNW][n] per-warp partial products (the U panel likewise)
    // reflector of column c (rows c+1..n-1) into dst; returns tau (0: nothing to reduce)
    auto make_reflector = [&](int c, float *dst) -> float {
        const float *col = Ap + coff(c, n) - c;
        float part = 0.0f;
        for (int i = c + 2 + tid; i < n; i += kT) part = fmaf(col[i], col[i], part);
        const float sig = block_sum_f(part, red);
        const float x1 = col[c + 1];
        float alpha = x1, tau = 0.0f, v1 = 0.0f;
        if (sig > 0.0f) {
            const float nn = fmaf(x1, x1, sig);
            const float nrm = sqrtf(nn);
            alpha = x1 >= 0.0f ? -nrm : nrm;
            v1 = x1 - alpha;
            tau = 1.0f / (nn - alpha * x1);
        }
        if (tid == 0) {
            eT[c] = alpha;
            tauv[c] = tau;
            v1s[c] = v1;
        }
        for (int i = c + 1 + tid; i < n; i += kT) dst[i] = i == c + 1 ? v1 : col[i];
        return tau;
    };
    // one pass over the columns j0..n-1 of the trailing block: with `upd`, the rank-2
    // update A -= v w^T + w v^T of the current reflector; with `acc`, pv = A vn on the
    // updated entries (column part by warp sums, row part into the warp's partial vector)
    auto fused_pass = [&](int j0, bool upd, bool acc) {
        if (acc) {
            for (int e = tid; e < kNW * n; e += kT) pw[e] = 0.0f;
            __syncthreads();
        }
        float *pwr = pw + (size_t)warp * n;
        for (int jc = j0 + warp; jc < n; jc += kNW) {
            float *col = Ap + coff(jc, n) - jc;
            const float vj = vcur[jc], wj = upd ? wv[jc] : 0.0f, vnj = acc ? vn[jc] : 0.0f;
            float dot = 0.0f;
            for (int i = jc + lane; i < n; i += 32) {
                float a = col[i];
                if (upd) {
                    a = fmaf(-vcur[i], wj, fmaf(-wv[i], vj, a));
                    col[i] = a;
                }
                if (acc) {
                    dot = fmaf(a, vn[i], dot);
                    if (i > jc) pwr[i] = fmaf(a, vnj, pwr[i]);  // row i is always this lane's
                }
            }
            if (acc) {
                dot = warp_sum_f(dot);
                if (lane == 0) pwr[jc] += dot;
            }
        }
        __syncthreads();
        if (acc) {
            for (int i = j0 + tid; i < n; i += kT) {
                float t = 0.0f;
#pragma unroll 8
                for (int w = 0; w < kNW; w++) t += pw[(size_t)w * n + i];
                pv[i] = t;
            }
            __syncthreads();
        }
    };
    if (tid == 0) {
        for (int i = n - 2 < 0 ? 0 : n - 2; i < n; i++) eT[i] = 0.0f, tauv[i] = 0.0f;
    }
    // reflector 0 (into vn) and its product with the untouched trailing block; then it becomes current
    float tau_cur = n >= 3 ? make_reflector(0, vn) : 0.0f;
    __syncthreads();
    if (tau_cur != 0.0f) fused_pass(1, false, true);
    if (n >= 3 && tid == 0) Ap[coff(0, n) + 1] = v1s[0];  // column 0 now holds reflector 0
    {
        float *t = vcur;
        vcur = vn;
        vn = t;
    }
    __syncthreads();
    for (int k = 0; k + 2 < n; k++) {
        if (tid == 0) dT[k] = Ap[coff(k, n)];
        const int m0 = k + 1;
        if (tau_cur != 0.0f) {
            // p = tau A v, K = (tau / 2) p.v, w = p - K v
            float part = 0.0f;
            for (int i = m0 + tid; i < n; i += kT) part = fmaf(pv[i], vcur[i], part);
            const float K = 0.5f * tau_cur * tau_cur * block_sum_f(part, red);
            for (int i = m0 + tid; i < n; i += kT) wv[i] = fmaf(-K, vcur[i], tau_cur * pv[i]);
            __syncthreads();
            // column k+1 alone first: reflector k+1 is formed from it
            float *col = Ap + coff(m0, n) - m0;
            const float vj = vcur[m0], wj = wv[m0];
            for (int i = m0 + tid; i < n; i += kT) col[i] = fmaf(-vcur[i], wj, fmaf(-wv[i], vj, col[i]));
            __syncthreads();
        }
        const bool has_next = k + 3 < n;
        const float tau_next = has_next ? make_reflector(m0, vn) : 0.0f;
        if (has_next) __syncthreads();
        if (tau_cur != 0.0f || tau_next != 0.0f) fused_pass(k + 2, tau_cur != 0.0f, tau_next != 0.0f);
        if (has_next && tid == 0) Ap[coff(m0, n) + 1] = v1s[m0];  // column k+1 now holds reflector k+1
        // reflector k+1 becomes the current one
        float *t = vcur;
        vcur = vn;
        vn = t;
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
    if (warp < d) {  // warp t: the eigenvalue of ascending index n-1-t (multisection, 32 points per round)
        const int t = warp, target = n - 1 - t;
        const float span = ghi - glo;
        float lo = glo - 1e-3f * span - 1e-30f, hi = ghi + 1e-3f * span + 1e-30f;
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
    // back-transformation x_j = H_0 ... H_{n-3} z_j, warp per column
    if (warp < d) {
        float *x = X + warp;
        for (int k = n - 3; k >= 0; k--) {
            const float tau = tauv[k];
            if (tau == 0.0f) continue;
            const int m0 = k + 1;
            float s = 0.0f;
            const float *vk = Ap + coff(k, n) - k;  // reflector k: vk[i], i = k+1..n-1
            for (int i = m0 + lane; i < n; i += 32) s = fmaf(vk[i], x[(size_t)i * kXS], s);
            s = tau * warp_sum_f(s);
            for (int i = m0 + lane; i < n; i += 32) x[(size_t)i * kXS] = fmaf(-s, vk[i], x[(size_t)i * kXS]);
        }
    }
    __syncthreads();

    // ---------------------------------------------------------------- 3. Newton correction
    // r = A x - sigma x (float-float; A's hi and lo parts, exact FP32 products), rounded into U
    for (int i = warp; i < n; i += kNW) {
        if (lane < d) {
            const float2 *Ar = A + (size_t)i * n;
            float S = 0.0f, Cc = 0.0f;
            for (int l = 0; l < n; l++) {
                const float2 av = Ar[l];
                const float xv = X[(size_t)l * kXS + lane];
                const float p = __fmul_rn(av.x, xv);
                float e = __fmaf_rn(av.x, xv, -p);
                e = __fmaf_rn(av.y, xv, e);
                const ff t = ffa::two_sum(S, p);
                S = t.hi;
                Cc = __fadd_rn(Cc, __fadd_rn(t.lo, e));
            }
            // minus sigma x (the product exact as a pair)
            const float xi = X[(size_t)i * kXS + lane], sg = lamv[lane];
            const float p = __fmul_rn(sg, xi);
            const float e = __fmaf_rn(sg, xi, -p);
            const ff t = ffa::two_sum(S, -p);
            U[(size_t)i * kXS + lane] = __fadd_rn(t.hi, __fadd_rn(Cc, __fsub_rn(t.lo, e)));
        }
    }
    __syncthreads();
    // u = Q^T r = H_{n-3} ... H_0 r, then u -= (z.u) z; warp per column
    if (warp < d) {
        float *u = U + warp;
        for (int k = 0; k + 2 < n; k++) {
            const float tau = tauv[k];
            if (tau == 0.0f) continue;
            const int m0 = k + 1;
            float s = 0.0f;
            const float *vk = Ap + coff(k, n) - k;
            for (int i = m0 + lane; i < n; i += 32) s = fmaf(vk[i], u[(size_t)i * kXS], s);
            s = tau * warp_sum_f(s);
            for (int i = m0 + lane; i < n; i += 32) u[(size_t)i * kXS] = fmaf(-s, vk[i], u[(size_t)i * kXS]);
        }
        float s = 0.0f;
        for (int i = lane; i < n; i += 32) s = fmaf(Zg[(size_t)i * 32 + warp], u[(size_t)i * kXS], s);
        s = warp_sum_f(s);
        for (int i = lane; i < n; i += 32) u[(size_t)i * kXS] = fmaf(-s, Zg[(size_t)i * 32 + warp], u[(size_t)i * kXS]);
    }
    __syncthreads();
    if (warp == 0 && lane < d) tri_solve_piv(dT, eT, n, lamv[lane], tiny, U + lane, scr, lane);
    __syncthreads();
    // y -= (z.y) z, then delta = Q y = H_0 ... H_{n-3} y; x' = x - delta kept as the pair (x, -delta)
    if (warp < d) {
        float *u = U + warp;
        float s = 0.0f;
        for (int i = lane; i < n; i += 32) s = fmaf(Zg[(size_t)i * 32 + warp], u[(size_t)i * kXS], s);
        s = warp_sum_f(s);
        for (int i = lane; i < n; i += 32) u[(size_t)i * kXS] = fmaf(-s, Zg[(size_t)i * 32 + warp], u[(size_t)i * kXS]);
        for (int k = n - 3; k >= 0; k--) {
            const float tau = tauv[k];
            if (tau == 0.0f) continue;
            const int m0 = k + 1;
            float t = 0.0f;
            const float *vk = Ap + coff(k, n) - k;
            for (int i = m0 + lane; i < n; i += 32) t = fmaf(vk[i], u[(size_t)i * kXS], t);
            t = tau * warp_sum_f(t);
            for (int i = m0 + lane; i < n; i += 32) u[(size_t)i * kXS] = fmaf(-t, vk[i], u[(size_t)i * kXS]);
        }
        float *x = X + warp;
        for (int i = lane; i < n; i += 32) {
            const ff t = ffa::two_sum(x[(size_t)i * kXS], -u[(size_t)i * kXS]);
            x[(size_t)i * kXS] = t.hi;
            u[(size_t)i * kXS] = t.lo;
        }
    }
    __syncthreads();

    // ---------------------------------------------------------------- 4. Rayleigh quotients, residuals, output
    ff *Wp = reinterpret_cast<ff *>(Ap);  // [n][kXS] w' = A x' (the reflectors are no longer needed)
    for (int i = warp; i < n; i += kNW) {
        if (lane < d) {
            const float2 *Ar = A + (size_t)i * n;
            ffa::acc S = ffa::acc_zero();
            for (int l = 0; l < n; l++) {
                const float2 av = Ar[l];
                ffa::acc_fma(S, ffa::make(av.x, av.y), ffa::make(X[(size_t)l * kXS + lane], U[(size_t)l * kXS + lane]));
            }
            Wp[(size_t)i * kXS + lane] = ffa::acc_value(S);
        }
    }
    __syncthreads();
    // per warp and column: partial x'.w' and x'.x' over the warp's rows i = warp, warp + 32, ...
    if (lane < d) {
        ffa::acc P = ffa::acc_zero(), Q = ffa::acc_zero();
        for (int i = warp; i < n; i += kNW) {
            const ff xv = ffa::make(X[(size_t)i * kXS + lane], U[(size_t)i * kXS + lane]);
            ffa::acc_fma(P, xv, Wp[(size_t)i * kXS + lane]);
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
            const ff r = ffa::sub(Wp[(size_t)i * kXS + j], ffa::mul(lam, xv));
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

size_t eig32_workspace_bytes(int n, int mats) { return align_up(sizeof(float) * (size_t)mats * 4 * n * 32, 256); }

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
    a.V = V;
    a.eig = eigvals;
    a.flag = flag_out;
    a.redo_count = redo_count;
    a.tol = tol;
    QFCA_LAUNCH("k_eig32", st, k_eig32<<<mats, kT, smem, st>>>(a));
    return cudaGetLastError();
}

}  // namespace qfca
