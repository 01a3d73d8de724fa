// eig.cu -- top-d eigenpairs of a symmetric C x C covariance (the eigen-
// decomposition of the single-image PCA fit, arXiv 2510.15602, Sec. 3.3) to
// FP64-class accuracy, with the O(C^3) work on the FP32 pipe.
//
// GB300's SIMT FP64 issues well under one DFMA per clock per SM (measured),
// so the Householder reduction runs in float-float arithmetic (ff.cuh: ~48
// significant bits from error-free FP32 transformations, 128 lanes/clk/SM).
// One thread-block cluster of R CTAs per matrix (R = 2 for C <= 256, up to 8),
// the lower triangle packed in shared memory, rows distributed cyclically:
//   1. Householder tridiagonalisation A = Q T Q^T.  Step k: every CTA holds
//      x = A[k+1.., k] (gathered through distributed shared memory at the end
//      of step k-1) and forms (v, tau) (float-float scalars, one thread); each
//      CTA computes its partial q of A v from the elements it stores (row part
//      and column part of the symmetric product) and pushes it into every
//      CTA; cluster barrier; p = tau sum_r q_r (fixed order),
//      w = p - (tau/2)(p.v) v; each CTA applies A -= v w^T + w v^T to its
//      lower-triangle rows and pushes the new column k+1 into every CTA;
//      cluster barrier.
//   2. Shifts by warp multisection on the FP32 Sturm count; float-float
//      inverse iteration on T (LU with partial pivoting, three solves, scratch
//      per warp in shared memory); selective Gram-Schmidt for shifts within
//      1e-3 ||T||; float-float Rayleigh quotients; stable descending order.
//      (Single-lane FP64 code would issue warp-wide FP64 instructions at the
//      FP64 pipe's rate: it cost milliseconds here.)
//   3. Back-transformation V = H_0 ... H_{n-3} Z in float-float, columns
//      distributed over the cluster; sign normalisation (largest-magnitude
//      entry positive); FP64 output.
// Every wait is a hardware barrier (cluster or CTA): no spin loop.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "ff.cuh"
#include "internal.cuh"

namespace cg = cooperative_groups;

namespace qfca {
namespace {

using ffa::ff;
constexpr int kT = 512;
constexpr int kNW = kT / 32;
constexpr size_t kSmemMax = 200 * 1024;
constexpr size_t kSmemOptIn = 227 * 1024;  // the opt-in maximum of dynamic shared memory per CTA

struct EigArgs {
    const ff *cov;  // [mats][n][n] float-float covariance
    int n, d, R;
    long region0;   // ff elements of the first shared region (packed rows; reused by phases 2/3)
    int nslots;     // warps that can hold an inverse-iteration scratch slot at once
    ff *dg, *ed, *tau, *v0;  // [mats][n]  tridiagonal T and the reflectors' scalars
    ff *Vh;                  // [mats][n][n]  Householder vectors (row k: v_k, length n-k-1)
    ff *Z;                   // [mats][d][n]  eigenvectors of T
    float *sig;              // [mats][d]
    ff *lam;                 // [mats][d]
    int *order;              // [mats][d]
    double *V;               // [mats][n][d]
    double *eig;             // [mats][d]
    const int *redo;         // [mats] or NULL: solve only the matrices whose entry is non-zero
};

__host__ __device__ inline long row_off(int l, int r, int R) {
    return (long)l * (r + 1) + (long)R * l * (l - 1) / 2;
}

__host__ __device__ inline long rows_elems(int n, int R) {
    long mx = 0;
    for (int r = 0; r < R; r++) {
        const int L = r < n ? (n - r + R - 1) / R : 0;
        const long e = row_off(L, r, R);
        if (e > mx) mx = e;
    }
    return mx;
}

// The two halves of a cluster barrier (all threads of every CTA take part).
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory"); }

__device__ __forceinline__ void acc_down(ffa::acc &A, int o) {
    ffa::acc B;
    B.s = __shfl_down_sync(0xffffffffu, A.s, o);
    B.c = __shfl_down_sync(0xffffffffu, A.c, o);
    ffa::acc_merge(A, B);
}

// Pairwise tree over the 16 per-warp sums (same order in every thread and CTA).
__device__ __forceinline__ ff tree16(const ffa::acc *red) {
    ffa::acc T[kNW];
#pragma unroll
    for (int w = 0; w < kNW; w++) T[w] = red[w];
#pragma unroll
    for (int step = 1; step < kNW; step <<= 1)
#pragma unroll
        for (int w = 0; w + step < kNW; w += 2 * step) ffa::acc_merge(T[w], T[w + step]);
    return ffa::acc_value(T[0]);
}

// One entry of the symmetric rank-2 update: a - (vi wj + wi vj), float-float,
// both products kept exact to their FMA error terms and summed into a once.
__device__ __forceinline__ ff rank2(ff a, ff vi, ff wj, ff wi, ff vj) {
    const float p1 = __fmul_rn(vi.hi, wj.hi);
    float e1 = __fmaf_rn(vi.hi, wj.hi, -p1);
    e1 = __fmaf_rn(vi.hi, wj.lo, e1);
    e1 = __fmaf_rn(vi.lo, wj.hi, e1);
    const float p2 = __fmul_rn(wi.hi, vj.hi);
    float e2 = __fmaf_rn(wi.hi, vj.hi, -p2);
    e2 = __fmaf_rn(wi.hi, vj.lo, e2);
    e2 = __fmaf_rn(wi.lo, vj.hi, e2);
    const ff s1 = ffa::two_sum(a.hi, -p1);
    const ff s2 = ffa::two_sum(s1.hi, -p2);
    const float lo = __fadd_rn(__fadd_rn(__fsub_rn(a.lo, __fadd_rn(e1, e2)), s1.lo), s2.lo);
    return ffa::fast_two_sum(s2.hi, lo);
}

// Deterministic block reduction; every thread gets the same value.
__device__ ff block_acc(ffa::acc A, ffa::acc *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc_down(A, o);
    __syncthreads();
    if (lane == 0) red[warp] = A;
    __syncthreads();
    // pairwise tree over the 16 warp sums (same order in every thread and CTA)
    ffa::acc T[kNW];
#pragma unroll
    for (int w = 0; w < kNW; w++) T[w] = red[w];
#pragma unroll
    for (int step = 1; step < kNW; step <<= 1)
#pragma unroll
        for (int w = 0; w + step < kNW; w += 2 * step) ffa::acc_merge(T[w], T[w + step]);
    __syncthreads();
    return ffa::acc_value(T[0]);
}

__device__ int sturm_count(const float *dg, const float *e2, int n, float x) {
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

// LU with partial pivoting of the tridiagonal T - sigma I, in float-float.
// u0i: reciprocal pivots, u1/u2: first/second super-diagonals of U, lm: multipliers.
__device__ void tri_factor(const ff *dg, const ff *ed, int n, ff sigma, ff tiny, ff *u0i, ff *u1, ff *u2, ff *lm,
                           uint8_t *piv) {
    using namespace ffa;
    const ff one = make(1.0f, 0.0f);
    ff r0 = sub(dg[0], sigma), r1 = n > 1 ? ed[0] : zero();
    for (int i = 0; i < n - 1; i++) {
        const ff s0 = ed[i], s1 = sub(dg[i + 1], sigma), s2 = (i + 1 < n - 1) ? ed[i + 1] : zero();
        if (!less(fabs_ff(r0), fabs_ff(s0))) {
            if (r0.hi == 0.0f) r0 = tiny;
            const ff inv = div(one, r0);
            const ff l = mul(s0, inv);
            u0i[i] = inv; u1[i] = r1; u2[i] = zero(); lm[i] = l; piv[i] = 0;
            r0 = sub(s1, mul(l, r1));
            r1 = s2;
        } else {
            const ff inv = div(one, s0);
            const ff l = mul(r0, inv);
            u0i[i] = inv; u1[i] = s1; u2[i] = s2; lm[i] = l; piv[i] = 1;
            const ff n0 = sub(r1, mul(l, s1)), n1 = neg(mul(l, s2));
            r0 = n0; r1 = n1;
        }
    }
    if (r0.hi == 0.0f) r0 = tiny;
    u0i[n - 1] = div(one, r0); u1[n - 1] = zero(); u2[n - 1] = zero();
}

__device__ void tri_solve(int n, const ff *u0i, const ff *u1, const ff *u2, const ff *lm, const uint8_t *piv, ff *x) {
    using namespace ffa;
    for (int i = 0; i < n - 1; i++) {
        if (piv[i]) { const ff t = x[i]; x[i] = x[i + 1]; x[i + 1] = t; }
        x[i + 1] = sub(x[i + 1], mul(lm[i], x[i]));
    }
    x[n - 1] = mul(x[n - 1], u0i[n - 1]);
    if (n >= 2) x[n - 2] = mul(sub(x[n - 2], mul(u1[n - 2], x[n - 1])), u0i[n - 2]);
    for (int i = n - 3; i >= 0; i--)
        x[i] = mul(sub(sub(x[i], mul(u1[i], x[i + 1])), mul(u2[i], x[i + 2])), u0i[i]);
}

__global__ void __launch_bounds__(kT, 1) k_eig_ff(EigArgs a) {
    cg::cluster_group cl = cg::this_cluster();
    const int R = a.R;
    const int r = (int)cl.block_rank();
    const int mat = blockIdx.x / R;
    // every CTA of the cluster leaves here together (before any cluster barrier)
    // when the FP32 + Newton solver has already solved this matrix
    if (a.redo && a.redo[mat] == 0) return;
    const int n = a.n, d = a.d;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nloc = r < n ? (n - r + R - 1) / R : 0;  // own rows i = r + l R

    extern __shared__ __align__(16) unsigned char smraw[];
    ff *rows = reinterpret_cast<ff *>(smraw);        // region 0
    const int nq = (n + 1) & ~1;                     // qbuf row stride (16-byte rows)
    ff *qbuf = rows + a.region0;                     // [R][nq] partial products pushed by every CTA
    ff *xa = qbuf + (size_t)R * nq;                  // [n] current column (x)
    ff *xb = xa + n;                                 // [n] next column
    ff *pbuf = xb + n;                               // [n] column part of the own partial product, then p
    ff *wbuf = pbuf + n;                             // [n]
    ff *pbuf2 = wbuf + n;                            // [n] row part (own rows)
    ff *colb = pbuf2 + n;                            // [n] column k+1 before the update, gathered from every CTA
    ff *pcol1 = colb + n;                            // [n] column part of the second row group
    ffa::acc *red = reinterpret_cast<ffa::acc *>(pcol1 + n);  // [kNW]
    ffa::acc *wsq = red + kNW;                                // [kNW] per-warp squared norms of the next column
    ff *fsc = reinterpret_cast<ff *>(wsq + kNW);              // [4] step scalars
    ff *dpart = fsc + 4;                                      // [8] per-CTA partial products q_r . v

    const ff *S = a.cov + (long)mat * n * n;
    ff *dg = a.dg + (long)mat * n, *ed = a.ed + (long)mat * n;
    ff *tau_g = a.tau + (long)mat * n, *v0_g = a.v0 + (long)mat * n;
    ff *Vh = a.Vh + (long)mat * n * n;

    // ---- own lower-triangle rows; column 0 below the diagonal into every CTA
    for (int l = 0; l < nloc; l++) {
        const int i = r + l * R;
        ff *row = rows + row_off(l, r, R);
        for (int j = tid; j <= i; j += kT) row[j] = S[(long)i * n + j];
    }
    __syncthreads();
    for (int l = tid; l < nloc; l += kT) {
        const int i = r + l * R;
        if (i >= 1) {
            const ff x = rows[row_off(l, r, R)];  // A[i][0]
            for (int dst = 0; dst < R; dst++) cl.map_shared_rank(xa, dst)[i - 1] = x;
        } else {
            dg[0] = rows[0];
        }
    }
    cl.sync();

    ff *xcur = xa, *xnext = xb;
    // ---------------------------------------------------------------- 1. tridiagonalisation
    // One cluster exchange per step: with its partial product q_r each CTA pushes
    // its own rows' entries of column k+1 (before the update); after the barrier
    // every CTA forms w and the updated column k+1 itself, with the same
    // float-float expression the row update uses, so the next step needs no
    // second exchange. The buffers that receive the pushes (qbuf, colb, dpart)
    // are released by a split barrier: each CTA arrives once it has read them and
    // waits just before its next push, so the wait is normally already satisfied.
    ff sig;
    {
        ffa::acc A = ffa::acc_zero();
        for (int j = 1 + tid; j < n - 1; j += kT) ffa::acc_fma(A, xcur[j], xcur[j]);
        sig = block_acc(A, red);
    }
    for (int k = 0; k + 2 < n; k++) {
        const int m = n - k - 1;
        // ---- the reflector (one thread, while the others start on the product)
        if (tid == 0) {
            const ff alpha = xcur[0];
            ff tau = ffa::zero(), ek = alpha, v0 = alpha;
            if (sig.hi > 0.0f) {
                const ff mu = ffa::sqrt_newton(ffa::add(ffa::mul(alpha, alpha), sig));
                if (alpha.hi >= 0.0f) { v0 = ffa::add(alpha, mu); ek = ffa::neg(mu); }
                else { v0 = ffa::sub(alpha, mu); ek = mu; }
                tau = ffa::div_newton(ffa::make(2.0f, 0.0f), ffa::add(ffa::mul(v0, v0), sig));
            }
            fsc[0] = tau;
            fsc[1] = v0;
            fsc[2] = ffa::scale(tau, 0.5f);
            if (r == 0) { tau_g[k] = tau; v0_g[k] = v0; ed[k] = ek; }
            if (k >= 1 && k % R == r) dg[k] = rows[row_off(k / R, r, R) + k];  // updated by step k-1
        }
        int l0 = (k + 1 - r + R - 1) / R;  // first own row with i >= k+1
        if (l0 < 0) l0 = 0;
        int l2 = (k + 2 - r + R - 1) / R;  // first own row with i >= k+2
        if (l2 < 0) l2 = 0;
        // ---- own partial product of A with x (x_0 = alpha in place of v_0; the
        // difference (v_0 - alpha) A e_0 touches only own rows and is added below):
        // column part (sum over own rows i > jc of A[i][jc] x_i): thread (g, c) takes
        // column k+1+c and every other own row below it (row group g), the longest
        // columns on the last warps (warp 0 also forms the reflector);
        // row part (sum over j <= i of A[i][j] x_j): 8 lanes per own row, 4 rows per warp.
        {
            const int g = tid >> 8;
            for (int c = 255 - (tid & 255); c < m; c += 256) {
                const int jc = k + 1 + c;
                ffa::acc Q0 = ffa::acc_zero(), Q1 = ffa::acc_zero();  // two chains for ILP
                int lc = (jc + 1 - r + R - 1) / R;
                if (lc < 0) lc = 0;
                int l = lc + g;
                for (; l + 2 < nloc; l += 4) {
                    const int i0 = r + l * R, i1 = i0 + 2 * R;  // i >= jc + 1 >= k + 2
                    ffa::acc_fma(Q0, rows[row_off(l, r, R) + jc], xcur[i0 - k - 1]);
                    ffa::acc_fma(Q1, rows[row_off(l + 2, r, R) + jc], xcur[i1 - k - 1]);
                }
                if (l < nloc) ffa::acc_fma(Q0, rows[row_off(l, r, R) + jc], xcur[r + l * R - k - 1]);
                ffa::acc_merge(Q0, Q1);
                (g ? pcol1 : pbuf)[c] = ffa::acc_value(Q0);
            }
        }
        {
            const int s8 = lane & 7;
            for (int base = l0 + warp * 4; base < nloc; base += 4 * kNW) {  // warp-uniform
                const int l = base + (lane >> 3);
                ffa::acc Q0 = ffa::acc_zero(), Q1 = ffa::acc_zero();
                int i = -1;
                if (l < nloc) {
                    i = r + l * R;
                    const ff *row = rows + row_off(l, r, R);
                    int j = k + 1 + s8;
                    for (; j + 8 <= i; j += 16) {
                        ffa::acc_fma(Q0, row[j], xcur[j - k - 1]);
                        ffa::acc_fma(Q1, row[j + 8], xcur[j + 8 - k - 1]);
                    }
                    if (j <= i) ffa::acc_fma(Q0, row[j], xcur[j - k - 1]);
                    ffa::acc_merge(Q0, Q1);
                }
#pragma unroll
                for (int o = 4; o > 0; o >>= 1) {
                    ffa::acc B;
                    B.s = __shfl_xor_sync(0xffffffffu, Q0.s, o);
                    B.c = __shfl_xor_sync(0xffffffffu, Q0.c, o);
                    ffa::acc_merge(Q0, B);
                }
                if (i >= 0 && s8 == 0) pbuf2[i - k - 1] = ffa::acc_value(Q0);
            }
        }
        __syncthreads();
        const ff tau = fsc[0], v0 = fsc[1], htau = fsc[2];
        const bool reflect = tau.hi != 0.0f;
        if (r == 0)
            for (int j = tid; j < m; j += kT) Vh[(long)k * n + j] = j == 0 ? v0 : xcur[j];
        if (reflect) {
            if (k > 0) cluster_wait();  // every CTA has read the previous step's pushes
            // ---- push q_r and this CTA's entries of column k+1 to every CTA, with q_r . v
            ffa::acc D = ffa::acc_zero();
            const ff dv = ffa::sub(v0, xcur[0]);  // v_0 - alpha
            for (int j = 2 * tid; j < m; j += 2 * kT) {  // two entries per 16-byte remote store
                float4 q2;
#pragma unroll
                for (int h = 0; h < 2; h++) {
                    const int jj = j + h, i = jj + k + 1;
                    ff q = ffa::zero();
                    if (jj < m) {
                        q = ffa::add(pbuf[jj], pcol1[jj]);
                        if (i >= r && (i - r) % R == 0)
                            q = ffa::add(q, ffa::add(pbuf2[jj], ffa::mul(dv, rows[row_off((i - r) / R, r, R) + k + 1])));
                        ffa::acc_fma(D, q, jj == 0 ? v0 : xcur[jj]);
                    }
                    if (h == 0) { q2.x = q.hi; q2.y = q.lo; } else { q2.z = q.hi; q2.w = q.lo; }
                }
                for (int dst = 0; dst < R; dst++)
                    *reinterpret_cast<float4 *>(cl.map_shared_rank(qbuf, dst) + (size_t)r * nq + j) = q2;
            }
            for (int l = l2 + tid; l < nloc; l += kT) {
                const int i = r + l * R;
                const ff c = rows[row_off(l, r, R) + k + 1];
                for (int dst = 0; dst < R; dst++) cl.map_shared_rank(colb, dst)[i - k - 2] = c;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc_down(D, o);
            if (lane == 0) red[warp] = D;
            __syncthreads();
            if (warp == 0) {
                const ff dr = tree16(red);
                if (lane < R) cl.map_shared_rank(dpart, lane)[r] = dr;
            }
            cl.sync();
            // ---- p = tau sum_r q_r ;  p.v = tau sum_r (q_r . v) ;  w = p - (tau/2)(p.v) v
            ffa::acc PV = ffa::acc_zero();
            for (int s2 = 0; s2 < R; s2++) ffa::acc_add(PV, dpart[s2]);
            const ff pv = ffa::mul(tau, ffa::acc_value(PV));
            const ff K = ffa::mul(htau, pv);
            for (int j = tid; j < m; j += kT) {
                ffa::acc P = ffa::acc_zero();
                for (int s2 = 0; s2 < R; s2++) ffa::acc_add(P, qbuf[(size_t)s2 * nq + j]);
                const ff pj = ffa::mul(tau, ffa::acc_value(P));
                wbuf[j] = ffa::sub(pj, ffa::mul(K, j == 0 ? v0 : xcur[j]));
            }
            __syncthreads();
            // ---- the updated column k+1 (all of it, in every CTA) and its squared norm
            ffa::acc SQ = ffa::acc_zero();
            const ff w0 = wbuf[0];
            for (int jn = tid; jn < m - 1; jn += kT) {  // row i = k + 2 + jn, ii = i - k - 1 = jn + 1
                const ff nv = rank2(colb[jn], xcur[jn + 1], w0, wbuf[jn + 1], v0);
                xnext[jn] = nv;
                if (jn >= 1) ffa::acc_fma(SQ, nv, nv);
            }
            cluster_arrive();  // done with qbuf, colb and dpart of this step
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc_down(SQ, o);
            if (lane == 0) wsq[warp] = SQ;
            // ---- rank-2 update of own rows (lower part, from column k+1)
            for (int l = l0 + warp; l < nloc; l += kNW) {
                const int i = r + l * R;
                ff *row = rows + row_off(l, r, R);
                const int ii = i - k - 1;
                const ff vi = ii == 0 ? v0 : xcur[ii];
                const ff wi = wbuf[ii];
                for (int j = k + 1 + lane; j <= i; j += 32) {
                    const int jj = j - k - 1;
                    row[j] = rank2(row[j], vi, wbuf[jj], wi, jj == 0 ? v0 : xcur[jj]);
                }
            }
        } else {
            // no reflection: the next column is column k+1 as it stands
            if (k > 0) cluster_wait();
            for (int l = l2 + tid; l < nloc; l += kT) {
                const int i = r + l * R;
                const ff c = rows[row_off(l, r, R) + k + 1];
                for (int dst = 0; dst < R; dst++) cl.map_shared_rank(colb, dst)[i - k - 2] = c;
            }
            cl.sync();
            ffa::acc SQ = ffa::acc_zero();
            for (int jn = tid; jn < m - 1; jn += kT) {
                xnext[jn] = colb[jn];
                if (jn >= 1) ffa::acc_fma(SQ, colb[jn], colb[jn]);
            }
            cluster_arrive();
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc_down(SQ, o);
            if (lane == 0) wsq[warp] = SQ;
        }
        __syncthreads();
        sig = tree16(wsq);  // squared norm of the next column's x[1..], the same in every thread
        ff *t = xcur;
        xcur = xnext;
        xnext = t;
    }
    if (n >= 3) cluster_wait();  // completes the last step's arrive
    __syncthreads();
    if (tid == 0) {
        if (r == 0) {
            ed[n - 1] = ffa::zero();
            tau_g[n - 1] = ffa::zero();
            v0_g[n - 1] = ffa::zero();
            if (n >= 2) { tau_g[n - 2] = ffa::zero(); v0_g[n - 2] = ffa::zero(); }
        }
        if (n >= 3 && (n - 2) % R == r) dg[n - 2] = rows[row_off((n - 2) / R, r, R) + n - 2];
        if (n >= 2 && (n - 1) % R == r) {
            const ff *row = rows + row_off((n - 1) / R, r, R);
            ed[n - 2] = row[n - 2];
            dg[n - 1] = row[n - 1];
        }
    }
    cl.sync();

    // ---------------------------------------------------------------- 2. eigenpairs of T
    ff *dgs = rows;  // region 0 reused: T (ff), FP32 Sturm data, then per-warp LU slots
    ff *eds = dgs + n;
    float *dg32 = reinterpret_cast<float *>(eds + n);
    float *e232 = dg32 + n;
    float *redf = e232 + n;  // [2 * kNW]
    ff *slots = reinterpret_cast<ff *>(redf + 2 * kNW + 2);
    const size_t slot_ff = (size_t)5 * n + (n + 7) / 8;  // u0i, u1, u2, lm, z  + piv bytes
    for (int i = tid; i < n; i += kT) {
        dgs[i] = dg[i];
        eds[i] = ed[i];
        dg32[i] = dg[i].hi;
        e232[i] = __fmul_rn(ed[i].hi, ed[i].hi);
    }
    __syncthreads();
    float glo = 3e38f, ghi = -3e38f;
    for (int i = tid; i < n; i += kT) {
        const float rr = (i > 0 ? fabsf(eds[i - 1].hi) : 0.0f) + (i < n - 1 ? fabsf(eds[i].hi) : 0.0f);
        glo = fminf(glo, dgs[i].hi - rr);
        ghi = fmaxf(ghi, dgs[i].hi + rr);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        glo = fminf(glo, __shfl_xor_sync(0xffffffffu, glo, o));
        ghi = fmaxf(ghi, __shfl_xor_sync(0xffffffffu, ghi, o));
    }
    if (lane == 0) { redf[warp] = glo; redf[kNW + warp] = ghi; }
    __syncthreads();
    glo = redf[0];
    ghi = redf[kNW];
    for (int w = 1; w < kNW; w++) { glo = fminf(glo, redf[w]); ghi = fmaxf(ghi, redf[kNW + w]); }
    const float tnorm = fmaxf(fabsf(glo), fabsf(ghi)) + 1e-30f;
    ff *Zm = a.Z + (long)mat * d * n;
    // my eigenvalue indices: t = r + (warp + kNW * round) * R, one per warp per round
    const int per_cta = d > r ? (d - r + R - 1) / R : 0;
    for (int base = 0; base < per_cta; base += a.nslots) {
        const int j = base + warp;
        if (warp < a.nslots && j < per_cta) {
            const int t = r + j * R;
            const int target = n - 1 - t;
            const float span = ghi - glo;
            float lo = glo - 1e-3f * span - 1e-30f, hi = ghi + 1e-3f * span + 1e-30f;
            for (int round = 0; round < 12; round++) {
                const float x = lo + (hi - lo) * (float)(lane + 1) / 33.0f;
                const int c = sturm_count(dg32, e232, n, x);
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
                if (hi - lo <= 4.0f * 1.2e-7f * fmaxf(fabsf(lo), fabsf(hi)) + 1e-30f) break;
            }
            if (lane == 0) {
                const ff sigma = ffa::two_sum(0.5f * lo, 0.5f * hi);
                a.sig[(long)mat * d + t] = sigma.hi;
                ff *sl = slots + (size_t)warp * slot_ff;
                ff *u0i = sl, *u1 = sl + n, *u2 = sl + 2 * n, *lm = sl + 3 * n, *z = sl + 4 * n;
                uint8_t *pv = reinterpret_cast<uint8_t *>(sl + 5 * n);
                tri_factor(dgs, eds, n, sigma, ffa::make(3.6e-15f * tnorm, 0.0f), u0i, u1, u2, lm, pv);
                // deterministic start vector from an integer hash
                for (int i = 0; i < n; i++) {
                    unsigned h = (unsigned)(i + 1) * 2654435761u ^ (unsigned)(t + 1) * 40503u;
                    h ^= h >> 15;
                    h *= 2246822519u;
                    h ^= h >> 13;
                    z[i] = ffa::make(1.0f + 0.5f * ((float)(h & 0xffffu) / 65536.0f - 0.5f), 0.0f);
                }
                for (int it = 0; it < 3; it++) {
                    tri_solve(n, u0i, u1, u2, lm, pv, z);
                    ffa::acc N2 = ffa::acc_zero();
                    for (int i = 0; i < n; i++) ffa::acc_fma(N2, z[i], z[i]);
                    const ff inv = ffa::div(ffa::make(1.0f, 0.0f), ffa::sqrt(ffa::acc_value(N2)));
                    for (int i = 0; i < n; i++) z[i] = ffa::mul(z[i], inv);
                }
                ff *zg = Zm + (long)t * n;
                for (int i = 0; i < n; i++) zg[i] = z[i];
            }
        }
        __syncthreads();
    }
    cl.sync();
    if (r == 0) {
        const float *sg = a.sig + (long)mat * d;
        for (int t = 1; t < d; t++) {
            ff *zt = Zm + (long)t * n;
            bool any = false;
            for (int s2 = 0; s2 < t; s2++) {
                if (fabsf(sg[s2] - sg[t]) >= 1e-3f * tnorm) continue;
                const ff *zs = Zm + (long)s2 * n;
                ffa::acc P = ffa::acc_zero();
                for (int i = tid; i < n; i += kT) ffa::acc_fma(P, zs[i], zt[i]);
                const ff c = block_acc(P, red);
                for (int i = tid; i < n; i += kT) zt[i] = ffa::sub(zt[i], ffa::mul(c, zs[i]));
                __syncthreads();
                any = true;
            }
            if (any) {
                ffa::acc P = ffa::acc_zero();
                for (int i = tid; i < n; i += kT) ffa::acc_fma(P, zt[i], zt[i]);
                const ff inv = ffa::div(ffa::make(1.0f, 0.0f), ffa::sqrt(block_acc(P, red)));
                for (int i = tid; i < n; i += kT) zt[i] = ffa::mul(zt[i], inv);
                __syncthreads();
            }
        }
        ff *lam = a.lam + (long)mat * d;
        int *order = a.order + (long)mat * d;
        if (tid < d) {
            const ff *z = Zm + (long)tid * n;
            ffa::acc Q = ffa::acc_zero();
            for (int i = 0; i < n; i++) {
                ffa::acc T = ffa::acc_zero();
                ffa::acc_fma(T, dgs[i], z[i]);
                if (i > 0) ffa::acc_fma(T, eds[i - 1], z[i - 1]);
                if (i < n - 1) ffa::acc_fma(T, eds[i], z[i + 1]);
                ffa::acc_fma(Q, z[i], ffa::acc_value(T));
            }
            lam[tid] = ffa::acc_value(Q);
        }
        __syncthreads();
        if (tid == 0) {
            for (int t = 0; t < d; t++) order[t] = t;
            for (int x = 1; x < d; x++) {
                const int v = order[x];
                int y = x - 1;
                while (y >= 0 && ffa::less(lam[order[y]], lam[v])) { order[y + 1] = order[y]; y--; }
                order[y + 1] = v;
            }
            for (int t = 0; t < d; t++) a.eig[(long)mat * d + t] = ffa::to_double(lam[order[t]]);
        }
    }
    cl.sync();

    // ---------------------------------------------------------------- 3. back-transformation (ff)
    const int ncol = d > r ? (d - r + R - 1) / R : 0;
    const int *order = a.order + (long)mat * d;
    ff *Wo = rows;  // [n][ncol], region 0 reused
    ff *vk = qbuf;  // [n]
    ff *coef = pbuf;
    for (int e = tid; e < n * ncol; e += kT) {
        const int i = e / ncol, c = e % ncol;
        Wo[e] = Zm[(long)order[r + c * R] * n + i];
    }
    __syncthreads();
    for (int k = n - 3; k >= 0; k--) {
        const ff tk = tau_g[k];
        if (tk.hi == 0.0f) continue;
        const int m = n - k - 1;
        for (int i = tid; i < m; i += kT) vk[i] = Vh[(long)k * n + i];
        __syncthreads();
        for (int c = warp; c < ncol; c += kNW) {
            ffa::acc Q = ffa::acc_zero();
            for (int i = lane; i < m; i += 32) ffa::acc_fma(Q, vk[i], Wo[(size_t)(k + 1 + i) * ncol + c]);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc_down(Q, o);
            if (lane == 0) coef[c] = ffa::mul(tk, ffa::acc_value(Q));
        }
        __syncthreads();
        for (int e = tid; e < m * ncol; e += kT) {
            const int i = e / ncol, c = e % ncol;
            ff &w = Wo[(size_t)(k + 1 + i) * ncol + c];
            w = ffa::sub(w, ffa::mul(coef[c], vk[i]));
        }
        __syncthreads();
    }
    // sign: largest-magnitude entry positive (first on ties)
    double *sgn = reinterpret_cast<double *>(wbuf);
    for (int c = warp; c < ncol; c += kNW) {
        float best = -1.0f;
        int bi = 0x7fffffff;
        for (int i = lane; i < n; i += 32) {
            const float v = fabsf(Wo[(size_t)i * ncol + c].hi);
            if (v > best) { best = v; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const float ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (lane == 0) sgn[c] = Wo[(size_t)bi * ncol + c].hi < 0.0f ? -1.0 : 1.0;
    }
    __syncthreads();
    double *V = a.V + (long)mat * n * d;
    for (int e = tid; e < n * ncol; e += kT) {
        const int i = e / ncol, c = e % ncol;
        V[(long)i * d + (r + c * R)] = sgn[c] * ffa::to_double(Wo[e]);
    }
    cl.sync();  // no CTA leaves while others may still write into its shared memory
}

// Shared-memory plan of one CTA for cluster size R: region 0 holds the packed
// rows (phase 1), then T and the per-warp inverse-iteration slots (phase 2),
// then the CTA's columns of the eigenvectors (phase 3).
size_t smem_plan(int n, int d, int R, long *region0, int *nslots) {
    const long rows = rows_elems(n, R);
    const int ncol = (d + R - 1) / R;
    const long t_part = 2L * n + (long)((2 * sizeof(float) * n + 2 * sizeof(float) * kNW + 8 + 7) / sizeof(ff));
    const long slot = 5L * n + (n + 7) / 8;
    const int per_cta = ncol;
    int ns = kNW < per_cta ? kNW : per_cta;
    if (ns < 1) ns = 1;
    long reg = rows;
    // as many slots as fit in the packed-row region, at least one
    while (ns > 1 && t_part + ns * slot > reg) ns--;
    if (t_part + ns * slot > reg) reg = t_part + ns * slot;
    if ((long)n * ncol > reg) reg = (long)n * ncol;
    reg = (reg + 1) & ~1L;  // qbuf starts on a 16-byte boundary
    *region0 = reg;
    *nslots = ns;
    return sizeof(ff) * ((size_t)reg + (size_t)R * ((n + 1) & ~1) + 7 * (size_t)n) + 2 * sizeof(ffa::acc) * kNW +
           sizeof(ff) * (4 + 8);
}

// Cluster size: the smallest power of two R whose shared-memory plan fits,
// raised for small batches (a matrix's reduction is latency-bound, so idle SMs
// are better spent on fewer rows per CTA): aim for about half of the SMs across
// the batch.  Where that gives 8 (C = 512), six CTAs are used when their plan
// fits the opt-in maximum: every step's exchange grows with R, so a matrix
// takes less time on six (6.2 against 11.0 ms for 16 matrices of 512), and 25
// clusters of six fit on 152 SMs against 19 of eight.
int pick_R(int n, int d, int mats, int n_sm) {
    int R = 0;
    for (int r = 2; r <= 8; r *= 2) {
        long reg;
        int ns;
        if (smem_plan(n, d, r, &reg, &ns) <= kSmemMax) { R = r; break; }
    }
    if (R == 0) return 0;
    const bool raised = R < 8 && 2 * R * mats <= n_sm / 2;
    while (R < 8 && 2 * R * mats <= n_sm / 2) R *= 2;
    if (R == 8 && !raised) {
        long reg;
        int ns;
        if (smem_plan(n, d, 6, &reg, &ns) <= kSmemOptIn) R = 6;
    }
    return R;
}

}  // namespace

struct EigPlan {
    size_t e32, flags, dg, ed, tau, v0, Vh, Z, sig, lam, order, total;
};

static EigPlan eig_plan(int n, int d, int mats) {
    EigPlan p{};
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = align_up(o + bytes, 256);
        return at;
    };
    p.e32 = take(eig32_ok(n, d) ? eig32_workspace_bytes(n, mats) : 0);
    p.flags = take(sizeof(int) * (size_t)mats);
    p.dg = take(sizeof(ff) * (size_t)mats * n);
    p.ed = take(sizeof(ff) * (size_t)mats * n);
    p.tau = take(sizeof(ff) * (size_t)mats * n);
    p.v0 = take(sizeof(ff) * (size_t)mats * n);
    p.Vh = take(sizeof(ff) * (size_t)mats * n * n);
    p.Z = take(sizeof(ff) * (size_t)mats * d * n);
    p.sig = take(sizeof(float) * (size_t)mats * d);
    p.lam = take(sizeof(ff) * (size_t)mats * d);
    p.order = take(sizeof(int) * (size_t)mats * d);
    p.total = o;
    return p;
}

size_t eig_workspace_bytes(int n, int d, int mats) { return eig_plan(n, d, mats).total; }

// cov_ff: [mats][n][n] float-float pairs (hi, lo) of the covariance.
cudaError_t launch_eig(const void *cov_ff, int n, int d, int mats, double *V, double *eigvals, void *ws,
                       int *status, cudaStream_t st, float tol) {
    const EigPlan p = eig_plan(n, d, mats);
    char *b = (char *)ws;
    const int *redo = nullptr;
    if (eig32_ok(n, d)) {
        int *flags = (int *)(b + p.flags);
        cudaError_t e = launch_eig32(cov_ff, n, d, mats, V, eigvals, b + p.e32, flags,
                                     status ? status + kRedoCountSlot : nullptr, tol, st);
        if (e != cudaSuccess) return e;
        redo = flags;
    }
    int dev = 0, n_sm = 0;
    cudaError_t eq = cudaGetDevice(&dev);
    if (eq == cudaSuccess) eq = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (eq != cudaSuccess) return eq;
    const int R = pick_R(n, d, mats, n_sm);
    if (R == 0) return cudaErrorNotSupported;
    long region0 = 0;
    int nslots = 1;
    const size_t smem = smem_plan(n, d, R, &region0, &nslots);
    static DeviceOnce attrs;
    cudaError_t e0 = device_once(attrs, dev, [] {
        return cudaFuncSetAttribute(k_eig_ff, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    });
    if (e0 != cudaSuccess) return e0;
    EigArgs a;
    a.redo = redo;
    a.cov = (const ff *)cov_ff;
    a.n = n;
    a.d = d;
    a.R = R;
    a.region0 = region0;
    a.nslots = nslots;
    a.dg = (ff *)(b + p.dg);
    a.ed = (ff *)(b + p.ed);
    a.tau = (ff *)(b + p.tau);
    a.v0 = (ff *)(b + p.v0);
    a.Vh = (ff *)(b + p.Vh);
    a.Z = (ff *)(b + p.Z);
    a.sig = (float *)(b + p.sig);
    a.lam = (ff *)(b + p.lam);
    a.order = (int *)(b + p.order);
    a.V = V;
    a.eig = eigvals;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(R * mats);
    cfg.blockDim = dim3(kT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = R;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaSuccess;
    QFCA_LAUNCH("k_eig_ff", st, e = cudaLaunchKernelEx(&cfg, k_eig_ff, a));
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace qfca
