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
//      of step k-1) and forms (v, tau) (scalars in FP64 by one thread); each
//      CTA computes its partial q of A v from the elements it stores (row part
//      and column part of the symmetric product) and pushes it into every
//      CTA; cluster barrier; p = tau sum_r q_r (fixed order),
//      w = p - (tau/2)(p.v) v; each CTA applies A -= v w^T + w v^T to its
//      lower-triangle rows and pushes the new column k+1 into every CTA;
//      cluster barrier.
//   2. Shifts by warp multisection on the FP32 Sturm count; FP64 inverse
//      iteration on T (LU with partial pivoting, three solves); selective
//      Gram-Schmidt for shifts within 1e-3 ||T||; FP64 Rayleigh quotients;
//      stable descending order.
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

struct EigArgs {
    const ff *cov;  // [mats][n][n] float-float covariance
    int n, d, R;
    long region0;   // ff elements of the first shared region (packed rows; reused by phases 2/3)
    double *dg, *ed, *tau, *v0;  // [mats][n]
    ff *Vh;                      // [mats][n][n]  Householder vectors (row k: v_k, length n-k-1)
    double *Z;                   // [mats][d][n]
    double *lu;                  // [mats][d][5][n]
    uint8_t *piv;                // [mats][d][n]
    float *sig;                  // [mats][d]
    double *lam;                 // [mats][d]
    int *order;                  // [mats][d]
    double *V;                   // [mats][n][d]
    double *eig;                 // [mats][d]
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

__device__ __forceinline__ void acc_down(ffa::acc &A, int o) {
    ffa::acc B;
    B.s = __shfl_down_sync(0xffffffffu, A.s, o);
    B.c = __shfl_down_sync(0xffffffffu, A.c, o);
    ffa::acc_merge(A, B);
}

// Deterministic block reduction; every thread gets the same value.
__device__ ff block_acc(ffa::acc A, ffa::acc *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc_down(A, o);
    __syncthreads();
    if (lane == 0) red[warp] = A;
    __syncthreads();
    ffa::acc T = red[0];
    for (int w = 1; w < kNW; w++) ffa::acc_merge(T, red[w]);
    __syncthreads();
    return ffa::acc_value(T);
}

__device__ double block_sum_d(double v, double *redd) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) redd[warp] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < kNW; w++) t += redd[w];
    __syncthreads();
    return t;
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

// LU with partial pivoting of the tridiagonal T - sigma I (FP64); u0i: reciprocal pivots.
__device__ void tri_factor(const double *dg, const double *ed, int n, double sigma, double tiny, double *u0i,
                           double *u1, double *u2, double *lm, uint8_t *piv) {
    double r0 = dg[0] - sigma, r1 = n > 1 ? ed[0] : 0.0;
    for (int i = 0; i < n - 1; i++) {
        const double s0 = ed[i], s1 = dg[i + 1] - sigma, s2 = (i + 1 < n - 1) ? ed[i + 1] : 0.0;
        if (fabs(r0) >= fabs(s0)) {
            if (r0 == 0.0) r0 = tiny;
            const double inv = 1.0 / r0;
            const double l = s0 * inv;
            u0i[i] = inv; u1[i] = r1; u2[i] = 0.0; lm[i] = l; piv[i] = 0;
            r0 = s1 - l * r1;
            r1 = s2;
        } else {
            const double inv = 1.0 / s0;
            const double l = r0 * inv;
            u0i[i] = inv; u1[i] = s1; u2[i] = s2; lm[i] = l; piv[i] = 1;
            const double n0 = r1 - l * s1, n1 = -l * s2;
            r0 = n0; r1 = n1;
        }
    }
    if (r0 == 0.0) r0 = tiny;
    u0i[n - 1] = 1.0 / r0; u1[n - 1] = 0.0; u2[n - 1] = 0.0;
}

__device__ void tri_solve(int n, const double *u0i, const double *u1, const double *u2, const double *lm,
                          const uint8_t *piv, double *x) {
    for (int i = 0; i < n - 1; i++) {
        if (piv[i]) { const double t = x[i]; x[i] = x[i + 1]; x[i + 1] = t; }
        x[i + 1] -= lm[i] * x[i];
    }
    x[n - 1] *= u0i[n - 1];
    if (n >= 2) x[n - 2] = (x[n - 2] - u1[n - 2] * x[n - 1]) * u0i[n - 2];
    for (int i = n - 3; i >= 0; i--) x[i] = (x[i] - u1[i] * x[i + 1] - u2[i] * x[i + 2]) * u0i[i];
}

__global__ void __launch_bounds__(kT, 1) k_eig_ff(EigArgs a) {
    cg::cluster_group cl = cg::this_cluster();
    const int R = a.R;
    const int r = (int)cl.block_rank();
    const int mat = blockIdx.x / R;
    const int n = a.n, d = a.d;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nloc = r < n ? (n - r + R - 1) / R : 0;  // own rows i = r + l R

    extern __shared__ __align__(16) unsigned char smraw[];
    ff *rows = reinterpret_cast<ff *>(smraw);        // region 0
    ff *qbuf = rows + a.region0;                     // [R][n] partial products pushed by every CTA
    ff *xa = qbuf + (size_t)R * n;                   // [n] current column (x)
    ff *xb = xa + n;                                 // [n] next column
    ff *pbuf = xb + n;                               // [n]
    ff *wbuf = pbuf + n;                             // [n]
    ffa::acc *red = reinterpret_cast<ffa::acc *>(wbuf + n);  // [kNW]
    ff *fsc = reinterpret_cast<ff *>(red + kNW);             // [4] step scalars in ff
    double *scal = reinterpret_cast<double *>(fsc + 4);      // [4]

    const ff *S = a.cov + (long)mat * n * n;
    double *dg = a.dg + (long)mat * n, *ed = a.ed + (long)mat * n;
    double *tau_g = a.tau + (long)mat * n, *v0_g = a.v0 + (long)mat * n;
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
            dg[0] = ffa::to_double(rows[0]);
        }
    }
    cl.sync();

    ff *xcur = xa, *xnext = xb;
    // ---------------------------------------------------------------- 1. tridiagonalisation
    for (int k = 0; k + 2 < n; k++) {
        const int m = n - k - 1;
        ffa::acc A = ffa::acc_zero();
        for (int j = 1 + tid; j < m; j += kT) ffa::acc_fma(A, xcur[j], xcur[j]);
        const ff sig = block_acc(A, red);  // identical in every CTA of the cluster
        if (tid == 0) {
            const double alpha = ffa::to_double(xcur[0]);
            const double sigma = ffa::to_double(sig);
            double tau = 0.0, ek = alpha, v0 = alpha;
            if (sigma > 0.0) {
                const double mu = sqrt(alpha * alpha + sigma);
                v0 = alpha >= 0.0 ? alpha + mu : alpha - mu;
                ek = alpha >= 0.0 ? -mu : mu;
                tau = 2.0 / (v0 * v0 + sigma);
            }
            scal[0] = tau;
            fsc[0] = ffa::from_double(tau);
            fsc[1] = ffa::from_double(v0);
            fsc[2] = ffa::from_double(0.5 * tau);
            if (r == 0) { tau_g[k] = tau; v0_g[k] = v0; ed[k] = ek; }
        }
        __syncthreads();
        const double tau_d = scal[0];
        const ff tau = fsc[0], v0 = fsc[1], htau = fsc[2];
        if (r == 0)
            for (int j = tid; j < m; j += kT) Vh[(long)k * n + j] = j == 0 ? v0 : xcur[j];
        int l0 = (k + 1 - r + R - 1) / R;  // first own row with i >= k+1
        if (l0 < 0) l0 = 0;
        if (tau_d != 0.0) {
            // ---- column part of the own partial product: sum over own rows i > jc of A[i][jc] v_i
            for (int jc = k + 1 + tid; jc < n; jc += kT) {
                ffa::acc Q = ffa::acc_zero();
                int lc = (jc + 1 - r + R - 1) / R;
                if (lc < 0) lc = 0;
                for (int l = lc; l < nloc; l++) {
                    const int i = r + l * R;  // i >= jc + 1 >= k + 2: v_i = x_{i-k-1}
                    ffa::acc_fma(Q, rows[row_off(l, r, R) + jc], xcur[i - k - 1]);
                }
                pbuf[jc - k - 1] = ffa::acc_value(Q);
            }
            __syncthreads();
            // ---- plus the row part for own rows i >= k+1: sum_{j=k+1..i} A[i][j] v_j
            for (int l = l0 + warp; l < nloc; l += kNW) {
                const int i = r + l * R;
                const ff *row = rows + row_off(l, r, R);
                ffa::acc Q = ffa::acc_zero();
                for (int j = k + 1 + lane; j <= i; j += 32) ffa::acc_fma(Q, row[j], j == k + 1 ? v0 : xcur[j - k - 1]);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc_down(Q, o);
                if (lane == 0) {
                    ffa::acc_add(Q, pbuf[i - k - 1]);
                    pbuf[i - k - 1] = ffa::acc_value(Q);
                }
            }
            __syncthreads();
            for (int j = tid; j < m; j += kT) {
                const ff q = pbuf[j];
                for (int dst = 0; dst < R; dst++) cl.map_shared_rank(qbuf, dst)[(size_t)r * n + j] = q;
            }
            cl.sync();
            // ---- p = tau sum_r q_r ; w = p - (tau/2)(p.v) v
            ffa::acc PV = ffa::acc_zero();
            for (int j = tid; j < m; j += kT) {
                ffa::acc P = ffa::acc_zero();
                for (int s = 0; s < R; s++) ffa::acc_add(P, qbuf[(size_t)s * n + j]);
                const ff p = ffa::mul(tau, ffa::acc_value(P));
                pbuf[j] = p;
                ffa::acc_fma(PV, p, j == 0 ? v0 : xcur[j]);
            }
            const ff pv = block_acc(PV, red);
            const ff K = ffa::mul(htau, pv);
            for (int j = tid; j < m; j += kT) wbuf[j] = ffa::sub(pbuf[j], ffa::mul(K, j == 0 ? v0 : xcur[j]));
            __syncthreads();
            // ---- rank-2 update of own rows (lower part); push the new column k+1
            for (int l = l0 + warp; l < nloc; l += kNW) {
                const int i = r + l * R;
                ff *row = rows + row_off(l, r, R);
                const int ii = i - k - 1;
                const ff vi = ii == 0 ? v0 : xcur[ii];
                const ff wi = wbuf[ii];
                for (int j = k + 1 + lane; j <= i; j += 32) {
                    const int jj = j - k - 1;
                    const ff t = ffa::add(ffa::mul(vi, wbuf[jj]), ffa::mul(wi, jj == 0 ? v0 : xcur[jj]));
                    const ff nv = ffa::sub(row[j], t);
                    row[j] = nv;
                    if (jj == 0 && i >= k + 2)
                        for (int dst = 0; dst < R; dst++) cl.map_shared_rank(xnext, dst)[i - k - 2] = nv;
                }
            }
        } else {
            // no reflection: only gather the next column
            int lg = (k + 2 - r + R - 1) / R;
            if (lg < 0) lg = 0;
            for (int l = lg + tid; l < nloc; l += kT) {
                const int i = r + l * R;
                const ff nv = rows[row_off(l, r, R) + k + 1];
                for (int dst = 0; dst < R; dst++) cl.map_shared_rank(xnext, dst)[i - k - 2] = nv;
            }
        }
        __syncthreads();
        if (tid == 0 && (k + 1) % R == r) dg[k + 1] = ffa::to_double(rows[row_off((k + 1) / R, r, R) + k + 1]);
        cl.sync();
        ff *t = xcur;
        xcur = xnext;
        xnext = t;
    }
    if (tid == 0) {
        if (r == 0) {
            ed[n - 1] = 0.0;
            tau_g[n - 1] = 0.0;
            v0_g[n - 1] = 0.0;
            if (n >= 2) { tau_g[n - 2] = 0.0; v0_g[n - 2] = 0.0; }
        }
        if (n >= 2 && (n - 1) % R == r) {
            const ff *row = rows + row_off((n - 1) / R, r, R);
            ed[n - 2] = ffa::to_double(row[n - 2]);
            dg[n - 1] = ffa::to_double(row[n - 1]);
        }
    }
    cl.sync();

    // ---------------------------------------------------------------- 2. eigenpairs of T
    double *dgs = reinterpret_cast<double *>(rows);  // region 0 reused
    double *eds = dgs + n;
    double *redd = eds + n;                           // [2 * kNW]
    float *dg32 = reinterpret_cast<float *>(redd + 2 * kNW);
    float *e232 = dg32 + n;
    for (int i = tid; i < n; i += kT) {
        dgs[i] = dg[i];
        eds[i] = ed[i];
        dg32[i] = (float)dg[i];
        e232[i] = (float)(ed[i] * ed[i]);
    }
    __syncthreads();
    double glo = 1e300, ghi = -1e300;
    for (int i = tid; i < n; i += kT) {
        const double rr = (i > 0 ? fabs(eds[i - 1]) : 0.0) + (i < n - 1 ? fabs(eds[i]) : 0.0);
        glo = fmin(glo, dgs[i] - rr);
        ghi = fmax(ghi, dgs[i] + rr);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        glo = fmin(glo, __shfl_xor_sync(0xffffffffu, glo, o));
        ghi = fmax(ghi, __shfl_xor_sync(0xffffffffu, ghi, o));
    }
    if (lane == 0) { redd[warp] = glo; redd[kNW + warp] = ghi; }
    __syncthreads();
    glo = redd[0];
    ghi = redd[kNW];
    for (int w = 1; w < kNW; w++) { glo = fmin(glo, redd[w]); ghi = fmax(ghi, redd[kNW + w]); }
    __syncthreads();
    const double tnorm = fmax(fabs(glo), fabs(ghi)) + 1e-300;
    double *Zm = a.Z + (long)mat * d * n;
    for (int t = r + warp * R; t < d; t += kNW * R) {
        const int target = n - 1 - t;
        const float span = (float)(ghi - glo);
        float lo = (float)glo - 1e-3f * span - 1e-30f, hi = (float)ghi + 1e-3f * span + 1e-30f;
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
            const double sigma = 0.5 * ((double)lo + (double)hi);
            a.sig[(long)mat * d + t] = (float)sigma;
            double *lu = a.lu + ((long)mat * d + t) * 5 * n;
            uint8_t *pv = a.piv + ((long)mat * d + t) * n;
            tri_factor(dgs, eds, n, sigma, 2.2e-16 * tnorm, lu, lu + n, lu + 2 * n, lu + 3 * n, pv);
            double *z = Zm + (long)t * n;
            for (int i = 0; i < n; i++) z[i] = 1.0 + 0.5 * sin(0.7 * (double)(i + 1) + 1.3 * (double)(t + 1));
            for (int it = 0; it < 3; it++) {
                tri_solve(n, lu, lu + n, lu + 2 * n, lu + 3 * n, pv, z);
                double nrm = 0.0;
                for (int i = 0; i < n; i++) nrm = fma(z[i], z[i], nrm);
                nrm = 1.0 / sqrt(nrm);
                for (int i = 0; i < n; i++) z[i] *= nrm;
            }
        }
    }
    cl.sync();
    if (r == 0) {
        const float *sg = a.sig + (long)mat * d;
        for (int t = 1; t < d; t++) {
            double *zt = Zm + (long)t * n;
            bool any = false;
            for (int s = 0; s < t; s++) {
                if (fabs((double)sg[s] - (double)sg[t]) >= 1e-3 * tnorm) continue;
                const double *zs = Zm + (long)s * n;
                double part = 0.0;
                for (int i = tid; i < n; i += kT) part += zs[i] * zt[i];
                const double c = block_sum_d(part, redd);
                for (int i = tid; i < n; i += kT) zt[i] -= c * zs[i];
                __syncthreads();
                any = true;
            }
            if (any) {
                double part = 0.0;
                for (int i = tid; i < n; i += kT) part += zt[i] * zt[i];
                const double inv = 1.0 / sqrt(block_sum_d(part, redd));
                for (int i = tid; i < n; i += kT) zt[i] *= inv;
                __syncthreads();
            }
        }
        double *lam = a.lam + (long)mat * d;
        int *order = a.order + (long)mat * d;
        if (tid < d) {
            const double *z = Zm + (long)tid * n;
            double acc = 0.0;
            for (int i = 0; i < n; i++) {
                double tz = dgs[i] * z[i];
                if (i > 0) tz += eds[i - 1] * z[i - 1];
                if (i < n - 1) tz += eds[i] * z[i + 1];
                acc = fma(z[i], tz, acc);
            }
            lam[tid] = acc;
        }
        __syncthreads();
        if (tid == 0) {
            for (int t = 0; t < d; t++) order[t] = t;
            for (int x = 1; x < d; x++) {
                const int v = order[x];
                int y = x - 1;
                while (y >= 0 && lam[order[y]] < lam[v]) { order[y + 1] = order[y]; y--; }
                order[y + 1] = v;
            }
            for (int t = 0; t < d; t++) a.eig[(long)mat * d + t] = lam[order[t]];
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
        Wo[e] = ffa::from_double(Zm[(long)order[r + c * R] * n + i]);
    }
    __syncthreads();
    for (int k = n - 3; k >= 0; k--) {
        const double td = tau_g[k];
        if (td == 0.0) continue;
        const int m = n - k - 1;
        if (tid == 0) fsc[3] = ffa::from_double(td);
        for (int i = tid; i < m; i += kT) vk[i] = Vh[(long)k * n + i];
        __syncthreads();
        const ff tk = fsc[3];
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

// Shared-memory plan of one CTA for cluster size R.
size_t smem_plan(int n, int d, int R, long *region0) {
    long reg = rows_elems(n, R);
    const int ncol = (d + R - 1) / R;
    const long p2 = (long)((2 * sizeof(double) * n + 2 * sizeof(double) * kNW + 2 * sizeof(float) * n + 7) / sizeof(ff));
    const long p3 = (long)n * ncol;
    if (p2 > reg) reg = p2;
    if (p3 > reg) reg = p3;
    *region0 = reg;
    return sizeof(ff) * ((size_t)reg + (size_t)R * n + 4 * (size_t)n) + sizeof(ffa::acc) * kNW + sizeof(ff) * 4 +
           sizeof(double) * 4;
}

int pick_R(int n, int d) {
    for (int R = 2; R <= 8; R *= 2) {
        long reg;
        if (smem_plan(n, d, R, &reg) <= kSmemMax) return R;
    }
    return 0;
}

}  // namespace

struct EigPlan {
    size_t dg, ed, tau, v0, Vh, Z, lu, piv, sig, lam, order, total;
};

static EigPlan eig_plan(int n, int d, int mats) {
    EigPlan p{};
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = align_up(o + bytes, 256);
        return at;
    };
    p.dg = take(sizeof(double) * (size_t)mats * n);
    p.ed = take(sizeof(double) * (size_t)mats * n);
    p.tau = take(sizeof(double) * (size_t)mats * n);
    p.v0 = take(sizeof(double) * (size_t)mats * n);
    p.Vh = take(sizeof(ff) * (size_t)mats * n * n);
    p.Z = take(sizeof(double) * (size_t)mats * d * n);
    p.lu = take(sizeof(double) * (size_t)mats * d * 5 * n);
    p.piv = take((size_t)mats * d * n);
    p.sig = take(sizeof(float) * (size_t)mats * d);
    p.lam = take(sizeof(double) * (size_t)mats * d);
    p.order = take(sizeof(int) * (size_t)mats * d);
    p.total = o;
    return p;
}

size_t eig_workspace_bytes(int n, int d, int mats) { return eig_plan(n, d, mats).total; }

// cov_ff: [mats][n][n] float-float pairs (hi, lo) of the covariance.
cudaError_t launch_eig(const void *cov_ff, int n, int d, int mats, double *V, double *eigvals, void *ws,
                       cudaStream_t st) {
    const int R = pick_R(n, d);
    if (R == 0) return cudaErrorNotSupported;
    long region0 = 0;
    const size_t smem = smem_plan(n, d, R, &region0);
    static int attr_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (attr_dev != dev) {
        cudaError_t e = cudaFuncSetAttribute(k_eig_ff, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        if (e != cudaSuccess) return e;
        attr_dev = dev;
    }
    const EigPlan p = eig_plan(n, d, mats);
    char *b = (char *)ws;
    EigArgs a;
    a.cov = (const ff *)cov_ff;
    a.n = n;
    a.d = d;
    a.R = R;
    a.region0 = region0;
    a.dg = (double *)(b + p.dg);
    a.ed = (double *)(b + p.ed);
    a.tau = (double *)(b + p.tau);
    a.v0 = (double *)(b + p.v0);
    a.Vh = (ff *)(b + p.Vh);
    a.Z = (double *)(b + p.Z);
    a.lu = (double *)(b + p.lu);
    a.piv = (uint8_t *)(b + p.piv);
    a.sig = (float *)(b + p.sig);
    a.lam = (double *)(b + p.lam);
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
