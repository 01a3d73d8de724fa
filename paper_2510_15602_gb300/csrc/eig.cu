// eig.cu -- top-d eigenpairs of a symmetric C x C covariance in FP64 (the
// eigendecomposition of the single-image PCA fit, arXiv 2510.15602, Sec. 3.3).
//
// One thread-block cluster of kR = 8 CTAs per matrix (GB300's FP64 pipe is
// ~2 DFMA/clk/SM, so one matrix is spread over 8 SMs):
//   1. Householder tridiagonalisation A = Q T Q^T.  Row i of the trailing
//      matrix lives in CTA (i mod 8) -- in shared memory when it fits, else in
//      global memory.  Step k: every CTA reads row k (= column k) from its
//      owner through distributed shared memory and forms the reflector
//      (v, tau) redundantly; each CTA computes p = tau A v for its own rows
//      and broadcasts them into every CTA's p vector (DSMEM stores); cluster
//      barrier; w = p - (tau/2)(p.v) v; each CTA applies the rank-2 update
//      A -= v w^T + w v^T to its own rows; cluster barrier.
//   2. Shifts: each eigenvalue of T by warp-wide multisection on the FP32
//      Sturm count (33 points per round);  inverse iteration in FP64 on T
//      (LU with partial pivoting, three solves) gives the eigenvector of T;
//      vectors whose shifts lie within 1e-3 ||T|| of each other are
//      re-orthogonalised (Gram-Schmidt); FP64 Rayleigh quotients give the
//      eigenvalues, sorted descending.
//   3. Back-transformation V = H_0 ... H_{n-3} Z, each CTA for its own
//      columns; sign normalisation (largest-magnitude entry positive).
// All waits are cluster barriers (hardware), so no spin loop can hang.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "internal.cuh"

namespace cg = cooperative_groups;

namespace qfca {
namespace {

constexpr int kR = 8;
constexpr int kT = 512;
constexpr int kNW = kT / 32;
constexpr size_t kRowsSmemMax = 150 * 1024;

struct EigArgs {
    const double *cov;  // [mats][n][n]
    int n, d;
    int rows_in_smem;
    double *rows_g;     // [mats][kR][rows_per][n]   (when rows are not in smem)
    double *dg, *ed, *tau, *v0;  // [mats][n]
    double *Z;                   // [mats][d][n]
    double *lu;                  // [mats][d][5][n]
    uint8_t *piv;                // [mats][d][n]
    float *sig;                  // [mats][d]
    double *lam;                 // [mats][d]
    int *order;                  // [mats][d]
    double *V;                   // [mats][n][d]
    double *eig;                 // [mats][d]
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ double block_sum(double v, double *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double t = lane < kNW ? red[lane] : 0.0;
        t = warp_sum(t);
        if (lane == 0) red[0] = t;
    }
    __syncthreads();
    const double t = red[0];
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

// LU factorisation with partial pivoting of the tridiagonal T - sigma I (FP64).
// u0i: reciprocal pivots, u1/u2: first/second super-diagonals of U, lm: multipliers.
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

__global__ void __cluster_dims__(kR, 1, 1) __launch_bounds__(kT, 1) k_eig_cluster(EigArgs a) {
    cg::cluster_group cl = cg::this_cluster();
    const int r = (int)cl.block_rank();
    const int mat = blockIdx.x / kR;
    const int n = a.n, d = a.d;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int rows_per = (n + kR - 1) / kR;
    const int ncol = d > r ? (d - r + kR - 1) / kR : 0;  // own output columns j = r, r+kR, ...

    extern __shared__ __align__(16) double sm[];
    double *rows = a.rows_in_smem ? sm : a.rows_g + ((long)mat * kR + r) * rows_per * n;
    double *vsh = sm + (a.rows_in_smem ? (size_t)rows_per * n : 0);
    double *psh = vsh + n;
    double *wsh = psh + n;
    double *red = wsh + n;
    double *coef = red + 32;
    double *Wo = coef + 64;  // [n][ncol]

    const double *S = a.cov + (long)mat * n * n;
    double *dg = a.dg + (long)mat * n, *ed = a.ed + (long)mat * n;
    double *tau_g = a.tau + (long)mat * n, *v0_g = a.v0 + (long)mat * n;

    // rows of CTA `who` (local row lr): pointer valid cluster-wide
    auto row_of = [&](int who, int lr) -> double * {
        if (a.rows_in_smem) return cl.map_shared_rank(sm, who) + (size_t)lr * n;
        return a.rows_g + (((long)mat * kR + who) * rows_per + lr) * n;
    };

    for (int lr = 0; lr * kR + r < n; lr++)
        for (int j = tid; j < n; j += kT) rows[(size_t)lr * n + j] = S[(long)(lr * kR + r) * n + j];
    cl.sync();

    // ---------------------------------------------------------------- 1. tridiagonalisation
    for (int k = 0; k + 2 < n; k++) {
        const int m = n - k - 1;
        const int owner = k % kR;
        const double *rk = row_of(owner, k / kR);
        double part = 0.0;
        for (int i = tid; i < m; i += kT) {
            const double x = rk[k + 1 + i];
            vsh[i] = x;
            if (i >= 1) part += x * x;
        }
        const double sigma = block_sum(part, red);
        const double alpha = vsh[0];
        double tau = 0.0, ek = alpha, v0 = alpha;
        if (sigma > 0.0) {
            const double mu = sqrt(alpha * alpha + sigma);
            v0 = alpha >= 0.0 ? alpha + mu : alpha - mu;
            ek = alpha >= 0.0 ? -mu : mu;
            tau = 2.0 / (v0 * v0 + sigma);
        }
        __syncthreads();  // every thread has read alpha = vsh[0]
        if (tid == 0) vsh[0] = v0;
        if (r == 0 && tid == 0) { tau_g[k] = tau; v0_g[k] = v0; ed[k] = ek; }
        if (r == owner && tid == 0) dg[k] = rk[k];
        __syncthreads();
        if (tau == 0.0) continue;  // identical in every CTA of the cluster
        // first own row index >= k+1
        const int i0 = (k + 1) + ((r - (k + 1)) % kR + kR) % kR;
        for (int i = i0 + warp * kR; i < n; i += kNW * kR) {
            const double *row = rows + (size_t)(i / kR) * n + (k + 1);
            double acc = 0.0;
            for (int j = lane; j < m; j += 32) acc = fma(row[j], vsh[j], acc);
            acc = warp_sum(acc) * tau;
            if (lane < kR) cl.map_shared_rank(psh, lane)[i - k - 1] = acc;
        }
        cl.sync();
        double pv = 0.0;
        for (int i = tid; i < m; i += kT) pv += psh[i] * vsh[i];
        const double K = 0.5 * tau * block_sum(pv, red);
        for (int i = tid; i < m; i += kT) wsh[i] = psh[i] - K * vsh[i];
        __syncthreads();
        for (int i = i0 + warp * kR; i < n; i += kNW * kR) {
            double *row = rows + (size_t)(i / kR) * n + (k + 1);
            const double vi = vsh[i - k - 1], wi = wsh[i - k - 1];
            for (int j = lane; j < m; j += 32) row[j] = row[j] - vi * wsh[j] - wi * vsh[j];
        }
        cl.sync();
    }
    if (tid == 0) {
        if (n >= 2) {
            if (r == (n - 2) % kR) dg[n - 2] = rows[(size_t)((n - 2) / kR) * n + (n - 2)];
            if (r == (n - 1) % kR) ed[n - 2] = rows[(size_t)((n - 1) / kR) * n + (n - 2)];
            if (r == 0) { tau_g[n - 2] = 0.0; v0_g[n - 2] = 0.0; }
        }
        if (r == (n - 1) % kR) dg[n - 1] = rows[(size_t)((n - 1) / kR) * n + (n - 1)];
        if (r == 0) { ed[n - 1] = 0.0; tau_g[n - 1] = 0.0; v0_g[n - 1] = 0.0; }
    }
    cl.sync();

    // ---------------------------------------------------------------- 2. eigenpairs of T
    float *dg32 = reinterpret_cast<float *>(psh);
    float *e232 = dg32 + n;
    for (int i = tid; i < n; i += kT) {
        dg32[i] = (float)dg[i];
        e232[i] = (float)(ed[i] * ed[i]);
    }
    double glo = 1e300, ghi = -1e300;
    for (int i = tid; i < n; i += kT) {
        const double rr = (i > 0 ? fabs(ed[i - 1]) : 0.0) + (i < n - 1 ? fabs(ed[i]) : 0.0);
        glo = fmin(glo, dg[i] - rr);
        ghi = fmax(ghi, dg[i] + rr);
    }
    // block min / max
    for (int o = 16; o > 0; o >>= 1) {
        glo = fmin(glo, __shfl_xor_sync(0xffffffffu, glo, o));
        ghi = fmax(ghi, __shfl_xor_sync(0xffffffffu, ghi, o));
    }
    __syncthreads();
    if (lane == 0) { red[warp] = glo; coef[warp] = ghi; }
    __syncthreads();
    glo = red[0];
    ghi = coef[0];
    for (int w = 1; w < kNW; w++) { glo = fmin(glo, red[w]); ghi = fmax(ghi, coef[w]); }
    __syncthreads();
    const double tnorm = fmax(fabs(glo), fabs(ghi)) + 1e-300;
    double *Zm = a.Z + (long)mat * d * n;
    for (int t = r + warp * kR; t < d; t += kNW * kR) {
        const int target = n - 1 - t;  // ascending index of the (t+1)-th largest eigenvalue
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
            tri_factor(dg, ed, n, sigma, 2.2e-16 * tnorm, lu, lu + n, lu + 2 * n, lu + 3 * n, pv);
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
    // selective re-orthogonalisation, Rayleigh quotients and ordering (rank 0)
    if (r == 0) {
        const float *sg = a.sig + (long)mat * d;
        for (int t = 1; t < d; t++) {
            double *zt = Zm + (long)t * n;
            bool any = false;
            for (int s = 0; s < t; s++) {
                if (fabs((double)sg[s] - (double)sg[t]) >= 1e-3 * tnorm) continue;
                const double *zs = Zm + (long)s * n;
                double part2 = 0.0;
                for (int i = tid; i < n; i += kT) part2 += zs[i] * zt[i];
                const double c = block_sum(part2, red);
                for (int i = tid; i < n; i += kT) zt[i] -= c * zs[i];
                __syncthreads();
                any = true;
            }
            if (any) {
                double part2 = 0.0;
                for (int i = tid; i < n; i += kT) part2 += zt[i] * zt[i];
                const double inv = 1.0 / sqrt(block_sum(part2, red));
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
                double tz = dg[i] * z[i];
                if (i > 0) tz += ed[i - 1] * z[i - 1];
                if (i < n - 1) tz += ed[i] * z[i + 1];
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

    // ---------------------------------------------------------------- 3. back-transformation of own columns
    const int *order = a.order + (long)mat * d;
    for (int e = tid; e < n * ncol; e += kT) {
        const int i = e / ncol, c = e % ncol;
        Wo[e] = Zm[(long)order[r + c * kR] * n + i];
    }
    __syncthreads();
    for (int k = n - 3; k >= 0; k--) {
        const double tau = tau_g[k];
        if (tau == 0.0) continue;
        const int m = n - k - 1;
        const double *rk = row_of(k % kR, k / kR);
        for (int i = tid; i < m; i += kT) vsh[i] = (i == 0) ? v0_g[k] : rk[k + 1 + i];
        __syncthreads();
        for (int c = warp; c < ncol; c += kNW) {
            double acc = 0.0;
            for (int i = lane; i < m; i += 32) acc = fma(vsh[i], Wo[(size_t)(k + 1 + i) * ncol + c], acc);
            acc = warp_sum(acc);
            if (lane == 0) coef[c] = tau * acc;
        }
        __syncthreads();
        for (int e = tid; e < m * ncol; e += kT) {
            const int i = e / ncol, c = e % ncol;
            Wo[(size_t)(k + 1 + i) * ncol + c] -= coef[c] * vsh[i];
        }
        __syncthreads();
    }
    // sign: largest-magnitude entry positive (first on ties)
    for (int c = warp; c < ncol; c += kNW) {
        double best = -1.0;
        int bi = 0x7fffffff;
        for (int i = lane; i < n; i += 32) {
            const double v = fabs(Wo[(size_t)i * ncol + c]);
            if (v > best) { best = v; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (lane == 0) coef[c] = Wo[(size_t)bi * ncol + c] < 0.0 ? -1.0 : 1.0;
    }
    __syncthreads();
    double *V = a.V + (long)mat * n * d;
    for (int e = tid; e < n * ncol; e += kT) {
        const int i = e / ncol, c = e % ncol;
        V[(long)i * d + (r + c * kR)] = coef[c] * Wo[e];
    }
    cl.sync();  // no CTA leaves while others may still read its shared memory
}

}  // namespace

struct EigPlan {
    size_t rows_g, dg, ed, tau, v0, Z, lu, piv, sig, lam, order, total;
    int rows_in_smem;
    size_t smem;
};

static EigPlan eig_plan(int n, int d, int mats) {
    EigPlan p{};
    const int rows_per = (n + kR - 1) / kR;
    const size_t rows_bytes = sizeof(double) * (size_t)rows_per * n;
    p.rows_in_smem = rows_bytes <= kRowsSmemMax;
    const int ncol_max = (d + kR - 1) / kR;
    p.smem = (p.rows_in_smem ? rows_bytes : 0) + sizeof(double) * (3 * (size_t)n + 32 + 64 + (size_t)n * ncol_max);
    size_t o = 0;
    auto take = [&](size_t bytes) {
        const size_t at = o;
        o = align_up(o + bytes, 256);
        return at;
    };
    p.rows_g = take(p.rows_in_smem ? 0 : sizeof(double) * (size_t)mats * kR * rows_per * n);
    p.dg = take(sizeof(double) * (size_t)mats * n);
    p.ed = take(sizeof(double) * (size_t)mats * n);
    p.tau = take(sizeof(double) * (size_t)mats * n);
    p.v0 = take(sizeof(double) * (size_t)mats * n);
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

cudaError_t launch_eig(const double *cov, int n, int d, int mats, double *V, double *eigvals, void *ws,
                       cudaStream_t st) {
    const EigPlan p = eig_plan(n, d, mats);
    if (p.smem > 227 * 1024) return cudaErrorNotSupported;
    static int attr_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (attr_dev != dev) {
        cudaError_t e = cudaFuncSetAttribute(k_eig_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        if (e != cudaSuccess) return e;
        attr_dev = dev;
    }
    char *b = (char *)ws;
    EigArgs a;
    a.cov = cov;
    a.n = n;
    a.d = d;
    a.rows_in_smem = p.rows_in_smem;
    a.rows_g = (double *)(b + p.rows_g);
    a.dg = (double *)(b + p.dg);
    a.ed = (double *)(b + p.ed);
    a.tau = (double *)(b + p.tau);
    a.v0 = (double *)(b + p.v0);
    a.Z = (double *)(b + p.Z);
    a.lu = (double *)(b + p.lu);
    a.piv = (uint8_t *)(b + p.piv);
    a.sig = (float *)(b + p.sig);
    a.lam = (double *)(b + p.lam);
    a.order = (int *)(b + p.order);
    a.V = V;
    a.eig = eigvals;
    QFCA_LAUNCH("k_eig_cluster", st, k_eig_cluster<<<kR * mats, kT, p.smem, st>>>(a));
    return cudaGetLastError();
}

}  // namespace qfca
