// fit.cu -- single-image PCA fit (arXiv 2510.15602, Sec. 3.3) on the GPU in FP64.
//
//   k_mean      mu_c = (1/N) sum_p x_cp                          (FP64 sums)
//   k_cov_tile  split-K partial sums of (x_p - mu)(x_p - mu)^T over 64x64
//               tiles of the upper triangle                       (FP64 DFMA)
//   k_cov_reduce  fixed-order sum of the split partials, scaled by 1/N,
//               mirrored to full storage                          (deterministic)
//   k_eig       top-d eigenpairs of the symmetric C x C covariance, one CTA
//               per matrix: Householder tridiagonalisation (FP64), bisection
//               on the Sturm count of the tridiagonal (FP32, as a shift only),
//               inverse iteration (FP64), Gram-Schmidt, Rayleigh quotients,
//               back-transformation by the stored reflectors, sign
//               normalisation (largest-magnitude entry positive).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "internal.cuh"

namespace qfca {
namespace {

constexpr int kTile = 64;
constexpr int kKStep = 16;
constexpr int kEigThreads = 512;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide FP64 sum with a fixed reduction order.  red: >= 32 doubles of smem.
__device__ double block_sum(double v, double *red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (warp == 0) {
        t = lane < nw ? red[lane] : 0.0;
        t = warp_sum(t);
        if (lane == 0) red[0] = t;
    }
    __syncthreads();
    t = red[0];
    __syncthreads();
    return t;
}

__global__ void k_mean(const float *__restrict__ X, int layout, int C, long N, double *__restrict__ mean) {
    __shared__ double red[32];
    const int c = blockIdx.x;
    double s = 0.0;
    if (layout == QFCA_NCHW) {
        const float *row = X + (long)c * N;
        for (long p = threadIdx.x; p < N; p += blockDim.x) s += (double)row[p];
    } else {
        for (long p = threadIdx.x; p < N; p += blockDim.x) s += (double)X[p * C + c];
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) mean[c] = s / (double)N;
}

// One CTA = one (tile pair, split).  256 threads, each 4x4 outputs of the 64x64 tile.
// Linear index of an upper-triangle tile pair (i <= j) of an nt x nt tile grid -> (i, j).
__device__ __forceinline__ int2 tile_pair(int p, int nt) {
    int i = 0;
    while (p >= nt - i) { p -= nt - i; i++; }
    return make_int2(i, i + p);
}

__global__ void __launch_bounds__(256) k_cov_tile(const float *__restrict__ X, int layout, int C, long N,
                                                  const double *__restrict__ mean, int nt, int n_pairs,
                                                  long chunk, double *__restrict__ part) {
    __shared__ double As[kKStep][kTile + 2];
    __shared__ double Bs[kKStep][kTile + 2];
    const int pair = blockIdx.x % n_pairs;
    const int split = blockIdx.x / n_pairs;
    const int2 tp = tile_pair(pair, nt);
    const int ti = tp.x, tj = tp.y;
    const long p0 = (long)split * chunk;
    const long p1 = min(N, p0 + chunk);
    const int tid = threadIdx.x;
    const int ty = tid >> 4, tx = tid & 15;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = 0.0;

    for (long pk = p0; pk < p1; pk += kKStep) {
        // stage 64 channels x 16 pixels of each operand, centred, as FP64
#pragma unroll
        for (int rep = 0; rep < 4; rep++) {
            const int e = tid + rep * 256;     // 0..1023
            int cl, kk;
            if (layout == QFCA_NCHW) { cl = e >> 4; kk = e & 15; }
            else { kk = e >> 6; cl = e & 63; }
            const long p = pk + kk;
            const int ca = ti * kTile + cl, cb = tj * kTile + cl;
            double va = 0.0, vb = 0.0;
            if (p < p1) {
                if (ca < C) va = (double)(layout == QFCA_NCHW ? X[(long)ca * N + p] : X[p * C + ca]) - mean[ca];
                if (cb < C) vb = (double)(layout == QFCA_NCHW ? X[(long)cb * N + p] : X[p * C + cb]) - mean[cb];
            }
            As[kk][cl] = va;
            Bs[kk][cl] = vb;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kKStep; kk++) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; i++) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; j++) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    double *out = part + ((long)split * n_pairs + pair) * (kTile * kTile);
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) out[(ty * 4 + i) * kTile + tx * 4 + j] = acc[i][j];
}

__global__ void k_cov_reduce(const double *__restrict__ part, int nt, int n_pairs, int n_split, int C, long N,
                             double *__restrict__ cov) {
    const int pair = blockIdx.x;
    const int2 tp = tile_pair(pair, nt);
    const int ti = tp.x, tj = tp.y;
    const double inv = 1.0 / (double)N;
    for (int e = threadIdx.x; e < kTile * kTile; e += blockDim.x) {
        const int li = e / kTile, lj = e % kTile;
        const int i = ti * kTile + li, j = tj * kTile + lj;
        if (i >= C || j >= C) continue;
        double s = 0.0;
        for (int sp = 0; sp < n_split; sp++) s += part[((long)sp * n_pairs + pair) * (kTile * kTile) + e];
        s *= inv;
        if (ti != tj || i <= j) {
            cov[(long)i * C + j] = s;
            cov[(long)j * C + i] = s;
        }
    }
}

// ------------------------------------------------------------------ eigensolver

// Number of eigenvalues of the symmetric tridiagonal (dg, e2 = off^2) below x (FP32 Sturm count).
__device__ int sturm_count_f32(const float *dg, const float *e2, int n, float x) {
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

// Solve (T - sigma I) z = rhs by Gaussian elimination with partial pivoting,
// in place on rhs (length n).  dg/ed: FP64 tridiagonal.  u0,u1,u2,lm,piv: scratch [n].
__device__ void tridiag_solve(const double *dg, const double *ed, int n, double sigma, double tiny,
                              double *u0, double *u1, double *u2, double *lm, uint8_t *piv, double *rhs) {
    double r0 = dg[0] - sigma, r1 = n > 1 ? ed[0] : 0.0, r2 = 0.0;
    for (int i = 0; i < n - 1; i++) {
        const double s0 = ed[i], s1 = dg[i + 1] - sigma, s2 = (i + 1 < n - 1) ? ed[i + 1] : 0.0;
        if (fabs(r0) >= fabs(s0)) {
            if (r0 == 0.0) r0 = tiny;
            const double l = s0 / r0;
            u0[i] = r0; u1[i] = r1; u2[i] = r2; lm[i] = l; piv[i] = 0;
            r0 = s1 - l * r1;
            r1 = s2 - l * r2;
            r2 = 0.0;
        } else {
            const double l = r0 / s0;
            u0[i] = s0; u1[i] = s1; u2[i] = s2; lm[i] = l; piv[i] = 1;
            const double n0 = r1 - l * s1, n1 = r2 - l * s2;
            r0 = n0; r1 = n1; r2 = 0.0;
        }
    }
    if (r0 == 0.0) r0 = tiny;
    u0[n - 1] = r0; u1[n - 1] = 0.0; u2[n - 1] = 0.0;
    // forward: apply P and L
    for (int i = 0; i < n - 1; i++) {
        if (piv[i]) { const double t = rhs[i]; rhs[i] = rhs[i + 1]; rhs[i + 1] = t; }
        rhs[i + 1] -= lm[i] * rhs[i];
    }
    // backward: U
    rhs[n - 1] = rhs[n - 1] / u0[n - 1];
    if (n >= 2) rhs[n - 2] = (rhs[n - 2] - u1[n - 2] * rhs[n - 1]) / u0[n - 2];
    for (int i = n - 3; i >= 0; i--) rhs[i] = (rhs[i] - u1[i] * rhs[i + 1] - u2[i] * rhs[i + 2]) / u0[i];
}

struct EigScratch {
    double *dg, *ed, *tau;      // [n]
    float *dg32, *e232;         // [n]
    double *Z;                  // [d][n]  tridiagonal eigenvectors, then [n][d] after back-transform
    double *W;                  // [n][d]
    double *u0, *u1, *u2, *lm;  // [d][n]
    uint8_t *piv;               // [d][n]
    double *lam;                // [d]
    int *order;                 // [d]
};

// A: n x n symmetric (full storage), overwritten.  One CTA of kEigThreads threads.
__global__ void __launch_bounds__(kEigThreads) k_eig(double *__restrict__ A, int n, int d, EigScratch s,
                                                     double *__restrict__ V, double *__restrict__ eigvals) {
    __shared__ double vsh[kMaxC];
    __shared__ double wsh[kMaxC];
    __shared__ double red[32];
    __shared__ double coef[kMaxD];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int NW = kEigThreads / 32;

    // ---- 1. Householder tridiagonalisation A = Q T Q^T; v_k kept in row k of A.
    for (int k = 0; k + 2 < n; k++) {
        const int m = n - k - 1;
        double part = 0.0;
        for (int i = tid; i < m; i += kEigThreads) {
            const double x = A[(long)(k + 1 + i) * n + k];
            vsh[i] = x;
            if (i >= 1) part += x * x;
        }
        const double sigma = block_sum(part, red);
        const double alpha = vsh[0];
        double tau = 0.0, ek = alpha;
        if (sigma > 0.0) {
            const double mu = sqrt(alpha * alpha + sigma);
            const double v0 = alpha >= 0.0 ? alpha + mu : alpha - mu;
            ek = alpha >= 0.0 ? -mu : mu;
            tau = 2.0 / (v0 * v0 + sigma);
            __syncthreads();
            if (tid == 0) vsh[0] = v0;
            __syncthreads();
        }
        if (tid == 0) { s.tau[k] = tau; s.ed[k] = ek; s.dg[k] = A[(long)k * n + k]; }
        // keep v_k in row k (columns k+1..n-1), which the trailing update never touches again
        for (int i = tid; i < m; i += kEigThreads) A[(long)k * n + k + 1 + i] = vsh[i];
        if (tau == 0.0) { __syncthreads(); continue; }
        // p = tau * A_sub v : one warp per row
        for (int i = warp; i < m; i += NW) {
            const double *row = A + (long)(k + 1 + i) * n + (k + 1);
            double acc = 0.0;
            for (int j = lane; j < m; j += 32) acc = fma(row[j], vsh[j], acc);
            acc = warp_sum(acc);
            if (lane == 0) wsh[i] = tau * acc;
        }
        __syncthreads();
        double pv = 0.0;
        for (int i = tid; i < m; i += kEigThreads) pv += wsh[i] * vsh[i];
        const double K = 0.5 * tau * block_sum(pv, red);
        for (int i = tid; i < m; i += kEigThreads) wsh[i] = wsh[i] - K * vsh[i];
        __syncthreads();
        // A_sub -= v w^T + w v^T
        for (int i = warp; i < m; i += NW) {
            double *row = A + (long)(k + 1 + i) * n + (k + 1);
            const double vi = vsh[i], wi = wsh[i];
            for (int j = lane; j < m; j += 32) row[j] = row[j] - vi * wsh[j] - wi * vsh[j];
        }
        __syncthreads();
    }
    if (tid == 0) {
        if (n >= 2) {
            s.dg[n - 2] = A[(long)(n - 2) * n + (n - 2)];
            s.ed[n - 2] = A[(long)(n - 1) * n + (n - 2)];
            s.tau[n - 2] = 0.0;
        }
        s.dg[n - 1] = A[(long)(n - 1) * n + (n - 1)];
        s.ed[n - 1] = 0.0;
        s.tau[n - 1] = 0.0;
    }
    __syncthreads();
    for (int i = tid; i < n; i += kEigThreads) {
        s.dg32[i] = (float)s.dg[i];
        s.e232[i] = (float)(s.ed[i] * s.ed[i]);
    }
    // Gershgorin interval and scale
    double glo = 1e300, ghi = -1e300, tmax = 0.0;
    for (int i = tid; i < n; i += kEigThreads) {
        const double r = (i > 0 ? fabs(s.ed[i - 1]) : 0.0) + (i < n - 1 ? fabs(s.ed[i]) : 0.0);
        glo = fmin(glo, s.dg[i] - r);
        ghi = fmax(ghi, s.dg[i] + r);
        tmax = fmax(tmax, fabs(s.dg[i]) + r);
    }
    // block min/max via red (reuse block_sum on transformed values is awkward; do it explicitly)
    for (int o = 16; o > 0; o >>= 1) {
        glo = fmin(glo, __shfl_xor_sync(0xffffffffu, glo, o));
        ghi = fmax(ghi, __shfl_xor_sync(0xffffffffu, ghi, o));
        tmax = fmax(tmax, __shfl_xor_sync(0xffffffffu, tmax, o));
    }
    __shared__ double mm[3][NW];
    if (lane == 0) { mm[0][warp] = glo; mm[1][warp] = ghi; mm[2][warp] = tmax; }
    __syncthreads();
    if (tid == 0) {
        for (int w = 1; w < NW; w++) {
            mm[0][0] = fmin(mm[0][0], mm[0][w]);
            mm[1][0] = fmax(mm[1][0], mm[1][w]);
            mm[2][0] = fmax(mm[2][0], mm[2][w]);
        }
    }
    __syncthreads();
    glo = mm[0][0];
    ghi = mm[1][0];
    tmax = fmax(mm[2][0], 1e-300);

    // ---- 2. shifts: the (t+1)-th largest eigenvalue by FP32 bisection; 3. inverse iteration (FP64)
    if (tid < d) {
        const int t = tid;
        const int target = n - 1 - t;  // ascending index
        const float span = (float)(ghi - glo);
        float lo = (float)glo - 1e-3f * span - 1e-30f, hi = (float)ghi + 1e-3f * span + 1e-30f;
        for (int it = 0; it < 80; it++) {
            const float mid = 0.5f * (lo + hi);
            if (mid <= lo || mid >= hi) break;
            if (sturm_count_f32(s.dg32, s.e232, n, mid) > target) hi = mid;
            else lo = mid;
            if (hi - lo <= 2.0f * 1.2e-7f * fmaxf(fabsf(lo), fabsf(hi))) break;
        }
        const double sigma = 0.5 * ((double)lo + (double)hi);
        double *z = s.Z + (long)t * n;
        // deterministic, non-degenerate start vector
        for (int i = 0; i < n; i++) z[i] = 1.0 + 0.5 * sin(0.7 * (double)(i + 1) + 1.3 * (double)(t + 1));
        const double tiny = 2.2e-16 * tmax;
        for (int it = 0; it < 5; it++) {
            tridiag_solve(s.dg, s.ed, n, sigma, tiny, s.u0 + (long)t * n, s.u1 + (long)t * n,
                          s.u2 + (long)t * n, s.lm + (long)t * n, s.piv + (long)t * n, z);
            double nrm = 0.0;
            for (int i = 0; i < n; i++) nrm = fma(z[i], z[i], nrm);
            nrm = 1.0 / sqrt(nrm);
            for (int i = 0; i < n; i++) z[i] *= nrm;
        }
    }
    __syncthreads();
    // ---- 4. Gram-Schmidt over the d tridiagonal eigenvectors (in descending order)
    for (int t = 1; t < d; t++) {
        double *zt = s.Z + (long)t * n;
        for (int q = warp; q < t; q += NW) {
            const double *zq = s.Z + (long)q * n;
            double acc = 0.0;
            for (int i = lane; i < n; i += 32) acc = fma(zq[i], zt[i], acc);
            acc = warp_sum(acc);
            if (lane == 0) coef[q] = acc;
        }
        __syncthreads();
        double part = 0.0;
        for (int i = tid; i < n; i += kEigThreads) {
            double v = zt[i];
            for (int q = 0; q < t; q++) v -= coef[q] * s.Z[(long)q * n + i];
            zt[i] = v;
            part += v * v;
        }
        const double nrm = block_sum(part, red);
        const double inv = 1.0 / sqrt(nrm);
        for (int i = tid; i < n; i += kEigThreads) zt[i] *= inv;
        __syncthreads();
    }
    // ---- 5. Rayleigh quotients z^T T z and a stable descending order
    if (tid < d) {
        const double *z = s.Z + (long)tid * n;
        double acc = 0.0;
        for (int i = 0; i < n; i++) {
            double tz = s.dg[i] * z[i];
            if (i > 0) tz += s.ed[i - 1] * z[i - 1];
            if (i < n - 1) tz += s.ed[i] * z[i + 1];
            acc = fma(z[i], tz, acc);
        }
        s.lam[tid] = acc;
    }
    __syncthreads();
    if (tid == 0) {
        for (int t = 0; t < d; t++) s.order[t] = t;
        for (int a = 1; a < d; a++) {  // insertion sort, descending, stable
            const int x = s.order[a];
            int b = a - 1;
            while (b >= 0 && s.lam[s.order[b]] < s.lam[x]) { s.order[b + 1] = s.order[b]; b--; }
            s.order[b + 1] = x;
        }
    }
    __syncthreads();
    // W[i][j] = Z_sorted: row-major [n][d]
    for (int e = tid; e < n * d; e += kEigThreads) {
        const int i = e / d, j = e % d;
        s.W[e] = s.Z[(long)s.order[j] * n + i];
    }
    __syncthreads();
    // ---- 6. back-transformation V = H_0 ... H_{n-3} W
    for (int k = n - 3; k >= 0; k--) {
        const double tau = s.tau[k];
        if (tau == 0.0) continue;
        const int m = n - k - 1;
        const double *v = A + (long)k * n + (k + 1);
        for (int j = warp; j < d; j += NW) {
            double acc = 0.0;
            for (int i = lane; i < m; i += 32) acc = fma(v[i], s.W[(long)(k + 1 + i) * d + j], acc);
            acc = warp_sum(acc);
            if (lane == 0) coef[j] = tau * acc;
        }
        __syncthreads();
        for (int e = tid; e < m * d; e += kEigThreads) {
            const int i = e / d, j = e % d;
            s.W[(long)(k + 1 + i) * d + j] -= coef[j] * v[i];
        }
        __syncthreads();
    }
    // ---- 7. sign normalisation and output
    for (int j = warp; j < d; j += NW) {
        double best = -1.0;
        int bi = 0x7fffffff;
        for (int i = lane; i < n; i += 32) {
            const double a = fabs(s.W[(long)i * d + j]);
            if (a > best) { best = a; bi = i; }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if (lane == 0) coef[j] = s.W[(long)bi * d + j] < 0.0 ? -1.0 : 1.0;
    }
    __syncthreads();
    for (int e = tid; e < n * d; e += kEigThreads) V[e] = coef[e % d] * s.W[e];
    if (tid < d) eigvals[tid] = s.lam[s.order[tid]];
}

struct FitLayout {
    size_t off_part, off_cov, off_eig, total;
    int n_pairs, n_split;
    long chunk;
};

FitLayout fit_layout(int C, long N, int d) {
    FitLayout L{};
    const int nt = (C + kTile - 1) / kTile;
    L.n_pairs = nt * (nt + 1) / 2;
    // about 4 CTAs per SM over 152 SMs, chunks of >= 256 pixels
    int want = (4 * 152 + L.n_pairs - 1) / L.n_pairs;
    long chunk = (N + want - 1) / want;
    chunk = ((chunk + kKStep - 1) / kKStep) * kKStep;
    if (chunk < 256) chunk = 256;
    L.chunk = chunk;
    L.n_split = (int)((N + chunk - 1) / chunk);
    size_t o = 0;
    L.off_part = o; o = align_up(o + sizeof(double) * (size_t)L.n_split * L.n_pairs * kTile * kTile, 256);
    L.off_cov = o; o = align_up(o + sizeof(double) * (size_t)C * C, 256);
    L.off_eig = o;
    const size_t n = C;
    size_t e = 0;
    e += 3 * n * sizeof(double);              // dg, ed, tau
    e += 2 * n * sizeof(float);               // dg32, e232
    e += 2 * n * d * sizeof(double);          // Z, W
    e += 4 * n * d * sizeof(double);          // u0,u1,u2,lm
    e += n * d;                               // piv
    e += d * sizeof(double) + d * sizeof(int) + 16 * 64;
    o = align_up(o + e, 256);
    L.total = o;
    return L;
}

}  // namespace

size_t fit_workspace_bytes(int C, long N, int d) { return fit_layout(C, N, d).total; }

cudaError_t launch_fit(const float *X, int layout, int H, int W, int C, int d, double *mean, double *V,
                       double *eigvals, void *ws, cudaStream_t st) {
    const long N = (long)H * W;
    const FitLayout L = fit_layout(C, N, d);
    char *base = (char *)ws;
    double *part = (double *)(base + L.off_part);
    double *cov = (double *)(base + L.off_cov);
    const int nt = (C + kTile - 1) / kTile;
    QFCA_LAUNCH("k_mean", st, k_mean<<<C, 256, 0, st>>>(X, layout, C, N, mean));
    QFCA_LAUNCH("k_cov_tile_f64", st,
                k_cov_tile<<<L.n_pairs * L.n_split, 256, 0, st>>>(X, layout, C, N, mean, nt, L.n_pairs, L.chunk, part));
    QFCA_LAUNCH("k_cov_reduce", st, k_cov_reduce<<<L.n_pairs, 256, 0, st>>>(part, nt, L.n_pairs, L.n_split, C, N, cov));
    // eigensolver scratch
    char *e = base + L.off_eig;
    EigScratch s;
    const size_t n = C;
    s.dg = (double *)e; e += n * sizeof(double);
    s.ed = (double *)e; e += n * sizeof(double);
    s.tau = (double *)e; e += n * sizeof(double);
    s.Z = (double *)e; e += n * d * sizeof(double);
    s.W = (double *)e; e += n * d * sizeof(double);
    s.u0 = (double *)e; e += n * d * sizeof(double);
    s.u1 = (double *)e; e += n * d * sizeof(double);
    s.u2 = (double *)e; e += n * d * sizeof(double);
    s.lm = (double *)e; e += n * d * sizeof(double);
    s.lam = (double *)e; e += d * sizeof(double);
    s.dg32 = (float *)e; e += n * sizeof(float);
    s.e232 = (float *)e; e += n * sizeof(float);
    s.order = (int *)e; e += d * sizeof(int);
    s.piv = (uint8_t *)e;
    QFCA_LAUNCH("k_eig", st, k_eig<<<1, kEigThreads, 0, st>>>(cov, C, d, s, V, eigvals));
    return cudaGetLastError();
}

}  // namespace qfca
