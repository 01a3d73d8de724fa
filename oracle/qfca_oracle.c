/*
 * qfca_oracle.c -- plain, slow, FP64 CPU oracle for the QFCA hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file: only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no code, header, table or constant with
 * the CUDA library; it follows the paper's definitions directly, with no
 * blocking, fusion or reordering beyond what the definitions state.
 *
 * Steps (arXiv 2510.15602):
 *   fit       -- single-image PCA (Sec. 3.3): mean, covariance, full
 *                eigendecomposition by the textbook cyclic Jacobi method,
 *                top-d eigenvectors in descending eigenvalue order.
 *   project   -- Y = (X - mean) V, the principal components (Sec. 3.3).
 *   quantize  -- N equally spaced values per component (Sec. 3.1):
 *                q = min(B-1, floor((y - lo) / (hi - lo) * B)).
 *   ref_hist  -- reference histogram R_b: count of pixels in bin b.
 *   score     -- per-pixel histogram P_b over the (2r+1)^2 window clipped at
 *                the image border (Sec. 3.1), and the 1-D Wasserstein-1
 *                distance to R in bin units, which for histograms is the L1
 *                distance of the normalised CDFs (supplement, Wasserstein
 *                closed form): D = sum_b |cumP_b * N_ref - cumR_b * N_loc|,
 *                EMD = D / (N_loc * N_ref); score = mean over components
 *                (channel averaging, Sec. 3).
 *
 * Readings where the paper is silent (each is listed with the design notes):
 *   - covariance normalised by 1/N (N = H*W); the scale does not move the
 *     eigenvectors;
 *   - eigenvalue ties: the lower original index first; each eigenvector is
 *     signed so that its largest-magnitude entry is positive (first such
 *     entry on ties);
 *   - bins: the component maximum goes to bin B-1; hi == lo gives bin 0;
 *     fixed ranges clamp to [0, B-1];
 *   - windows are clipped (not padded) at the border; EMD is in bin units.
 *
 * Build: gcc -O2 -fPIC -shared -ffp-contract=off -o liboracle.so qfca_oracle.c -lm
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_NCHW 0
#define ORC_NHWC 1

/* Feature value of channel c at pixel p (p = y*W + x). */
static double feat(const float *X, int layout, int C, long N, int c, long p)
{
    if (layout == ORC_NCHW)
        return (double)X[(long)c * N + p];
    return (double)X[p * (long)C + c];
}

/* ------------------------------------------------------------------ fit */

/* Textbook cyclic Jacobi (Golub & Van Loan, Sec. 8.5): A (n x n, row-major,
 * symmetric) is overwritten; eigenvalues land on its diagonal and Q (n x n,
 * row-major) receives the eigenvectors as columns.  Returns sweeps used. */
static int jacobi_eig(double *A, int n, double *Q)
{
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++)
            Q[(long)i * n + j] = (i == j) ? 1.0 : 0.0;
    double frob = 0.0;
    for (long i = 0; i < (long)n * n; i++)
        frob += A[i] * A[i];
    frob = sqrt(frob);
    int sweep;
    for (sweep = 0; sweep < 100; sweep++) {
        double off = 0.0;
        for (int i = 0; i < n; i++)
            for (int j = 0; j < n; j++)
                if (i != j)
                    off += A[(long)i * n + j] * A[(long)i * n + j];
        off = sqrt(off);
        if (off <= 1e-15 * frob || off == 0.0)
            break;
        for (int p = 0; p < n - 1; p++) {
            for (int q = p + 1; q < n; q++) {
                double apq = A[(long)p * n + q];
                if (apq == 0.0)
                    continue;
                double app = A[(long)p * n + p], aqq = A[(long)q * n + q];
                /* rotation angle that annihilates a_pq */
                double tau = (aqq - app) / (2.0 * apq);
                double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                double c = 1.0 / sqrt(1.0 + t * t);
                double s = t * c;
                /* A <- A J (columns p, q) */
                for (int k = 0; k < n; k++) {
                    double akp = A[(long)k * n + p], akq = A[(long)k * n + q];
                    A[(long)k * n + p] = c * akp - s * akq;
                    A[(long)k * n + q] = s * akp + c * akq;
                }
                /* A <- J^T A (rows p, q) */
                for (int k = 0; k < n; k++) {
                    double apk = A[(long)p * n + k], aqk = A[(long)q * n + k];
                    A[(long)p * n + k] = c * apk - s * aqk;
                    A[(long)q * n + k] = s * apk + c * aqk;
                }
                A[(long)p * n + q] = 0.0;
                A[(long)q * n + p] = 0.0;
                /* Q <- Q J */
                for (int k = 0; k < n; k++) {
                    double qkp = Q[(long)k * n + p], qkq = Q[(long)k * n + q];
                    Q[(long)k * n + p] = c * qkp - s * qkq;
                    Q[(long)k * n + q] = s * qkp + c * qkq;
                }
            }
        }
    }
    return sweep;
}

/* Covariance of the feature map: cov[i][j] = (1/N) sum_p (x_ip - mu_i)(x_jp - mu_j). */
void orc_covariance(const float *X, int layout, int H, int W, int C, double *mean, double *cov)
{
    long N = (long)H * W;
    for (int c = 0; c < C; c++) {
        double s = 0.0;
        for (long p = 0; p < N; p++)
            s += feat(X, layout, C, N, c, p);
        mean[c] = s / (double)N;
    }
    for (int i = 0; i < C; i++) {
        for (int j = i; j < C; j++) {
            double s = 0.0;
            for (long p = 0; p < N; p++)
                s += (feat(X, layout, C, N, i, p) - mean[i]) * (feat(X, layout, C, N, j, p) - mean[j]);
            cov[(long)i * C + j] = s / (double)N;
            cov[(long)j * C + i] = s / (double)N;
        }
    }
}

/* Eigendecomposition of a symmetric C x C matrix, sorted descending (ties:
 * lower original index first), each eigenvector sign-normalised.  Writes the
 * top-d eigenvectors to V (C x d, column k = component k), their eigenvalues
 * to eigvals[d], and all C eigenvalues to all_eigvals (may be NULL). */
int orc_eigh_topd(const double *S, int C, int d, double *V, double *eigvals, double *all_eigvals)
{
    double *A = (double *)malloc(sizeof(double) * C * C);
    double *Q = (double *)malloc(sizeof(double) * C * C);
    int *order = (int *)malloc(sizeof(int) * C);
    if (!A || !Q || !order) {
        free(A); free(Q); free(order);
        return -1;
    }
    memcpy(A, S, sizeof(double) * C * C);
    int sweeps = jacobi_eig(A, C, Q);
    /* stable selection sort by descending eigenvalue */
    for (int i = 0; i < C; i++)
        order[i] = i;
    for (int i = 0; i < C; i++) {
        int best = i;
        for (int j = i + 1; j < C; j++) {
            double lj = A[(long)order[j] * C + order[j]], lb = A[(long)order[best] * C + order[best]];
            if (lj > lb || (lj == lb && order[j] < order[best]))
                best = j;
        }
        int tmp = order[i]; order[i] = order[best]; order[best] = tmp;
    }
    for (int i = 0; i < C; i++)
        if (all_eigvals)
            all_eigvals[i] = A[(long)order[i] * C + order[i]];
    for (int k = 0; k < d; k++) {
        int col = order[k];
        eigvals[k] = A[(long)col * C + col];
        /* sign: largest-magnitude entry positive (first on ties) */
        int imax = 0;
        double amax = -1.0;
        for (int c = 0; c < C; c++) {
            double a = fabs(Q[(long)c * C + col]);
            if (a > amax) { amax = a; imax = c; }
        }
        double sgn = Q[(long)imax * C + col] < 0.0 ? -1.0 : 1.0;
        for (int c = 0; c < C; c++)
            V[(long)c * d + k] = sgn * Q[(long)c * C + col];
    }
    free(A); free(Q); free(order);
    return sweeps;
}

/* PCA fit on a single image (Sec. 3.3). */
int orc_fit(const float *X, int layout, int H, int W, int C, int d,
            double *mean, double *V, double *eigvals, double *all_eigvals, double *cov_out)
{
    double *cov = cov_out ? cov_out : (double *)malloc(sizeof(double) * C * C);
    if (!cov)
        return -1;
    orc_covariance(X, layout, H, W, C, mean, cov);
    int rc = orc_eigh_topd(cov, C, d, V, eigvals, all_eigvals);
    if (!cov_out)
        free(cov);
    return rc;
}

/* ------------------------------------------------------------------ project */

/* Y[k][p] = sum_c (x_cp - mean_c) V[c][k]  (FP64). */
void orc_project(const float *X, int layout, int H, int W, int C, const double *mean,
                 const double *V, int d, double *Y)
{
    long N = (long)H * W;
    for (int k = 0; k < d; k++)
        for (long p = 0; p < N; p++) {
            double s = 0.0;
            for (int c = 0; c < C; c++)
                s += (feat(X, layout, C, N, c, p) - mean[c]) * V[(long)c * d + k];
            Y[(long)k * N + p] = s;
        }
}

/* ------------------------------------------------------------------ quantize */

/* Uniform quantisation of each component into B bins (Sec. 3.1).
 * mode 0: lo/hi = the component's min/max over the image (written to lo_out,
 *         hi_out); mode 1: lo/hi given (lo_in, hi_in), values clamped.
 * fp32_decision != 0 takes the bin decision in single precision on values
 * rounded to float, with the formula t = (y - lo) / (hi - lo); q = (int)(t * B),
 * so a kernel deciding in FP32 can be compared bit for bit.  Otherwise the
 * decision is q = floor((y - lo) / (hi - lo) * B) in FP64. */
void orc_quantize(const double *Y, int d, long N, int B, int mode, const double *lo_in,
                  const double *hi_in, int fp32_decision, double *lo_out, double *hi_out, uint8_t *q)
{
    for (int k = 0; k < d; k++) {
        const double *y = Y + (long)k * N;
        double lo, hi;
        if (mode == 0) {
            lo = y[0];
            hi = y[0];
            for (long p = 1; p < N; p++) {
                if (y[p] < lo) lo = y[p];
                if (y[p] > hi) hi = y[p];
            }
        } else {
            lo = lo_in[k];
            hi = hi_in[k];
        }
        if (lo_out) lo_out[k] = lo;
        if (hi_out) hi_out[k] = hi;
        for (long p = 0; p < N; p++) {
            long b;
            if (fp32_decision) {
                float yf = (float)y[p], lf = (float)lo, hf = (float)hi;
                if (!(hf > lf)) {
                    b = 0;
                } else {
                    volatile float num = yf - lf;
                    volatile float den = hf - lf;
                    volatile float t = num / den;
                    volatile float v = t * (float)B;
                    if (v < 0.0f) b = 0;
                    else b = (long)v;
                }
            } else {
                if (!(hi > lo))
                    b = 0;
                else
                    b = (long)floor((y[p] - lo) / (hi - lo) * (double)B);
            }
            if (b < 0) b = 0;
            if (b > B - 1) b = B - 1;
            q[(long)k * N + p] = (uint8_t)b;
        }
    }
}

/* R[k][b] = number of pixels of component k in bin b. */
void orc_ref_hist(const uint8_t *q, int d, long N, int B, uint32_t *R)
{
    for (int k = 0; k < d; k++) {
        for (int b = 0; b < B; b++)
            R[(long)k * B + b] = 0;
        for (long p = 0; p < N; p++)
            R[(long)k * B + q[(long)k * N + p]]++;
    }
}

/* ------------------------------------------------------------------ score */

/* Histogram L[b] of one component plane q[H][W] over the window of pixel
 * (y, x): rows [y-r, y+r] x cols [x-r, x+r] clipped to the image.  Returns
 * N_loc, the number of pixels in the clipped window. */
long orc_window_hist(const uint8_t *q, int H, int W, int B, int r, int y, int x, int64_t *L)
{
    for (int b = 0; b < B; b++)
        L[b] = 0;
    long n = 0;
    for (int yy = y - r; yy <= y + r; yy++)
        for (int xx = x - r; xx <= x + r; xx++)
            if (yy >= 0 && yy < H && xx >= 0 && xx < W) {
                L[q[(long)yy * W + xx]]++;
                n++;
            }
    return n;
}

/* The quantized value of bin b of a component quantized between lo and hi
 * into B equally spaced values (Sec. 3.1): the centre of the bin. */
static double bin_value(double lo, double hi, int B, int b)
{
    return lo + ((double)b + 0.5) * (hi - lo) / (double)B;
}

/* Window histogram + 1-D EMD per component + mean over components.
 * q: [d][H][W] bins; R: [d][B]; Nref: reference mass.  Writes score[H][W]
 * (FP64), and optionally numer[d][H][W] (exact D, bin units) and nloc[H][W].
 * Units: with lo/hi NULL the distance between bins a and b is |a - b| (bin
 * units); with lo/hi ([d], the component's quantisation range) it is the
 * distance of the quantized values |Q_a - Q_b| (value units), so the W1
 * closed form weighs the CDF difference after bin b by Q_{b+1} - Q_b. */
int orc_score(const uint8_t *q, int d, int H, int W, int B, int r, const uint32_t *R,
              uint64_t Nref, double *score, int64_t *numer, int32_t *nloc, const double *lo,
              const double *hi)
{
    long N = (long)H * W;
    int64_t *L = (int64_t *)malloc(sizeof(int64_t) * (B > 0 ? B : 1));
    if (!L)
        return -1;
    for (int y = 0; y < H; y++) {
        for (int x = 0; x < W; x++) {
            int y0 = y - r < 0 ? 0 : y - r, y1 = y + r > H - 1 ? H - 1 : y + r;
            int x0 = x - r < 0 ? 0 : x - r, x1 = x + r > W - 1 ? W - 1 : x + r;
            int64_t Nloc = (int64_t)(y1 - y0 + 1) * (x1 - x0 + 1);
            if (nloc)
                nloc[(long)y * W + x] = (int32_t)Nloc;
            double s = 0.0;
            for (int k = 0; k < d; k++) {
                for (int b = 0; b < B; b++)
                    L[b] = 0;
                for (int yy = y0; yy <= y1; yy++)
                    for (int xx = x0; xx <= x1; xx++)
                        L[q[(long)k * N + (long)yy * W + xx]]++;
                int64_t cumL = 0, cumR = 0, D = 0;
                double Dv = 0.0;
                for (int b = 0; b < B; b++) {
                    cumL += L[b];
                    cumR += (int64_t)R[(long)k * B + b];
                    int64_t diff = cumL * (int64_t)Nref - cumR * Nloc;
                    int64_t ad = diff < 0 ? -diff : diff;
                    D += ad;
                    if (lo && b + 1 < B)
                        Dv += (double)ad * (bin_value(lo[k], hi[k], B, b + 1) - bin_value(lo[k], hi[k], B, b));
                }
                if (numer)
                    numer[(long)k * N + (long)y * W + x] = D;
                s += (lo ? Dv : (double)D) / ((double)Nloc * (double)Nref);
            }
            score[(long)y * W + x] = s / (double)d;
        }
    }
    free(L);
    return 0;
}

/* One pixel of orc_score: the window histogram of (y, x) per component
 * (orc_window_hist), its EMD numerator D_k against R_k, and the mean over
 * components of D_k / (N_loc N_ref) (Sec. 3.1, Sec. 3).  Writes numer[d]
 * when non-NULL; returns the score, or -1 on allocation failure. */
double orc_score_at(const uint8_t *q, int d, int H, int W, int B, int r, const uint32_t *R,
                    uint64_t Nref, int y, int x, int64_t *numer)
{
    long N = (long)H * W;
    int64_t *L = (int64_t *)malloc(sizeof(int64_t) * (B > 0 ? B : 1));
    if (!L)
        return -1.0;
    double s = 0.0;
    for (int k = 0; k < d; k++) {
        long Nloc = orc_window_hist(q + (long)k * N, H, W, B, r, y, x, L);
        int64_t cumL = 0, cumR = 0, D = 0;
        for (int b = 0; b < B; b++) {
            cumL += L[b];
            cumR += (int64_t)R[(long)k * B + b];
            int64_t diff = cumL * (int64_t)Nref - cumR * (int64_t)Nloc;
            D += diff < 0 ? -diff : diff;
        }
        if (numer)
            numer[k] = D;
        s += (double)D / ((double)Nloc * (double)Nref);
    }
    free(L);
    return s / (double)d;
}

/* ------------------------------------------------- Algorithm 1 + association */

/* Algorithm 1 (Sec. 3.1, quantized patch mismatch score) for one window and one
 * component.  The patch histogram P (N_loc pixels) and the reference R (N_ref
 * pixels) have different masses; both are scaled to the common mass
 * N_loc * N_ref first (P'_i = P_i N_ref, R'_j = R_j N_loc), so the two-pointer
 * walk transports whole integers.  Each step compares the current bins: if
 * P'_i < R'_j the whole remainder of P'_i goes to bin j (charged to E_i at
 * distance |i - j|, bin units), R'_j shrinks and i advances; otherwise R'_j
 * goes, P'_i shrinks and j advances.  Enum[i] receives the mass-weighted
 * distance charged to bin i (an exact integer; the paper's E_i before its
 * final division is Enum[i], and E_i = Enum[i] / P'_i).  Returns the number of
 * steps (at most 2B - 1). */
int orc_alg1(const int64_t *P, const int64_t *R, int B, int64_t Nloc, int64_t Nref, int64_t *Enum)
{
    int64_t *Pw = (int64_t *)malloc(sizeof(int64_t) * (B > 0 ? B : 1));
    int64_t *Rw = (int64_t *)malloc(sizeof(int64_t) * (B > 0 ? B : 1));
    if (!Pw || !Rw) {
        free(Pw);
        free(Rw);
        return -1;
    }
    for (int b = 0; b < B; b++) {
        Pw[b] = P[b] * Nref;
        Rw[b] = R[b] * Nloc;
        Enum[b] = 0;
    }
    int i = 0, j = 0, steps = 0;
    while (i < B && j < B) {
        int64_t dist = i > j ? i - j : j - i;
        steps++;
        if (Pw[i] < Rw[j]) {
            Enum[i] += Pw[i] * dist;
            Rw[j] -= Pw[i];
            i++;
        } else {
            Enum[i] += Rw[j] * dist;
            Pw[i] -= Rw[j];
            j++;
        }
    }
    free(Pw);
    free(Rw);
    return steps;
}

/* Algorithm 1 with the paper's cost in value units: the same walk as
 * orc_alg1, each transported amount charged at |Q_i - Q_j| (Qv[b] the
 * quantized value of bin b).  Ev[i] receives the mass-weighted value distance
 * charged to bin i (E_i = Ev[i] / P'_i).  Returns the number of steps. */
int orc_alg1_values(const int64_t *P, const int64_t *R, int B, int64_t Nloc, int64_t Nref, const double *Qv,
                    double *Ev)
{
    int64_t *Pw = (int64_t *)malloc(sizeof(int64_t) * (B > 0 ? B : 1));
    int64_t *Rw = (int64_t *)malloc(sizeof(int64_t) * (B > 0 ? B : 1));
    if (!Pw || !Rw) {
        free(Pw);
        free(Rw);
        return -1;
    }
    for (int b = 0; b < B; b++) {
        Pw[b] = P[b] * Nref;
        Rw[b] = R[b] * Nloc;
        Ev[b] = 0.0;
    }
    int i = 0, j = 0, steps = 0;
    while (i < B && j < B) {
        double dist = fabs(Qv[i] - Qv[j]);
        steps++;
        if (Pw[i] < Rw[j]) {
            Ev[i] += (double)Pw[i] * dist;
            Rw[j] -= Pw[i];
            i++;
        } else {
            Ev[i] += (double)Rw[j] * dist;
            Pw[i] -= Rw[j];
            j++;
        }
    }
    free(Pw);
    free(Rw);
    return steps;
}

/* Gaussian smoothing of an H x W map with standard deviation sigma (the final
 * low-pass step, sigma_s): separable, taps |t| <= ceil(4 sigma) with weights
 * exp(-t^2 / (2 sigma^2)), renormalised over the taps that fall inside the
 * image.  sigma <= 0 copies.  Returns 0, or -1 on allocation failure. */
int orc_blur(const double *in, int H, int W, double sigma, double *out)
{
    long N = (long)H * W;
    if (!(sigma > 0.0)) {
        for (long p = 0; p < N; p++)
            out[p] = in[p];
        return 0;
    }
    double *tmp = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
    if (!tmp)
        return -1;
    int R4 = (int)ceil(4.0 * sigma);
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            double s = 0.0, w = 0.0;
            for (int t = -R4; t <= R4; t++)
                if (x + t >= 0 && x + t < W) {
                    double g = exp(-(double)t * t / (2.0 * sigma * sigma));
                    s += g * in[(long)y * W + x + t];
                    w += g;
                }
            tmp[(long)y * W + x] = s / w;
        }
    for (int y = 0; y < H; y++)
        for (int x = 0; x < W; x++) {
            double s = 0.0, w = 0.0;
            for (int t = -R4; t <= R4; t++)
                if (y + t >= 0 && y + t < H) {
                    double g = exp(-(double)t * t / (2.0 * sigma * sigma));
                    s += g * tmp[(long)(y + t) * W + x];
                    w += g;
                }
            out[(long)y * W + x] = s / w;
        }
    free(tmp);
    return 0;
}

/* The paper's scoring (Sec. 3.1 and the error-to-pixel association): for each
 * component k and each window centre p, Algorithm 1 gives the per-bin errors
 * E_{k,p}[b] = Enum[b] / (P_b N_ref) (0 for empty bins).  A pixel q takes,
 * from every window that contains it, the error of its own bin b_k(q), and
 * averages them (the association with sigma_p = infinity: a box average over
 * the window centres p with |p - q|_inf <= r inside the image); the score
 * before smoothing is the mean over components:
 *     raw(q) = (1/d) sum_k (1/n(q)) sum_{p in box(q)} E_{k,p}[b_k(q)].
 * Then the Gaussian smoothing orc_blur with standard deviation sigma_s.  Writes raw[H][W], score[H][W] and, when
 * non-NULL, comp[d][H][W] = the per-component averages.  Units: bin units with
 * lo/hi NULL, else value units (orc_alg1_values with the quantized values of
 * each component's range lo[k]..hi[k]).  Returns 0, or -1 on allocation failure. */
int orc_assoc(const uint8_t *q, int d, int H, int W, int B, int r, const uint32_t *R, uint64_t Nref,
              double sigma_s, double *raw, double *score, double *comp, const double *lo, const double *hi)
{
    long N = (long)H * W;
    double *E = (double *)malloc(sizeof(double) * (size_t)N * (B > 0 ? B : 1));
    int64_t *L = (int64_t *)malloc(sizeof(int64_t) * (B > 0 ? B : 1));
    int64_t *Rk = (int64_t *)malloc(sizeof(int64_t) * (B > 0 ? B : 1));
    int64_t *En = (int64_t *)malloc(sizeof(int64_t) * (B > 0 ? B : 1));
    double *Ev = (double *)malloc(sizeof(double) * (B > 0 ? B : 1));
    double *Qv = (double *)malloc(sizeof(double) * (B > 0 ? B : 1));
    if (!E || !L || !Rk || !En || !Ev || !Qv) {
        free(E);
        free(L);
        free(Rk);
        free(En);
        free(Ev);
        free(Qv);
        return -1;
    }
    for (long p = 0; p < N; p++)
        raw[p] = 0.0;
    for (int k = 0; k < d; k++) {
        const uint8_t *qk = q + (long)k * N;
        for (int b = 0; b < B; b++) {
            Rk[b] = (int64_t)R[(long)k * B + b];
            if (lo)
                Qv[b] = bin_value(lo[k], hi[k], B, b);
        }
        /* per-bin errors of every window of component k */
        for (int y = 0; y < H; y++)
            for (int x = 0; x < W; x++) {
                long Nloc = orc_window_hist(qk, H, W, B, r, y, x, L);
                double *e = E + ((long)y * W + x) * B;
                if (lo) {
                    if (orc_alg1_values(L, Rk, B, Nloc, (int64_t)Nref, Qv, Ev) < 0)
                        goto oom;
                    for (int b = 0; b < B; b++)
                        e[b] = L[b] > 0 ? Ev[b] / ((double)L[b] * (double)Nref) : 0.0;
                } else {
                    if (orc_alg1(L, Rk, B, Nloc, (int64_t)Nref, En) < 0)
                        goto oom;
                    for (int b = 0; b < B; b++)
                        e[b] = L[b] > 0 ? (double)En[b] / ((double)L[b] * (double)Nref) : 0.0;
                }
            }
        /* association: each pixel averages its own bin's error over the windows that contain it */
        for (int y = 0; y < H; y++)
            for (int x = 0; x < W; x++) {
                int bq = qk[(long)y * W + x];
                double s = 0.0;
                long n = 0;
                for (int py = y - r; py <= y + r; py++)
                    for (int px = x - r; px <= x + r; px++)
                        if (py >= 0 && py < H && px >= 0 && px < W) {
                            s += E[((long)py * W + px) * B + bq];
                            n++;
                        }
                double a = s / (double)n;
                if (comp)
                    comp[(long)k * N + (long)y * W + x] = a;
                raw[(long)y * W + x] += a;
            }
    }
    for (long p = 0; p < N; p++)
        raw[p] /= (double)d;
    if (orc_blur(raw, H, W, sigma_s, score) < 0)
        goto oom;
    free(E);
    free(L);
    free(Rk);
    free(En);
    free(Ev);
    free(Qv);
    return 0;
oom:
    free(E);
    free(L);
    free(Rk);
    free(En);
    free(Ev);
    free(Qv);
    return -1;
}

/* ------------------------------------------------------------ median reference */

static int cmp_u8(const void *a, const void *b)
{
    return (int)*(const uint8_t *)a - (int)*(const uint8_t *)b;
}

/* The median reference (Sec. 3.2): for each component, every full window
 * (centre at least r from each border, T^2 = (2r+1)^2 pixels) is sorted, and
 * for each rank m the reference's m-th value is the median over the windows of
 * their m-th smallest value; the reference is then the histogram of those T^2
 * values (R[k][b], N_ref = T^2).  The median is the lower median (the
 * ceil(Np/2)-th smallest of the Np windows' values).  Works on bin indices:
 * a non-decreasing quantiser commutes with order statistics, so the median of
 * the quantised values is the quantised median of the values.  Returns 0, -1 on
 * allocation failure, -2 when no full window exists (H or W <= 2r). */
int orc_median_ref(const uint8_t *q, int d, int H, int W, int B, int r, uint32_t *R)
{
    if (H <= 2 * r || W <= 2 * r)
        return -2;
    long N = (long)H * W;
    int T = 2 * r + 1, T2 = T * T;
    long Np = (long)(H - 2 * r) * (W - 2 * r);
    uint8_t *o = (uint8_t *)malloc((size_t)Np * T2);
    uint8_t *col = (uint8_t *)malloc((size_t)Np);
    if (!o || !col) {
        free(o);
        free(col);
        return -1;
    }
    for (int k = 0; k < d; k++) {
        const uint8_t *qk = q + (long)k * N;
        long p = 0;
        for (int y = r; y < H - r; y++)
            for (int x = r; x < W - r; x++, p++) {
                uint8_t *w = o + p * T2;
                int n = 0;
                for (int yy = y - r; yy <= y + r; yy++)
                    for (int xx = x - r; xx <= x + r; xx++)
                        w[n++] = qk[(long)yy * W + xx];
                qsort(w, (size_t)T2, 1, cmp_u8);
            }
        for (int b = 0; b < B; b++)
            R[(long)k * B + b] = 0;
        for (int m = 0; m < T2; m++) {
            for (long i = 0; i < Np; i++)
                col[i] = o[i * T2 + m];
            qsort(col, (size_t)Np, 1, cmp_u8);
            int med = col[(Np + 1) / 2 - 1];
            R[(long)k * B + med]++;
        }
    }
    free(o);
    free(col);
    return 0;
}

/* ------------------------------------------------------------ QFCA+ residual */

/* The QFCA+ feature preprocessing (Sec. 3.3): the features minus their PCA
 * reconstruction from the top dres components,
 *     F(X) = X - PCA^-1(PCA(X)) = (X - mean) - (X - mean) V V^T,
 * computed channel by channel in FP64 (the mean cancels: the reconstruction
 * adds it back).  V is [C][dres] (columns orthonormal).  Writes Fres[C][N]. */
void orc_residual(const float *X, int layout, int H, int W, int C, const double *mean, const double *V, int dres,
                  double *Fres)
{
    long N = (long)H * W;
    double *y = (double *)malloc(sizeof(double) * (dres > 0 ? dres : 1));
    if (!y)
        return;
    for (long p = 0; p < N; p++) {
        for (int k = 0; k < dres; k++) {
            double s = 0.0;
            for (int c = 0; c < C; c++)
                s += (feat(X, layout, C, N, c, p) - mean[c]) * V[(long)c * dres + k];
            y[k] = s;
        }
        for (int c = 0; c < C; c++) {
            double rec = 0.0;
            for (int k = 0; k < dres; k++)
                rec += V[(long)c * dres + k] * y[k];
            Fres[(long)c * N + p] = (feat(X, layout, C, N, c, p) - mean[c]) - rec;
        }
    }
    free(y);
}
