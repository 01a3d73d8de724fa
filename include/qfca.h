/*
 * qfca.h -- C ABI of libqfca.so, the GB300 (sm_103a) implementation of the
 * hot path of quantized feature correspondence analysis (QFCA, arXiv
 * 2510.15602): PCA projection of a dense feature map, per-component uniform
 * quantisation, per-pixel sliding-window histograms and the 1-D earth mover's
 * distance to a reference histogram, averaged over components into a score
 * map.
 *
 * Conventions (all entry points):
 *  - Every function returns a qfca_status.  Arguments are validated on the
 *    host before anything is enqueued; an invalid argument returns
 *    QFCA_ERR_INVALID_ARG and enqueues nothing.
 *  - Tensor arguments are DEVICE pointers owned by the caller unless stated
 *    otherwise.  The library owns only the context, its workspace (device
 *    scratch memory it allocates itself) and the resident class table.
 *  - Work is enqueued asynchronously on the caller's CUDA stream (`stream`,
 *    a cudaStream_t passed as void*, NULL = legacy default stream).  Results
 *    are valid once that stream has reached the enqueued work.
 *  - Calls that share one context share its workspace: issue them on one
 *    stream (or synchronise between streams).  Use one context per stream for
 *    concurrent single-image calls, or the batch / serving entry points.
 *  - A CUDA error (launch failure, device fault) returns QFCA_ERR_CUDA; it is
 *    sticky: destroy the context.  Messages: qfca_status_string(),
 *    qfca_last_error().  No C++ exception crosses this ABI.
 *
 * Notation (the paper's, Sec. 3): feature map F(I) in R^{C x H x W};
 * d principal components; B quantisation bins ("N" in Sec. 3.1); window
 * radius r (patch size 2r+1); reference histogram R_k[b] with mass N_ref;
 * local window histogram P_k[b] with mass N_loc (the window clipped to the
 * image).
 */
#ifndef QFCA_H
#define QFCA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int qfca_status;
#define QFCA_OK 0
#define QFCA_PENDING 1
#define QFCA_ERR_INVALID_ARG (-1)
#define QFCA_ERR_UNSUPPORTED (-2)
#define QFCA_ERR_OOM (-3)
#define QFCA_ERR_CUDA (-4)
#define QFCA_ERR_TIMEOUT (-5)
#define QFCA_ERR_BUSY (-6)

/* Feature-map layouts.  NCHW = [C][H][W] (channel planes), NHWC = [H][W][C]. */
#define QFCA_NCHW 0
#define QFCA_NHWC 1

/* Projection precisions.  All accumulate in FP32. */
#define QFCA_F32 0       /* FP32 SIMT FFMA */
#define QFCA_BF16 1      /* BF16 operands on tcgen05 tensor cores */
#define QFCA_FP8_E4M3 2  /* e4m3 operands: (x - mean) s_c per channel, and the basis V/s_c as an
                            e4m3 hi + lo pair scaled per component; all scales powers of two
                            (s_c from a pass over max |x|); NCHW maps with H*W % 4 == 0 and a
                            16-byte aligned X only (else QFCA_ERR_UNSUPPORTED); not in serving */

/* Quantisation ranges. */
#define QFCA_RANGE_IMAGE 0  /* lo/hi = each component's min/max over the image */
#define QFCA_RANGE_FIXED 1  /* lo/hi given by the caller; values clamped */

typedef struct qfca_ctx qfca_ctx;

/* One FP32 feature map F(I) (Sec. 3.1: F(I) in R^{C x H x W}). */
typedef struct {
    int H, W, C;
    int layout; /* QFCA_NCHW or QFCA_NHWC */
} qfca_fmap;

/* A PCA basis (Sec. 3.3): device pointers, FP64.
 *   mean    [C]      channel means
 *   V       [C][d]   row-major; column k is principal axis k (unit norm,
 *                    sign: largest-magnitude entry positive)
 *   eigvals [d]      descending eigenvalues of the 1/N covariance        */
typedef struct {
    double *mean;
    double *V;
    double *eigvals;
} qfca_basis;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device`.  `workspace_bytes` is the initial
 * workspace size (0 = a default); the workspace grows on demand (a blocking
 * cudaMalloc) the first time a larger problem arrives, so warm up once per
 * shape before timing or graph capture.  *out receives the context. */
qfca_status qfca_create(int device, size_t workspace_bytes, qfca_ctx **out);

/* Destroy a context and free its workspace (synchronises the device). */
qfca_status qfca_destroy(qfca_ctx *ctx);

/* Static description of a status code. */
const char *qfca_status_string(qfca_status s);

/* Last error message recorded on `ctx` ("" if none).  Valid until the next
 * call on the same context. */
const char *qfca_last_error(const qfca_ctx *ctx);

/* Library version string. */
const char *qfca_version(void);

/* ---------------------------------------------------------------- the path */

/* qfca_fit_pca -- single-image PCA fit (Sec. 3.3; the paper fits PCA on the
 * features of the one input image).
 *   X     device FP32 feature map described by `desc`.
 *   d     number of components, 1 <= d <= min(C, 64).
 *   out   device pointers receiving mean[C], V[C][d], eigvals[d] (FP64).
 * Computes mu = (1/N) sum_p x_p and Sigma = (1/N) sum_p (x_p - mu)(x_p - mu)^T
 * as qfca_covariance does (an FP32-class covariance: each entry within
 * 2^-25 R_i R_j of the exact one, R_c the channel's power-of-two range), then
 * the top-d eigenpairs of that Sigma.  For C <= 256 and d <= 32: FP32
 * Householder tridiagonalisation, multisection on the Sturm count, inverse
 * iteration and back-transformation in one CTA per matrix, then one Newton
 * correction per eigenvector whose residual A x - sigma x is formed in
 * float-float (pairs of FP32 words, about 48 bits), and float-float Rayleigh
 * quotients as eigenvalues; a matrix whose relative residual
 * |A x - lambda x| / |x| exceeds the context's tolerance (default 1e-10) times
 * |lambda_max| is solved again by the float-float solver below.  Otherwise
 * (and for those matrices): float-float Householder tridiagonalisation on a
 * thread-block cluster, multisection, inverse iteration,
 * back-transformation.  FP64 in and out.
 * Requires 2 <= C <= 512 and 2 <= H*W <= 2^23. */
qfca_status qfca_fit_pca(qfca_ctx *ctx, const float *X, qfca_fmap desc, int d,
                         const qfca_basis *out, void *stream);

/* qfca_covariance -- mean[C] and covariance Sigma[C][C] (FP64, full symmetric
 * storage, 1/N normalisation) of a feature map: the first half of the PCA fit
 * (Sec. 3.3).  Computed with exact integer arithmetic on the BF16 tensor
 * cores: each channel is scaled by a power of two and written as four signed
 * 7-bit digits (a 27-bit fixed-point value, per-element error <= 2^-28 of the
 * channel's power-of-two range), digit products are summed exactly, and the
 * level sums are combined in int64 (which bounds H*W to 2^23 pixels).
 * Requires 2 <= C <= 512, 2 <= H*W <= 2^23. */
qfca_status qfca_covariance(qfca_ctx *ctx, const float *X, qfca_fmap desc, double *mean_out,
                            double *cov_out, void *stream);

/* qfca_quantize -- projection Y = (X - mean) V (Sec. 3.3) followed by uniform
 * quantisation of each component into B equally spaced bins (Sec. 3.1) and
 * the reference histogram.
 *   precision   QFCA_F32, QFCA_BF16 or QFCA_FP8_E4M3 (FP32 accumulation in all).
 *   range_mode  QFCA_RANGE_IMAGE: lo_k/hi_k = min/max of component k;
 *               QFCA_RANGE_FIXED: lo_in/hi_in (device f32[d]) are used and
 *               values are clamped into [0, B-1].
 *   bins        device u8 [d][H][pitch]; pitch >= W and a multiple of 16.
 *               q = (int)(((y - lo)/(hi - lo)) * B) in FP32, clamped to
 *               [0, B-1]; hi == lo gives 0.
 *   lo_out, hi_out   device f32[d] (may be NULL).
 *   ref_hist_out     device u32 [d][B] (may be NULL): R_k[b] = #{p : q_kp = b}.
 *   Y_out            device f32 [d][H*W] (may be NULL): the projection.
 * Requires 2 <= B <= 255, d <= 64. */
qfca_status qfca_quantize(qfca_ctx *ctx, const float *X, qfca_fmap desc, const qfca_basis *basis,
                          int d, int B, int precision, int range_mode, const float *lo_in,
                          const float *hi_in, uint8_t *bins, int pitch, float *lo_out,
                          float *hi_out, uint32_t *ref_hist_out, float *Y_out, void *stream);

/* qfca_quantize_residual -- the QFCA+ features (Sec. 3.3) and their per-channel
 * quantisation: with the basis of qfca_fit_pca fitted with dres components,
 *   F = (X - mean) - (X - mean) V V^T        (all C channels, FP32),
 * the input minus its PCA reconstruction; then each channel is quantised into
 * B equally spaced bins between its image-wide min and max (as qfca_quantize,
 * range mode IMAGE) with its global histogram as reference.  Score the result
 * with qfca_score / qfca_score_assoc with d = C.
 *   basis          mean f64[C], V f64[C][dres] (column k = component k).
 *   bins           device u8 [C][H][pitch], 16-byte aligned, pitch >= W and a
 *                  multiple of 16.
 *   lo_out, hi_out device f32 [C] (may be NULL): the channel ranges.
 *   ref_hist_out   device u32 [C][B] (may be NULL).
 *   F_out          device f32 [C][H*W] (may be NULL): the residual features.
 * Requires 0 <= dres <= min(C, 32), C <= 512, 2 <= B <= 255. */
qfca_status qfca_quantize_residual(qfca_ctx *ctx, const float *X, qfca_fmap desc, const qfca_basis *basis,
                                   int dres, int B, uint8_t *bins, int pitch, float *lo_out, float *hi_out,
                                   uint32_t *ref_hist_out, float *F_out, void *stream);

/* qfca_score -- per-pixel window histogram and 1-D EMD against the
 * reference, averaged over the d components (Sec. 3.1; W1 closed form in
 * the supplement).  For pixel p with clipped window of N_loc pixels:
 *   D_k(p) = sum_{b=0}^{B-1} |cumP_b * N_ref - cumR_b * N_loc|   (exact),
 *   score(p) = (sum_k D_k(p)) / (d * N_loc * N_ref)              (FP32 out).
 * Units: lo = hi = NULL measures distances in bins (bins a and b are |a - b|
 * apart).  With lo, hi (device f32 [d], each component's quantisation range,
 * e.g. qfca_quantize's lo_out/hi_out) distances are those of the quantized
 * values, as Sec. 3.1 states Algorithm 1's cost: |a - b| w_k with
 * w_k = (hi_k - lo_k) / B (FP64), and
 *   score(p) = (sum_k w_k D_k(p)) / (d * N_loc * N_ref)   (FP64 sum, FP32 out).
 *   bins       device u8 [d][H][pitch], 16-byte aligned, pitch >= W and a
 *              multiple of 16 (tiles are staged by TMA); values >= B are
 *              treated as B-1.
 *   ref_hist   device u32 [d][B]; every row sums to ref_total = N_ref.
 *   score      device f32 [H][W].
 *   numer_out  device u64 [d][H][W] or NULL: the exact D_k(p).
 * Requires 1 <= r, 2 <= B <= 255, (2r+1) <= 127, d <= 512 (d planes: the
 * components, or all C channels of qfca_quantize_residual). */
qfca_status qfca_score(qfca_ctx *ctx, const uint8_t *bins, int H, int W, int pitch, int d, int B,
                       int r, const uint32_t *ref_hist, uint32_t ref_total, float *score,
                       uint64_t *numer_out, const float *lo, const float *hi, void *stream);

/* qfca_score_assoc -- the paper's own per-pixel scoring (Sec. 3.1):
 *   1. Algorithm 1 for every window and component: the window histogram P
 *      (clipped (2r+1)^2 window, N_loc pixels) is transported onto the
 *      reference R at the common mass N_loc * N_ref by the two-pointer walk
 *      over the bins; E_i = (mass moved out of bin i x bin distance) /
 *      (P_i N_ref), in bin units (0 for empty bins);
 *   2. the error-to-pixel association with sigma_p = infinity: pixel q of bin
 *      b takes E_i[b] from every window that contains it and averages them
 *      (a box average over the window centres within r of q);
 *   3. the mean over the d components, then a Gaussian smoothing with
 *      standard deviation sigma_s (separable, taps |t| <= ceil(4 sigma_s),
 *      weights renormalised over the taps inside the image).
 * The per-bin errors are rounded to a fixed point 2^-s (s <= 20, the largest
 * with (2r+1)^2 (B-1) 2^s < 2^32) so the association sums are exact; the one
 * rounding of each E_i is the only error before the final division.
 *   bins       device u8 [d][H][pitch], pitch >= W; values >= B count as B-1.
 *   ref_hist   device u32 [d][B]; every row sums to ref_total = N_ref.
 *   sigma_s    0 <= sigma_s <= 4 (0: no smoothing; the paper uses 1).
 *   score      device f32 [H][W].
 *   raw_out    device f32 [H][W] or NULL: the map before smoothing.
 *   comp_out   device f32 [d][H][W] or NULL: each component's associated
 *              error (the map before the mean over components).
 *   lo, hi     NULL: bin units (|Q_i - Q_j| = |i - j|).  Device f32 [d], each
 *              component's quantisation range: value units, the cost Sec. 3.1
 *              states (|Q_i - Q_j| = |i - j| (hi_k - lo_k) / B), applied to
 *              the exact bin-unit sums in FP64 before the component mean.
 * Requires 1 <= r, 2 <= B <= 255, d <= 512, 2r <= 248 (B <= 32), 2r <= 120
 * (B <= 128), 2r <= 56 (B <= 255), and a shared-memory plan (histograms and
 * running sums for the window columns, (2r+1)^2 reciprocals) within 200 KB
 * (r <= 31 always fits for B <= 64); QFCA_ERR_UNSUPPORTED otherwise. */
qfca_status qfca_score_assoc(qfca_ctx *ctx, const uint8_t *bins, int H, int W, int pitch, int d, int B,
                             int r, const uint32_t *ref_hist, uint32_t ref_total, float sigma_s,
                             float *score, float *raw_out, float *comp_out, const float *lo,
                             const float *hi, void *stream);

/* One image of qfca_score_assoc_batch (fields as in qfca_score_assoc). */
typedef struct {
    const uint8_t *bins;       /* device u8 [d][H][pitch] */
    int H, W, pitch, r;
    const uint32_t *ref_hist;  /* device u32 [d][B] */
    uint32_t ref_total;
    float *score;              /* device f32 [H][W], written */
    float *raw;                /* device f32 [H][W] or NULL */
    const float *lo, *hi;      /* device f32 [d] each, or NULL: value or bin units */
} qfca_assoc_image;

/* qfca_score_assoc_batch -- qfca_score_assoc for n images (own sizes and
 * radii, common d, B and sigma_s), each stage one launch per 64 images.
 * Results equal n single-image calls.  Requires 1 <= n <= 4096. */
qfca_status qfca_score_assoc_batch(qfca_ctx *ctx, const qfca_assoc_image *imgs, int n, int d, int B,
                                   float sigma_s, void *stream);

/* qfca_median_reference -- the median reference (Sec. 3.2): for each component,
 * every full window (centre at least r from each border, T^2 = (2r+1)^2
 * pixels) is sorted, and the reference's m-th value, m = 1..T^2, is the lower
 * median over the windows (the ceil(Np/2)-th smallest of the Np windows'
 * m-th values).  The result is their histogram, ref_out[k][b] (each row sums
 * to T^2: pass ref_total = (2r+1)^2 to qfca_score / qfca_score_assoc).  Bin
 * indices are used directly: a non-decreasing quantiser commutes with order
 * statistics, so this equals quantising the median of the unquantised values.
 *   bins     device u8 [d][H][pitch], pitch >= W; values >= B count as B-1.
 *   ref_out  device u32 [d][B], written.
 * Requires H > 2r, W > 2r, 1 <= r, 2 <= B <= 255, d <= 512, and the count table
 * of B x (T^2 + 1) words plus 32 window histograms within 200 KB of shared
 * memory (r <= 19 for B = 32, r <= 13 for B = 64, r <= 5 for B = 255);
 * QFCA_ERR_UNSUPPORTED otherwise.  Exact (integer). */
qfca_status qfca_median_reference(qfca_ctx *ctx, const uint8_t *bins, int H, int W, int pitch, int d, int B,
                                  int r, uint32_t *ref_out, void *stream);

/* One image of qfca_median_reference_batch (fields as in qfca_median_reference). */
typedef struct {
    const uint8_t *bins;  /* device u8 [d][H][pitch] */
    int H, W, pitch, r;
    uint32_t *ref_out;    /* device u32 [d][B], written */
} qfca_median_image;

/* qfca_median_reference_batch -- qfca_median_reference for n images (own sizes
 * and radii, common d and B), one launch per stage per 64 images.
 * Requires 1 <= n <= 4096. */
qfca_status qfca_median_reference_batch(qfca_ctx *ctx, const qfca_median_image *imgs, int n, int d, int B,
                                        void *stream);

/* qfca_metrics -- the evaluation of Sec. 4.2 for nimg score maps and their
 * ground-truth masks, after discarding `border` pixels on each side of every
 * map (the paper discards a border of the size of the window radius):
 *   out[0]  pixel AUROC over the kept pixels of all maps (Mann-Whitney, ties
 *           counting one half);
 *   out[1]  F1 at the optimal threshold (maximum of 2 TP / (predicted +
 *           anomalous) over every distinct score, score >= threshold
 *           predicting an anomaly);
 *   out[2]  AUPRO: the per-region overlap curve (false-positive rate over the
 *           normal pixels; mean over the 8-connected anomalous regions of
 *           every cropped mask of the fraction of the region at or above the
 *           threshold) integrated by trapezoids from (0, 0) up to fpr_limit,
 *           linearly interpolated there, divided by fpr_limit;
 *   out[3]  image-level AUROC of the maximum of each cropped map, an image
 *           being anomalous when its (whole) mask has an anomalous pixel.
 * NaN where a class is empty.  Every distinct score is a threshold (-0 and
 * +0 being one score; scores must not be NaN), so the curves are exact;
 * integer counts are exact and the FP64 sums use a fixed order
 * (deterministic results).
 *   scores  device f32 [nimg][H][W];  masks device u8 [nimg][H][W], non-zero =
 *   anomalous;  out device double[4].
 * Requires 1 <= nimg <= 4096, 2 border < H and < W, 0 < fpr_limit <= 1 and at
 * most 2^22 kept pixels per call (QFCA_ERR_UNSUPPORTED above).  Uses the
 * context's workspace (about 40 bytes per kept pixel). */
qfca_status qfca_metrics(qfca_ctx *ctx, const float *scores, const uint8_t *masks, int nimg, int H, int W, int border,
                         double fpr_limit, double *out, void *stream);

/* Synchronise the device and read-and-clear the context's device status
 * word.  Kernels whose bounded waits (on tensor-core completion, on a peer
 * stage) run out set bit 0 (value 1) there and return early instead of
 * hanging; the metric suite's union-find sets bit 4 (value 16) when one of its
 * loops reaches its iteration limit (its results are then not valid).
 * *out receives the word; returns QFCA_ERR_TIMEOUT when it was non-zero. */
qfca_status qfca_device_status(qfca_ctx *ctx, int *out);

/* Optional outputs of qfca_batch_run (each pointer may be NULL; the library
 * then keeps that intermediate in its workspace).  Per-image blocks are packed
 * image after image:
 *   mean [nimg][C], V [nimg][C][d], eigvals [nimg][d]  (FP64, as qfca_fit_pca)
 *   bins [nimg][d][H][pitch], 16-byte aligned, `pitch` >= W and a multiple of 16 (ignored when
 *        bins is NULL), ref_hist [nimg][d][B], lo/hi [nimg][d]. */
typedef struct {
    double *mean;
    double *V;
    double *eigvals;
    uint8_t *bins;
    int pitch;
    uint32_t *ref_hist;
    float *lo;
    float *hi;
} qfca_batch_outputs;

/* qfca_batch_run -- the whole path (Sec. 3.3 fit and projection, Sec. 3.1
 * quantisation, window histograms and EMD, channel mean) for nimg feature
 * maps of one shape stored one after the other in X (image i starts at
 * X + i*C*H*W), with each stage launched once for the whole batch: the
 * covariance tiles, eigensolver clusters, projection tiles, quantisation bands
 * and window tiles of every image share one grid.  Quantisation ranges are
 * each component's image-wide min/max; the reference of each image is its
 * own global histogram (N_ref = H*W).
 *   scores  device f32 [nimg][H][W].
 * Given the same bases, results equal nimg separate calls of qfca_quantize and
 * qfca_score bit for bit (same kernels, same arithmetic).  The FP32 + Newton
 * eigensolver (C <= 256, d <= 32) works on one matrix per CTA, so its bases do
 * not depend on the batch; the float-float solver (larger shapes, and matrices
 * that fail the residual check) grows its cluster size while the launch leaves
 * SMs free, which changes the order of its reductions with the number of
 * matrices: its bases agree with qfca_fit_pca's to about 1e-12 relative.
 * Requires 1 <= nimg <= 4096 and the limits of those entry points. */
qfca_status qfca_batch_run(qfca_ctx *ctx, const float *X, int nimg, qfca_fmap desc, int d, int B, int r,
                           int precision, float *scores, const qfca_batch_outputs *extra, void *stream);

/* qfca_batch_run_host -- qfca_batch_run with the feature maps and the score
 * maps in host memory: the end-to-end call of the batch path.  On `stream` it
 * enqueues the copy of X_host [nimg][C][H][W] (the layout of desc) into a
 * device staging buffer the context owns, the whole path of qfca_batch_run
 * (per-image fit, projection, quantisation, window EMD; Sec. 3.1, 3.3), and
 * the copy of the score maps into scores_host [nimg][H][W] (FP32); one
 * cudaMemcpyAsync each way.  Host buffers should be page-locked (pinned): then
 * the copies are asynchronous and the call can be captured in a CUDA graph;
 * pageable buffers work outside capture, with copies that wait for the host.
 * The staging buffer (4 (C + 1) H W bytes per image) grows on a larger call
 * and is freed with the context; it cannot grow during stream capture (run
 * the call once before capturing).  The host buffers must stay valid until
 * the stream reaches the call's end.  Same limits as qfca_batch_run. */
qfca_status qfca_batch_run_host(qfca_ctx *ctx, const float *X_host, int nimg, qfca_fmap desc, int d, int B, int r,
                                int precision, float *scores_host, void *stream);

/* qfca_batch_run_basis -- qfca_batch_run with the PCA bases already fitted
 * (the basis-resident part of the path: Sec. 3.3 projection, Sec. 3.1
 * quantisation with image-wide ranges and each image's own global histogram
 * as reference, window histograms and EMD, channel mean).
 *   mean  device f64 [nimg][C], V device f64 [nimg][C][d] (column k =
 *         component k), e.g. from qfca_fit_pca or qfca_batch_run's extra
 *         outputs; read, not written.
 *   extra as qfca_batch_run (mean, V and eigvals there are ignored).
 * Results equal qfca_batch_run's given the same bases, bit for bit. */
qfca_status qfca_batch_run_basis(qfca_ctx *ctx, const float *X, int nimg, qfca_fmap desc, const double *mean,
                                 const double *V, int d, int B, int r, int precision, float *scores,
                                 const qfca_batch_outputs *extra, void *stream);

/* qfca_batch_run_plus -- QFCA+ (Sec. 3.3) for nimg feature maps of one shape
 * stored one after the other in X: each image's PCA fitted with dres
 * components (Sec. 3.3 fit), its residual features over all C channels (the
 * input minus its PCA reconstruction, qfca_quantize_residual), each channel
 * quantised between its image-wide min and max with its global histogram as
 * reference (Sec. 3.1), and the window EMD averaged over all C channels; each
 * stage is one launch for the batch (the residual features of the batch are
 * kept in the workspace: 4 C H W bytes per image).
 *   scores  device f32 [nimg][H][W].
 *   extra   as qfca_batch_run with d = dres for mean, V, eigvals and d = C for
 *           bins [nimg][C][H][pitch], ref_hist [nimg][C][B], lo/hi [nimg][C].
 * Requires 1 <= dres <= min(C, 32), C <= 512, 2 <= B <= 255, 1 <= r <= 63,
 * 1 <= nimg <= 4096. */
qfca_status qfca_batch_run_plus(qfca_ctx *ctx, const float *X, int nimg, qfca_fmap desc, int dres, int B, int r,
                                float *scores, const qfca_batch_outputs *extra, void *stream);

/* One image of an uneven batch (qfca_score_batch). */
typedef struct {
    const float *X; /* device feature map, C channels in the batch's layout,
                       16-byte aligned for the TMA-fed BF16 projection */
    int H, W;       /* size, H*W >= 2 */
    int r;          /* window radius of this image, 1 <= r <= 63 */
    float *score;   /* device f32 [H][W], written */
} qfca_image;

/* qfca_score_batch -- the whole path of qfca_batch_run for n images of
 * different sizes and window radii (same C, layout, d, B, precision): each
 * image gets its own PCA fit (Sec. 3.3), image-wide quantisation ranges and
 * its own global histogram as reference (Sec. 3.1).  Every stage is one
 * persistent launch over a table of up to 64 images (more images: one launch
 * per 64), so the whole batch can be captured in one CUDA graph.  Results
 * equal n separate single-image calls (same kernels, same arithmetic).  With
 * autotuning on (qfca_set_autotune), the first call for a new set of shapes
 * outside stream capture times the window stage's candidate tilings and
 * keeps the fastest for later calls.  Requires 1 <= n <= 4096 and the limits
 * of the single-image entry points. */
qfca_status qfca_score_batch(qfca_ctx *ctx, const qfca_image *imgs, int n, int C, int layout, int d, int B,
                             int precision, void *stream);

/* Autotuning for qfca_score_batch and qfca_batch_run (and qfca_batch_run_basis):
 * the window stage's tiling (strip width, band height, components per CTA)
 * and the BF16 projection's ring depths (FP32 feature boxes in flight,
 * converted operand chunks ahead of the tensor cores).  0 = the built-in cost
 * model and the deepest rings that fit (default), 1 = measure the candidates
 * once per shape set (blocking, never under stream capture) and reuse the
 * fastest.  Results do not depend on either choice. */
qfca_status qfca_set_autotune(qfca_ctx *ctx, int mode);

/* The ring depths used by the context's most recent TMA-fed projection
 * (0, 0 before the first): FP32 feature boxes in flight and converted operand
 * chunks. */
qfca_status qfca_last_projection_tiling(qfca_ctx *ctx, int *stages, int *operand_buffers);

/* Use a given window-stage tiling for the context's later score launches
 * (strip width 64 or 128 threads, band height 1..64 rows, component groups
 * >= 1; more groups than components count as one per component), ahead of
 * the cost model and the autotuner; strip_width = 0 returns to them.  With
 * one component group each CTA sums all d components of its pixels in shared
 * memory and writes the score itself (bin units, no numerator output);
 * otherwise the per-component numerators go through a finalisation launch.
 * Results do not depend on the tiling.  A tiling that does not fit shared
 * memory for a call makes that call return QFCA_ERR_UNSUPPORTED. */
qfca_status qfca_set_tiling(qfca_ctx *ctx, int strip_width, int band_height, int component_groups);

/* The window-stage tiling used by the context's most recent score launch:
 * strip width (threads), band height (rows), component groups. */
qfca_status qfca_last_tiling(qfca_ctx *ctx, int *strip_width, int *band_height, int *component_groups);

/* The CDF walk of the window stage: the per-pixel sum over bins of
 * |cumP_b N_ref - cumR_b N_loc| (the W1 closed form of the supplement applied
 * to the histograms of Sec. 3.1).
 *   walk -1  default: the autotuner measures both walks where both exist and
 *            keeps the faster; without autotuning the per-thread walk runs;
 *         0  per thread: each thread walks the B bins of its own pixel in order;
 *         1  warp-shuffle segmented: two lanes per pixel walk 16 bins each, the
 *            lower half's count reaches the upper lane by a shuffle as its CDF
 *            offset and the partial sums are added by shuffles.  It exists for
 *            B = 32 with 32-bit numerators ((B-1)(2r+1)^2 N_ref < 2^32); other
 *            calls run the per-thread walk.
 * Applies to later score launches of the context, with a tiling set by
 * qfca_set_tiling or the cost model's.  The numerators are exact integers, so
 * results do not depend on the walk.  QFCA_ERR_INVALID_ARG outside [-1, 1]. */
qfca_status qfca_set_cdf_walk(qfca_ctx *ctx, int walk);

/* The CDF walk (0 per thread, 1 warp-shuffle) of the context's most recent
 * score launch. */
qfca_status qfca_last_cdf_walk(qfca_ctx *ctx, int *walk);

/* Bands per CTA of a tiling set by qfca_set_tiling: each CTA then takes a run
 * of that many consecutive bands of its strip and component group, and the
 * window histograms of Sec. 3.1 slide on from one band into the next (only the
 * first band of a run builds its windows from scratch), while the next band's
 * tile is fetched.  bands = 1 (default) is one band per CTA, 0 every band of
 * the strip.  With one component group (the fused form) a CTA takes one band.
 * The cost model and the autotuner choose the run themselves.  Results do not
 * depend on it.  QFCA_ERR_INVALID_ARG outside [0, 4096]. */
qfca_status qfca_set_band_run(qfca_ctx *ctx, int bands);

/* The bands per CTA of the context's most recent score launch. */
qfca_status qfca_last_band_run(qfca_ctx *ctx, int *bands);

/* qfca_score_noalloc -- the same computation as qfca_score (without the
 * optional numerator output), for callers that cannot allocate device memory:
 * code that runs under a host application or memory manager that owns every
 * device allocation, inside a process with a hard device-memory budget, or
 * in a latency-critical loop where the implicit synchronisation of
 * cudaMalloc/cudaFree is not acceptable.  It takes no context (creating one
 * allocates) and calls no cudaMalloc, cudaFree or allocating library routine.
 * The paper has no counterpart; this is an interface convenience.
 *
 * Its scratch (the per-pixel sums of the EMD numerators, 8 bytes per pixel)
 * is one file-scope device array of 4 MiB in the library, present on every
 * GPU that loads the library until the process exits.  Hence:
 *  - images are limited to H*W <= 524288 pixels; larger ones return
 *    QFCA_ERR_UNSUPPORTED without enqueuing anything;
 *  - every call shares that array (each call clears the pixels it uses on its
 *    stream before accumulating): calls that overlap on the GPU (on different
 *    streams, or from different threads, without ordering between them) race
 *    and give wrong results; serialise them on one stream;
 *  - work runs on the calling thread's current CUDA device; all pointers
 *    must belong to it.  Each call looks up the array's device address for
 *    that device (a lookup, no allocation; the first call on a device may
 *    load the library's module there, so make it before any CUDA stream
 *    capture).
 * Arguments, layouts and the result are those of qfca_score (d up to 512
 * planes); invalid arguments return QFCA_ERR_INVALID_ARG, CUDA errors
 * QFCA_ERR_CUDA.  A bounded wait inside the kernel that runs out is not
 * reported by this call (it returns before the work runs): it sets a status
 * word that qfca_score_noalloc_status reads. */
qfca_status qfca_score_noalloc(const uint8_t *bins, int H, int W, int pitch, int d, int B, int r,
                               const uint32_t *ref_hist, uint32_t ref_total, float *score,
                               void *stream);

/* Read and clear the status word of qfca_score_noalloc on the current device,
 * ordered after the work already enqueued on `stream` (the call waits for that
 * stream).  *out receives the word: 0 when every bounded wait of the calls
 * since the last read completed, non-zero when one ran out (that call's score
 * map is incomplete).  Returns QFCA_OK, QFCA_ERR_TIMEOUT (word non-zero) or
 * QFCA_ERR_CUDA.  Allocates nothing. */
qfca_status qfca_score_noalloc_status(int *out, void *stream);

/* Testing aid for the timeout report of qfca_score_noalloc: with
 * give_up_at_once != 0, each CTA's first tile wait in later calls gives up
 * without probing (the kernel then waits for its copies in flight, sets the
 * status word and returns, leaving that map incomplete); 0 restores the
 * normal limit.  Process-wide; not for production use. */
qfca_status qfca_score_noalloc_test_wait_limit(int give_up_at_once);

/* ---------------------------------------------------------------- serving
 *
 * A serving session keeps per-class PCA bases, quantisation ranges and
 * reference histograms resident on the device and scores single images as
 * they arrive (the paper's per-texture setting of Sec. 4: one reference per
 * texture class, fitted once).  Requests wait in a FIFO queue; a scheduler
 * thread admits them to the GPU as device memory (a fixed arena) and stream
 * slots free up, packs the admitted ones into one table-driven batch (one
 * launch per stage for up to max_batch images of mixed sizes and radii) and
 * keeps several batches in flight on separate streams, so requests that
 * arrive while others run start as soon as resources allow (continuous
 * batching).  A request's result does not depend on what it was batched with.
 * Per image: projection with the class basis (BF16 or FP32), quantisation
 * with the class's fixed range (values outside clamp to the end bins), the
 * window EMD against the class reference (N_ref = its total), the component
 * mean. */

typedef struct {
    int C, d, B;               /* shared by every class and request of the session */
    int precision;             /* QFCA_F32 or QFCA_BF16 */
    int max_batch;             /* images per launched batch, 1..64 */
    int streams;               /* batches in flight at once, 1..8 */
    int max_queue;             /* pending requests before submit answers QFCA_ERR_BUSY */
    size_t arena_bytes;        /* device memory for in-flight requests (admission budget) */
} qfca_serve_config;

#define QFCA_REQ_HOST_INPUT 1  /* X is pinned host memory (copied in on the batch's stream) */
#define QFCA_REQ_HOST_OUTPUT 2 /* score is pinned host memory (copied out on the batch's stream) */

typedef struct {
    int class_id;
    const float *X;            /* [C][H][W] FP32, NCHW; device unless QFCA_REQ_HOST_INPUT */
    int H, W;
    int r;                     /* window radius, 1..63 */
    float *score;              /* [H][W] FP32 out; device unless QFCA_REQ_HOST_OUTPUT */
    int flags;
} qfca_request;

typedef struct {
    int status;                /* qfca_status of the request */
    int batch_size;            /* images in the batch it ran in */
    double t_submit_us;        /* host steady-clock stamps, microseconds since the session started */
    double t_start_us;         /* batch launched */
    double t_done_us;          /* batch completed on the GPU (stream callback) */
    int stream;                /* index of the session stream the batch ran on (0 .. streams-1) */
    int reserved;
    uint64_t batch_seq;        /* sequence number of the batch in the session (1, 2, ...) */
} qfca_result;

/* Start the session's scheduler (one per context).  Allocates the arena and
 * the streams; QFCA_ERR_OOM when the arena cannot be allocated. */
qfca_status qfca_serve_start(qfca_ctx *ctx, const qfca_serve_config *cfg);

/* Copy a class into the session: mean [C] and V [C][d] (FP64, column k =
 * component k, as qfca_fit_pca writes them), the fixed range lo/hi [d] and the
 * reference histogram ref_hist [d][B] with N_ref = ref_total; all device
 * pointers, read before the call returns.  Re-registering an id replaces it
 * (requests already admitted keep the old copy until they finish). */
qfca_status qfca_register_class(qfca_ctx *ctx, int class_id, const double *mean, const double *V,
                                const float *lo, const float *hi, const uint32_t *ref_hist,
                                uint32_t ref_total);

/* Queue one request (non-blocking).  *ticket identifies it for qfca_poll.
 * QFCA_ERR_BUSY: the queue is full (retry later); QFCA_ERR_UNSUPPORTED: the
 * request can never fit the arena; QFCA_ERR_INVALID_ARG: bad request or
 * unknown class.  The caller keeps X and score alive until poll returns OK. */
qfca_status qfca_submit(qfca_ctx *ctx, const qfca_request *req, uint64_t *ticket);

/* Wait up to timeout_us (0: just look) for a request.  QFCA_OK: done, *out
 * filled and the ticket retired; QFCA_PENDING: not yet; QFCA_ERR_INVALID_ARG:
 * unknown ticket. */
qfca_status qfca_poll(qfca_ctx *ctx, uint64_t ticket, int timeout_us, qfca_result *out);

/* Drain every queued and in-flight request, then stop the scheduler and free
 * the session's device memory.  Unpolled results are discarded.  No other
 * serving call on the context may run concurrently with this one. */
qfca_status qfca_serve_stop(qfca_ctx *ctx);

/* Residual bound of the fit's FP32 + Newton eigensolver, relative to the
 * largest eigenvalue (default 1e-10): matrices above it are solved again by
 * the float-float solver.  0 sends every matrix to the float-float solver.
 * Applies to later fits on this context.  tol >= 0. */
qfca_status qfca_set_eig_tolerance(qfca_ctx *ctx, double tol);

/* Synchronise the device, then read and clear the number of matrices that the
 * float-float solver solved again (see qfca_set_eig_tolerance) since the last
 * read. */
qfca_status qfca_eig_redo_count(qfca_ctx *ctx, uint64_t *out);

/* ---------------------------------------------------------------- tracing */

/* Number of kernels the library has launched through `ctx` since creation
 * (every entry point counts its own launches; memsets are not counted). */
qfca_status qfca_launch_count(qfca_ctx *ctx, uint64_t *out);

/* Start timing kernel launches on `ctx`: every launch whose kernel name
 * contains `filter` (all kernels when filter is "" or NULL) is bracketed by
 * two CUDA events recorded on the launch's stream.  Clears earlier records. */
qfca_status qfca_trace_start(qfca_ctx *ctx, const char *filter);

/* Stop recording (records are kept until the next qfca_trace_start). */
qfca_status qfca_trace_stop(qfca_ctx *ctx);

/* Entry i (0-based) of the trace, aggregated per kernel name: name (copied
 * into name_out, at most 63 chars + NUL), total device time in ms and launch
 * count.  Synchronises on the recorded events.  Returns QFCA_ERR_INVALID_ARG
 * when i is past the last entry. */
qfca_status qfca_trace_get(qfca_ctx *ctx, int i, char *name_out, double *total_ms, uint64_t *launches);

#ifdef __cplusplus
}
#endif

#endif /* QFCA_H */
