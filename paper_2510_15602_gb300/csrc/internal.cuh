// internal.cuh -- declarations shared by the translation units of libqfca.so.
// Not part of the public ABI (include/qfca.h is).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>
#include <string>

#include "../../include/qfca.h"

namespace qfca {

constexpr int kMaxC = 512;   // channels supported by the fit and projection
constexpr int kMaxD = 64;    // components of a PCA projection
constexpr int kMaxPlanes = 512;  // bin planes scored per image (components, or all channels for QFCA+)
constexpr int kMaxResidual = 32;  // components removed by the QFCA+ residual
constexpr int kMaxB = 255;   // bins
// Images per launch of the table-driven stages (the table travels in the
// kernel's parameter block).
constexpr int kMaxBatch = 64;

// Once-per-device setup of a launcher's kernel attributes (dynamic shared
// memory limits, carve-outs, SM counts).  Launchers run on the caller's thread
// and on serving scheduler threads, so the record is taken under a mutex; a
// device's bit is set only after its setup succeeded (a failure is retried on
// the next launch).  Devices are numbered below 64.
struct DeviceOnce {
    std::mutex mu;
    uint64_t done = 0;
};

template <class F>
cudaError_t device_once(DeviceOnce &o, int dev, F &&setup) {
    std::lock_guard<std::mutex> lk(o.mu);
    const uint64_t bit = 1ull << (dev & 63);
    if (o.done & bit) return cudaSuccess;
    const cudaError_t e = setup();
    if (e == cudaSuccess) o.done |= bit;
    return e;
}

// ------------------------------------------------------------------ fit (fit.cu)

// Batched entry points take `nimg` images of one shape stored one after the
// other (feature maps C*H*W floats apart; per-image outputs likewise packed).

// Workspace bytes needed by the fit of nimg C-channel maps of N pixels.
// One image of a table-driven fit: feature map X (layout of the launch), N pixels.
struct FitJob {
    const float *X;
    long N;
};
cudaError_t launch_gram_cov_jobs(const FitJob *jobs, int n, int layout, int C, double *mean, double *cov, void *cov_ff,
                                 void *ws, int *status, cudaStream_t st);
// max |x| per channel (float bits) of each image: amax [n][C]
cudaError_t launch_chan_absmax_jobs(const FitJob *jobs, int n, int layout, int C, unsigned *amax, cudaStream_t st);
// Residual bound of the FP32 + Newton eigensolver relative to the largest
// eigenvalue; matrices above it are solved again by the float-float solver.
constexpr float kEigTolDefault = 1e-10f;
// Slot (in ints) of the context's status allocation that counts the matrices
// the float-float solver redid.
constexpr int kRedoCountSlot = 16;

cudaError_t launch_fit_jobs(const FitJob *jobs, int n, int layout, int C, int d, double *mean, double *V,
                            double *eigvals, void *ws, int *status, cudaStream_t st, float eig_tol = kEigTolDefault);

size_t fit_workspace_bytes(int C, long N, int d, int nimg);

// Enqueue the PCA fit of nimg images.  ws: device scratch of fit_workspace_bytes.
cudaError_t launch_fit(const float *X, int layout, int H, int W, int C, int d, int nimg,
                       double *mean, double *V, double *eigvals, void *ws, int *status, cudaStream_t st,
                       float eig_tol = kEigTolDefault);

// Mean and covariance of one feature map (gram.cu).
size_t gram_workspace_bytes(int C, long N, int nimg);
// cov_ff (may be NULL): the covariance also as float-float pairs (float2 [C][C]).
cudaError_t launch_gram_cov(const float *X, int layout, int C, long N, int nimg, double *mean, double *cov,
                            void *cov_ff, void *ws, int *status, cudaStream_t st);

// Top-d eigenpairs of `mats` symmetric n x n matrices given as float-float
// pairs (float2 [mats][n][n]) (eig.cu): the FP32 + Newton solver (eig32.cu)
// where the shape allows it, the float-float solver for the matrices it flags
// (and for every matrix of larger shapes).  status: the context's status
// allocation (the redo counter lives at status[kRedoCountSlot]) or NULL.
size_t eig_workspace_bytes(int n, int d, int mats);
cudaError_t launch_eig(const void *cov_ff, int n, int d, int mats, double *V, double *eigvals, void *ws,
                       int *status, cudaStream_t st, float tol = kEigTolDefault);
bool eig32_ok(int n, int d);
size_t eig32_workspace_bytes(int n, int mats);
cudaError_t launch_eig32(const void *cov_ff, int n, int d, int mats, double *V, double *eigvals, void *ws,
                         int *flag_out, int *redo_count, float tol, cudaStream_t st);

// ------------------------------------------------------------------ projection (project.cu)

size_t project_workspace_bytes(int C, long N, int d, int nimg);

// Y[k][p] = sum_c (x_cp - mean_c) V[c][k] in FP32 (precision QFCA_F32) or with
// BF16 operands on tcgen05 (QFCA_BF16); also the per-component min/max
// (as order-preserving u32 keys in mm_keys[2*d]).
// Y [nimg][d][N]; mm_keys [nimg][2 d kKeyStride]; mean/V per image packed.
cudaError_t launch_project(const float *X, int layout, int H, int W, int C, const double *mean,
                           const double *V, int d, int nimg, int precision, float *Y, uint32_t *mm_keys,
                           void *ws, int *status, cudaStream_t st);

// One image of the TMA-fed projection: X NCHW [C][N] (16-B aligned, N % 4 ==
// 0), prepared operands mean32 [Cp] and Vt (BF16 [DT][Cp]; FP8: the e4m3 hi
// then lo parts [2][DT][Cp], Cp = C rounded to 128, with the per-channel
// scale s_c [Cp] and the per-component 1/t_j [DT], all powers of two), Y
// [d][N], min/max keys mm [2 d kKeyStride] (initialised by the caller).
struct ProjJob {
    const float *X;
    long N;
    const float *mean32;
    const void *Vt;
    float *Y;
    uint32_t *mm;
    const float *scale = nullptr;
    const float *colscale = nullptr;
    // Fixed-range quantisation in the epilogue (bins given): bins [d][N / W][pitch] with
    // quant_bin(y, qlo[k], qhi[k], B) instead of Y and the min/max keys.
    const float *qlo = nullptr, *qhi = nullptr;
    uint8_t *bins = nullptr;
    int W = 0, pitch = 0, B = 0;
};
bool project_tma_ok(const float *X, long N, int layout);
size_t project_bf16_workspace_bytes(int C, long N, int d, int nimg);
size_t project_fp8_workspace_bytes(int C, int d, int nimg);
cudaError_t launch_project_fp8(const float *X, int layout, long N, int C, const double *mean, const double *V, int d,
                               int nimg, float *Y, uint32_t *mm_keys, void *ws, int *status, cudaStream_t st);
cudaError_t launch_prep_bf16(const double *mean, const double *V, int C, int d, int n, void *ws, float **mean32_out,
                             void **Vt_out, int *Cp_out, int *DT_out, cudaStream_t st);
// min/max keys of nimg images (contiguous [nimg][2 d kKeyStride]) to their start values
cudaError_t launch_init_keys(uint32_t *mm_keys, int d, int nimg, cudaStream_t st);
cudaError_t launch_project_tma(const ProjJob *jobs, int n, int C, int d, bool fp8, int *status, cudaStream_t st);

// Ring depths of the TMA-fed projection: FP32 feature boxes in flight (stages)
// and converted operand chunks ahead of the MMAs (na).  The launcher picks the
// deepest that fit shared memory unless the calling thread has set
// tl_proj_tiling (the API's autotuner does, around a call); the results do not
// depend on it.
struct ProjTiling {
    int stages, na;
};
extern thread_local const ProjTiling *tl_proj_tiling;
// The candidates that fit shared memory for (C, d); the depths the last launch on this thread used.
int project_tilings(int C, int d, bool fp8, ProjTiling *out, int max_out);
ProjTiling project_last_tiling();

// Per-component min/max keys live 128 B apart (one L2 line each):
// min of component j at mm_keys[j * kKeyStride], max at mm_keys[(d + j) * kKeyStride].
constexpr int kKeyStride = 32;

// Device status word bits (set by kernels; read by qfca_device_status).
constexpr int kStatusMmaTimeout = 1;
constexpr int kStatusMetricsLimit = 1 << 4;  // the metric suite's union-find ran out of its iteration limit

// ------------------------------------------------------------------ quantize (quantize.cu)

// bins [nimg][d][H][pitch], hist [nimg][d][B], lo/hi out [nimg][d]; fixed ranges are shared.
cudaError_t launch_quantize(const float *Y, long N, int H, int W, int d, int nimg, int B, int range_mode,
                            const uint32_t *mm_keys, const float *lo_in, const float *hi_in,
                            uint8_t *bins, int pitch, float *lo_out, float *hi_out,
                            uint32_t *hist, cudaStream_t st);

// One image of a table-driven quantisation: Y [d][H*W]; image range from the
// min/max keys mm (or, when mm is NULL, the fixed range lo_in/hi_in [d]);
// bins [d][H][pitch]; lo_out/hi_out [d] and hist [d][B] optional.
struct QuantJob {
    const float *Y;
    int H, W;
    const uint32_t *mm;
    const float *lo_in, *hi_in;
    uint8_t *bins;
    int pitch;
    float *lo_out, *hi_out;
    uint32_t *hist;
};
// zero_hist: clear each job's hist first (else the caller has).
cudaError_t launch_quantize_jobs(const QuantJob *jobs, int n, int d, int B, bool zero_hist, cudaStream_t st);

// ------------------------------------------------------------------ score (score.cu)

// One image of a score launch: bins [d][H][pitch] (16-B aligned, pitch a
// multiple of 16), reference [d][B] with N_ref = Nref, score [H][W],
// numer_out [d][H][W] u64 (optional).
struct ScoreJob {
    const uint8_t *bins;
    int H, W, pitch, r;
    const uint32_t *ref;
    uint32_t Nref;
    float *score;
    uint64_t *numer_out;
    // Value units: each component's quantisation range [d] (NULL: bin units).
    // Component k then weighs (hi_k - lo_k) / B per unit of bin distance.
    const float *lo = nullptr, *hi = nullptr;
};

// Tiling of the window-EMD kernel: strip width SW (64 or 128 threads), band
// height TH (1..64 rows) and number of component groups n_kg.
struct ScoreTiling {
    int SW, TH, n_kg;
    int walk;   // CDF walk of the interior pixels: 0 per thread, 1 warp-shuffle segmented (B = 32, u32 walk only)
    int bands;  // bands per CTA (a run of consecutive bands; the window carries over): 0 = every band of a strip
};

// Workspace of launch_score_jobs: the numerators D_k(p) of every job (or, when
// accumulating, their per-pixel sums).
size_t score_jobs_workspace_bytes(const ScoreJob *jobs, int n, int d);

// True when some tiling fits B bins and radius r in shared memory.
bool score_shape_ok(int B, int r);

// Window EMD + score of n images (one launch per kMaxBatch images).  tiling
// NULL: the built-in cost model picks one (written to *chosen when given).
// cudaErrorNotSupported: nothing was enqueued.
cudaError_t launch_score_jobs(const ScoreJob *jobs, int n, int d, int B, void *ws, bool ws_accumulates, int *status,
                              cudaStream_t st, const ScoreTiling *tiling, ScoreTiling *chosen);
// The same with a given probe limit for each CTA's first tile wait (the
// allocation-free path's timeout test gives 0).
cudaError_t launch_score_jobs_limited(const ScoreJob *jobs, int n, int d, int B, void *ws, bool ws_accumulates,
                                      int *status, cudaStream_t st, const ScoreTiling *tiling, ScoreTiling *chosen,
                                      uint32_t first_wait_tries);

// One image of the paper's scoring (assoc.cu): bins [d][H][pitch], reference
// [d][B] with N_ref = Nref, window radius r, final smoothing sigma_s (<= 0:
// none, at most 4); score [H][W]; raw [H][W] (before smoothing) and comp
// [d][H][W] (per-component associated errors) optional.
struct AssocJob {
    const uint8_t *bins;
    int H, W, pitch, r;
    const uint32_t *ref;
    uint32_t Nref;
    float sigma_s;
    float *score, *raw, *comp;
    const float *lo = nullptr, *hi = nullptr;  // value units as in ScoreJob (NULL: bin units)
};

// True when B bins and radius r fit the association kernel.
bool assoc_shape_ok(int B, int r);
size_t assoc_jobs_workspace_bytes(const AssocJob *jobs, int n, int d);
// Algorithm 1 + association + mean + smoothing for n images.  Returns
// cudaErrorNotSupported (nothing enqueued) when the shape does not fit and
// cudaErrorInvalidValue for sigma_s > 4.
cudaError_t launch_assoc_jobs(const AssocJob *jobs, int n, int d, int B, void *ws, cudaStream_t st);

// One image of the median reference (median.cu): bins [d][H][pitch], window
// radius r (H, W > 2r); ref_out [d][B] receives the histogram of the per-rank
// lower medians over the full windows (N_ref = (2r+1)^2).
struct MedianJob {
    const uint8_t *bins;
    int H, W, pitch, r;
    uint32_t *ref_out;
};

bool median_shape_ok(int B, int r);
size_t median_jobs_workspace_bytes(const MedianJob *jobs, int n, int d, int B);
// cudaErrorNotSupported (nothing enqueued) when B and r do not fit;
// cudaErrorInvalidValue when an image has no full window.
cudaError_t launch_median_jobs(const MedianJob *jobs, int n, int d, int B, void *ws, cudaStream_t st);

// QFCA+ residual features F = (X - mean) - (X - mean) V V^T over all C
// channels of nimg same-shaped images (residual.cu): per image X [C][N],
// mean [C], V [C][dres], F [C][N] f32 and min/max keys [2 C kKeyStride]
// (initialised here), packed image after image.  0 <= dres <= kMaxResidual.
cudaError_t launch_residual(const float *X, int layout, int H, int W, int C, const double *mean, const double *V,
                            int dres, int nimg, float *F, uint32_t *mm, cudaStream_t st);

// ------------------------------------------------------------------ context access (api.cu) for serve.cu

struct ServeState;
ServeState *&ctx_serve(qfca_ctx *ctx);
int ctx_device(qfca_ctx *ctx);
int *ctx_status_dev(qfca_ctx *ctx);
std::mutex &ctx_mutex(qfca_ctx *ctx);
qfca_status ctx_set_error(qfca_ctx *ctx, qfca_status s, const std::string &msg);
bool ctx_sticky(qfca_ctx *ctx);

// ------------------------------------------------------------------ TMA (tmap.cu)

// Encode a 3-D u8 tiled tensor map (no swizzle, zero fill out of bounds) into
// the 128-byte CUtensorMap at tmap_out.  dim0 is innermost.
cudaError_t make_tmap_u8_3d(void *tmap_out, const void *base, uint64_t dim0, uint64_t dim1, uint64_t dim2,
                            uint64_t stride1_bytes, uint64_t stride2_bytes, uint32_t box0, uint32_t box1);

// 2-D FP32 tiled tensor map (zero fill out of bounds); dim0 innermost.
// swizzle128: 128-byte swizzle in shared memory (the box's inner extent must
// be 128 bytes; 16-B chunk c of box row r lands at chunk c ^ (r & 7)).
cudaError_t make_tmap_f32_2d(void *tmap_out, const void *base, uint64_t dim0, uint64_t dim1, uint64_t stride1_bytes,
                             uint32_t box0, uint32_t box1, bool swizzle128 = false);

// ------------------------------------------------------------------ evaluation metrics (metrics.cu)

// Pixel AUROC, F1 max, AUPRO to fpr_limit and image-level AUROC of nimg maps (out: device double[4]).
long metrics_max_pixels();
size_t metrics_workspace_bytes(int nimg, int H, int W, int border);
cudaError_t launch_metrics(const float *scores, const uint8_t *masks, int nimg, int H, int W, int border,
                           double fpr_limit, double *out, void *ws, int *status, cudaStream_t st);

// ------------------------------------------------------------------ helpers

// Order-preserving map float -> u32 (larger float -> larger key).
__host__ __device__ inline uint32_t f2key(float f) {
    uint32_t u;
#ifdef __CUDA_ARCH__
    u = __float_as_uint(f);
#else
    memcpy(&u, &f, 4);
#endif
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__host__ __device__ inline float key2f(uint32_t k) {
    uint32_t u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float f;
    memcpy(&f, &u, 4);
    return f;
#endif
}

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

#ifdef __CUDACC__
// The image of a table-driven launch that owns index x (a CTA, block or tile):
// the last i in [0, n) with first(i) <= x, for first() non-decreasing and
// first(0) <= x.  Binary search: about log2(n) parameter loads instead of up to
// n - 1 in a scan.
template <class F>
__device__ __forceinline__ int table_image(int n, long x, F first) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (first(mid) <= x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}
#endif

// The bin of value y among B equally spaced bins between lo and hi (Sec. 3.1),
// decided in FP32 with IEEE-rounded operations in a fixed order:
//     t = (y - lo) / (hi - lo);  v = t * B;  q = clamp((int)v, 0, B-1);  hi == lo gives 0.
// Every kernel that quantises uses this function, so their bins agree bit for bit.
#ifdef __CUDACC__
__device__ __forceinline__ int quant_bin(float y, float lo, float hi, float fB, int B) {
    if (!(hi > lo)) return 0;
    const float t = __fdiv_rn(__fsub_rn(y, lo), __fsub_rn(hi, lo));
    const float v = __fmul_rn(t, fB);
    int q = v < 0.0f ? 0 : (int)v;
    return q > B - 1 ? B - 1 : q;
}
#endif

// ------------------------------------------------------------------ launch hook (tracing)

// Called around every kernel launch while an entry point runs on a context.
struct LaunchHook {
    virtual void before(const char *kernel, cudaStream_t st) = 0;
    virtual void after(const char *kernel, cudaStream_t st) = 0;
    virtual ~LaunchHook() = default;
};
extern thread_local LaunchHook *tl_hook;

#define QFCA_LAUNCH(kname, st, ...)                            \
    do {                                                       \
        if (::qfca::tl_hook) ::qfca::tl_hook->before(kname, st); \
        __VA_ARGS__;                                           \
        if (::qfca::tl_hook) ::qfca::tl_hook->after(kname, st);  \
    } while (0)

}  // namespace qfca
