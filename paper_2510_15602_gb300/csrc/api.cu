// api.cu -- host side of the C ABI (include/qfca.h): context, workspace,
// argument validation, and the enqueueing of the kernels on the caller's
// stream.  No C++ exception crosses the ABI; every entry point returns a
// qfca_status and records a message on the context.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>

#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "internal.cuh"

namespace qfca {
thread_local LaunchHook *tl_hook = nullptr;
}

namespace {

// Counts every launch; brackets launches whose kernel name matches the filter
// with CUDA events on the launch stream.
struct Tracer final : qfca::LaunchHook {
    uint64_t launches = 0;
    bool active = false;
    bool pending = false;
    std::string filter;
    struct Rec {
        const char *name;
        cudaEvent_t a, b;
    };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    size_t pool_used = 0;
    // aggregated view (filled by trace_get)
    std::vector<std::string> agg_name;
    std::vector<double> agg_ms;
    std::vector<uint64_t> agg_n;
    bool agg_valid = false;

    cudaEvent_t take() {
        if (pool_used == pool.size()) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
            pool.push_back(e);
        }
        return pool[pool_used++];
    }
    // While the stream is being captured into a CUDA graph the events must be
    // recorded as graph nodes (external records), so each replay re-records them.
    static void record(cudaEvent_t e, cudaStream_t st) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
            cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
        else
            cudaEventRecord(e, st);
    }
    void before(const char *k, cudaStream_t st) override {
        launches++;
        pending = false;
        if (!active) return;
        if (!filter.empty() && !strstr(k, filter.c_str())) return;
        Rec r{k, take(), take()};
        if (!r.a || !r.b) return;
        record(r.a, st);
        recs.push_back(r);
        pending = true;
        agg_valid = false;
    }
    void after(const char *, cudaStream_t st) override {
        if (pending) record(recs.back().b, st);
        pending = false;
    }
    void reset() {
        recs.clear();
        pool_used = 0;
        agg_valid = false;
    }
    cudaError_t aggregate() {
        if (agg_valid) return cudaSuccess;
        agg_name.clear();
        agg_ms.clear();
        agg_n.clear();
        for (const Rec &r : recs) {
            cudaError_t e = cudaEventSynchronize(r.b);
            if (e != cudaSuccess) return e;
            float ms = 0.f;
            e = cudaEventElapsedTime(&ms, r.a, r.b);
            if (e == cudaErrorInvalidResourceHandle || e == cudaErrorNotReady) {
                // events captured into a graph that has not been replayed yet were never recorded
                cudaGetLastError();
                continue;
            }
            if (e != cudaSuccess) return e;
            size_t i = 0;
            while (i < agg_name.size() && agg_name[i] != r.name) i++;
            if (i == agg_name.size()) {
                agg_name.emplace_back(r.name);
                agg_ms.push_back(0.0);
                agg_n.push_back(0);
            }
            agg_ms[i] += ms;
            agg_n[i] += 1;
        }
        agg_valid = true;
        return cudaSuccess;
    }
    ~Tracer() override {
        for (cudaEvent_t e : pool) cudaEventDestroy(e);
    }
};

}  // namespace

struct qfca_ctx {
    int device = 0;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    void *io = nullptr;                                 // device staging of qfca_batch_run_host (features, maps)
    size_t io_bytes = 0;
    int *status_dev = nullptr;  // device status word (bits set by kernels)
    bool sticky = false;
    std::string err;
    std::mutex mu;
    Tracer tracer;
    int autotune = 0;                                   // window-stage tiling: 0 model, 1 measured
    std::map<std::string, qfca::ScoreTiling> tuned;     // measured tilings per shape set
    qfca::ScoreTiling last_tiling{0, 0, 0};
    qfca::ScoreTiling forced{0, 0, 0};                  // window-stage tiling set by the caller (SW 0: none)
    int walk_mode = -1;                                 // CDF walk: -1 the autotuner's choice (else per thread), 0, 1
    int band_run = 1;                                   // bands per CTA of a forced tiling (0: a strip's every band)
    std::map<std::string, qfca::ProjTiling> proj_tuned; // measured projection ring depths per shape set
    qfca::ProjTiling last_proj{0, 0};
    float eig_tol = qfca::kEigTolDefault;               // residual bound of the FP32 + Newton eigensolver
    qfca::ServeState *serve = nullptr;                  // serving session (serve.cu)
};

namespace qfca {
ServeState *&ctx_serve(qfca_ctx *ctx) { return ctx->serve; }
int ctx_device(qfca_ctx *ctx) { return ctx->device; }
int *ctx_status_dev(qfca_ctx *ctx) { return ctx->status_dev; }
std::mutex &ctx_mutex(qfca_ctx *ctx) { return ctx->mu; }
qfca_status ctx_set_error(qfca_ctx *ctx, qfca_status s, const std::string &msg) {
    ctx->err = msg;
    if (s == QFCA_ERR_CUDA) ctx->sticky = true;
    return s;
}
bool ctx_sticky(qfca_ctx *ctx) { return ctx->sticky; }
}  // namespace qfca

namespace {

using namespace qfca;

// Installs the context's tracer as the launch hook for the current call.
struct HookScope {
    qfca::LaunchHook *prev;
    explicit HookScope(qfca_ctx *ctx) : prev(qfca::tl_hook) { qfca::tl_hook = &ctx->tracer; }
    ~HookScope() { qfca::tl_hook = prev; }
};

struct DeviceGuard {
    int prev = -1;
    bool changed = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) changed = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        if (changed) cudaSetDevice(prev);
    }
};

qfca_status fail(qfca_ctx *ctx, qfca_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (ctx) {
        ctx->err = buf;
        if (s == QFCA_ERR_CUDA) ctx->sticky = true;
    }
    return s;
}

qfca_status cuda_fail(qfca_ctx *ctx, cudaError_t e, const char *where) {
    return fail(ctx, QFCA_ERR_CUDA, "%s: %s (%s)", where, cudaGetErrorName(e), cudaGetErrorString(e));
}

// Grow the context workspace to at least `need` bytes (blocking; frees the old
// one).  Growing is not possible while `st` is being captured into a graph:
// the caller must run the same call once outside capture first.
qfca_status ensure_ws(qfca_ctx *ctx, size_t need, cudaStream_t st = nullptr) {
    if (need <= ctx->ws_bytes) return QFCA_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (st && cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
        return fail(ctx, QFCA_ERR_INVALID_ARG,
                    "the workspace must grow to %zu bytes during stream capture: run the call once before capturing",
                    need);
    if (ctx->ws) {
        cudaError_t e = cudaFree(ctx->ws);
        ctx->ws = nullptr;
        ctx->ws_bytes = 0;
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaFree(workspace)");
    }
    size_t sz = align_up(need + need / 4, 1 << 20);
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, sz);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, QFCA_ERR_OOM, "workspace of %zu bytes: %s", sz, cudaGetErrorString(e));
    }
    ctx->ws = p;
    ctx->ws_bytes = sz;
    return QFCA_OK;
}

qfca_status check_ctx(qfca_ctx *ctx) {
    if (!ctx) return QFCA_ERR_INVALID_ARG;
    if (ctx->sticky) return fail(ctx, QFCA_ERR_CUDA, "context has a sticky CUDA error: %s", ctx->err.c_str());
    return QFCA_OK;
}

qfca_status check_fmap(qfca_ctx *ctx, const float *X, const qfca_fmap &m) {
    if (!X) return fail(ctx, QFCA_ERR_INVALID_ARG, "X is NULL");
    if (m.layout != QFCA_NCHW && m.layout != QFCA_NHWC) return fail(ctx, QFCA_ERR_INVALID_ARG, "bad layout %d", m.layout);
    if (m.H < 1 || m.W < 1 || (long)m.H * m.W < 2) return fail(ctx, QFCA_ERR_INVALID_ARG, "bad H x W = %d x %d", m.H, m.W);
    if ((long)m.H * m.W > (1L << 23)) return fail(ctx, QFCA_ERR_UNSUPPORTED, "H*W = %ld > 2^23 pixels", (long)m.H * m.W);
    if (m.C < 2 || m.C > kMaxC) return fail(ctx, QFCA_ERR_UNSUPPORTED, "C = %d outside [2, %d]", m.C, kMaxC);
    return QFCA_OK;
}

size_t bytes_mmkeys(int d) { return align_up(sizeof(uint32_t) * 2 * d * kKeyStride, 256); }

bool capturing(cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
}

// The window stage of a batch, with the context's tiling policy: the cost
// model, or (autotune) the fastest of the candidate tilings measured once per
// shape set on this stream (outside capture), reused afterwards.
qfca_status run_score(qfca_ctx *ctx, const ScoreJob *jobs, int n, int d, int B, void *ws, cudaStream_t st,
                      const char *where) {
    const ScoreTiling *use = nullptr;
    ScoreTiling chosen{0, 0, 0};
    if (ctx->forced.SW > 0) {
        chosen = ctx->forced;
        chosen.walk = std::max(ctx->walk_mode, 0);
        chosen.bands = ctx->band_run;
        use = &chosen;
    } else if (ctx->walk_mode >= 0 && !ctx->autotune) {
        chosen = ScoreTiling{0, 0, 0, ctx->walk_mode};  // the cost model's tiling with this walk
        use = &chosen;
    } else if (ctx->autotune) {
        std::string key = std::to_string(n) + ":" + std::to_string(d) + ":" + std::to_string(B) + ":w" +
                          std::to_string(ctx->walk_mode);
        for (int i = 0; i < n; i++)
            key += ":" + std::to_string(jobs[i].H) + "x" + std::to_string(jobs[i].W) + "r" + std::to_string(jobs[i].r);
        auto it = ctx->tuned.find(key);
        if (it != ctx->tuned.end()) {
            chosen = it->second;
            use = &chosen;
        } else if (!capturing(st)) {
            cudaEvent_t a = nullptr, b = nullptr;
            if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess)
                return cuda_fail(ctx, cudaGetLastError(), "autotune events");
            float best_ms = 1e30f;
            ScoreTiling best{0, 0, 0};
            std::vector<ScoreTiling> cands;
            ScoreTiling model{0, 0, 0};
            const ScoreTiling model_walk{0, 0, 0, std::max(ctx->walk_mode, 0)};
            cudaError_t e = launch_score_jobs(jobs, n, d, B, ws, false, ctx->status_dev, st, &model_walk, &model);
            if (e != cudaSuccess) {
                cudaEventDestroy(a), cudaEventDestroy(b);
                return e == cudaErrorNotSupported ? fail(ctx, QFCA_ERR_UNSUPPORTED, "%s: no tiling fits", where)
                                                  : cuda_fail(ctx, e, where);
            }
            cands.push_back(model);
            // both CDF walks where the shuffle walk exists (B = 32), unless the caller fixed one
            std::vector<int> walks;
            if (ctx->walk_mode >= 0) walks.push_back(ctx->walk_mode);
            else walks = B == 32 ? std::vector<int>{0, 1} : std::vector<int>{0};
            // band runs of 1, 4 or every band of a strip (a fused tiling, one group, takes one band)
            for (int w : walks)
                for (int SW : {128, 64})
                    for (int TH : {8, 16, 32, 64})
                        for (int nk : {1, 2, 4, 8, 16, 32})
                            for (int br : {1, 4, 0})
                                if (nk <= d && (nk > 1 || br == 1)) cands.push_back(ScoreTiling{SW, TH, nk, w, br});
            for (const ScoreTiling &c : cands) {
                float tot = 0.0f;
                bool okc = true;
                for (int rep = 0; rep < 3 && okc; rep++) {
                    cudaEventRecord(a, st);
                    e = launch_score_jobs(jobs, n, d, B, ws, false, ctx->status_dev, st, &c, nullptr);
                    if (e == cudaErrorNotSupported) {
                        okc = false;
                        break;
                    }
                    if (e != cudaSuccess) {
                        cudaEventDestroy(a), cudaEventDestroy(b);
                        return cuda_fail(ctx, e, where);
                    }
                    cudaEventRecord(b, st);
                    if ((e = cudaEventSynchronize(b)) != cudaSuccess) {
                        cudaEventDestroy(a), cudaEventDestroy(b);
                        return cuda_fail(ctx, e, where);
                    }
                    float ms = 0.0f;
                    cudaEventElapsedTime(&ms, a, b);
                    if (rep > 0) tot += ms;  // the first run warms up
                }
                if (okc && tot < best_ms) best_ms = tot, best = c;
            }
            cudaEventDestroy(a), cudaEventDestroy(b);
            ctx->tuned[key] = best;
            chosen = best;
            use = &chosen;
        }
    }
    cudaError_t e = launch_score_jobs(jobs, n, d, B, ws, false, ctx->status_dev, st, use, &ctx->last_tiling);
    if (e == cudaErrorNotSupported) return fail(ctx, QFCA_ERR_UNSUPPORTED, "%s: no window tiling fits B = %d", where, B);
    if (e != cudaSuccess) return cuda_fail(ctx, e, where);
    return QFCA_OK;
}

// The projection of a call (`enqueue` initialises its own min/max keys, so it
// can run again) with the context's ring depths for `key`: with autotuning on,
// the candidates that fit are timed once per shape set on this stream (outside
// capture) and the fastest is kept.  Every candidate gives the same result.
template <class F>
cudaError_t run_projection(qfca_ctx *ctx, const std::string &key, int C, int d, cudaStream_t st, F &&enqueue) {
    ProjTiling chosen{0, 0};
    const ProjTiling *use = nullptr;
    if (ctx->autotune) {
        auto it = ctx->proj_tuned.find(key);
        if (it != ctx->proj_tuned.end()) {
            chosen = it->second;
            use = &chosen;
        } else if (!capturing(st)) {
            ProjTiling cand[32];
            const int nc = project_tilings(C, d, false, cand, 32);
            cudaEvent_t a = nullptr, b = nullptr;
            cudaError_t e = cudaEventCreate(&a);
            if (e == cudaSuccess) e = cudaEventCreate(&b);
            float best_ms = 1e30f;
            for (int i = 0; i < nc && e == cudaSuccess; i++) {
                tl_proj_tiling = &cand[i];
                float tot = 0.0f;
                for (int rep = 0; rep < 3 && e == cudaSuccess; rep++) {
                    e = cudaEventRecord(a, st);
                    if (e == cudaSuccess) e = enqueue();
                    if (e == cudaSuccess) e = cudaEventRecord(b, st);
                    if (e == cudaSuccess) e = cudaEventSynchronize(b);
                    float ms = 0.0f;
                    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
                    if (rep > 0) tot += ms;  // the first run warms up
                }
                if (e == cudaSuccess && tot < best_ms) best_ms = tot, chosen = cand[i];
            }
            tl_proj_tiling = nullptr;
            if (a) cudaEventDestroy(a);
            if (b) cudaEventDestroy(b);
            if (e != cudaSuccess) return e;
            if (nc > 0) {
                ctx->proj_tuned[key] = chosen;
                use = &chosen;
            }
        }
    }
    tl_proj_tiling = use;
    const cudaError_t e = enqueue();
    tl_proj_tiling = nullptr;
    ctx->last_proj = project_last_tiling();
    return e;
}

std::string shape_key(const char *what, int n, int C, int d, const std::vector<long> &sizes) {
    std::string k = std::string(what) + ":" + std::to_string(n) + ":" + std::to_string(C) + ":" + std::to_string(d);
    for (long s : sizes) k += ":" + std::to_string(s);
    return k;
}

}  // namespace

extern "C" {

const char *qfca_version(void) { return "qfca-gb300 0.1 (sm_103a)"; }

const char *qfca_status_string(qfca_status s) {
    switch (s) {
        case QFCA_OK: return "QFCA_OK";
        case QFCA_PENDING: return "QFCA_PENDING";
        case QFCA_ERR_INVALID_ARG: return "QFCA_ERR_INVALID_ARG";
        case QFCA_ERR_UNSUPPORTED: return "QFCA_ERR_UNSUPPORTED";
        case QFCA_ERR_OOM: return "QFCA_ERR_OOM";
        case QFCA_ERR_CUDA: return "QFCA_ERR_CUDA";
        case QFCA_ERR_TIMEOUT: return "QFCA_ERR_TIMEOUT";
        case QFCA_ERR_BUSY: return "QFCA_ERR_BUSY";
        default: return "QFCA_ERR_UNKNOWN";
    }
}

const char *qfca_last_error(const qfca_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

qfca_status qfca_create(int device, size_t workspace_bytes, qfca_ctx **out) {
    if (!out) return QFCA_ERR_INVALID_ARG;
    *out = nullptr;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return QFCA_ERR_CUDA;
    }
    if (device < 0 || device >= n) return QFCA_ERR_INVALID_ARG;
    qfca_ctx *ctx = new (std::nothrow) qfca_ctx();
    if (!ctx) return QFCA_ERR_OOM;
    ctx->device = device;
    DeviceGuard g(device);
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess) {
        delete ctx;
        return QFCA_ERR_CUDA;
    }
    if (prop.major * 10 + prop.minor < 100) {
        delete ctx;
        return QFCA_ERR_UNSUPPORTED;
    }
    const qfca_status s = ensure_ws(ctx, workspace_bytes ? workspace_bytes : (64u << 20));
    if (s != QFCA_OK) {
        delete ctx;
        return s;
    }
    if (cudaMalloc(&ctx->status_dev, 256) != cudaSuccess || cudaMemset(ctx->status_dev, 0, 256) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(ctx->ws);
        delete ctx;
        return QFCA_ERR_OOM;
    }
    *out = ctx;
    return QFCA_OK;
}

qfca_status qfca_destroy(qfca_ctx *ctx) {
    if (!ctx) return QFCA_ERR_INVALID_ARG;
    if (ctx->serve) qfca_serve_stop(ctx);
    {
        DeviceGuard g(ctx->device);
        if (ctx->ws || ctx->io || ctx->status_dev) cudaDeviceSynchronize();
        if (ctx->ws) cudaFree(ctx->ws);
        if (ctx->io) cudaFree(ctx->io);
        if (ctx->status_dev) cudaFree(ctx->status_dev);
    }
    delete ctx;
    return QFCA_OK;
}

qfca_status qfca_fit_pca(qfca_ctx *ctx, const float *X, qfca_fmap desc, int d, const qfca_basis *out,
                         void *stream) {
    qfca_status s = check_ctx(ctx);
    if (s) return s;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if ((s = check_fmap(ctx, X, desc))) return s;
    if (!out || !out->mean || !out->V || !out->eigvals) return fail(ctx, QFCA_ERR_INVALID_ARG, "basis pointers NULL");
    if (d < 1 || d > desc.C || d > kMaxD) return fail(ctx, QFCA_ERR_INVALID_ARG, "d = %d outside [1, min(C, %d)]", d, kMaxD);
    DeviceGuard g(ctx->device);
    HookScope hs(ctx);
    const long N = (long)desc.H * desc.W;
    if ((s = ensure_ws(ctx, fit_workspace_bytes(desc.C, N, d, 1), (cudaStream_t)stream))) return s;
    cudaError_t e = launch_fit(X, desc.layout, desc.H, desc.W, desc.C, d, 1, out->mean, out->V, out->eigvals, ctx->ws,
                               ctx->status_dev, (cudaStream_t)stream, ctx->eig_tol);
    if (e == cudaErrorNotSupported) return fail(ctx, QFCA_ERR_UNSUPPORTED, "eigensolver shape C=%d d=%d", desc.C, d);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "qfca_fit_pca");
    return QFCA_OK;
}

qfca_status qfca_covariance(qfca_ctx *ctx, const float *X, qfca_fmap desc, double *mean_out, double *cov_out,
                            void *stream) {
    qfca_status s = check_ctx(ctx);
    if (s) return s;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if ((s = check_fmap(ctx, X, desc))) return s;
    if (!mean_out || !cov_out) return fail(ctx, QFCA_ERR_INVALID_ARG, "mean_out / cov_out NULL");
    DeviceGuard g(ctx->device);
    HookScope hs(ctx);
    const long N = (long)desc.H * desc.W;
    if ((s = ensure_ws(ctx, gram_workspace_bytes(desc.C, N, 1), (cudaStream_t)stream))) return s;
    cudaError_t e = launch_gram_cov(X, desc.layout, desc.C, N, 1, mean_out, cov_out, nullptr, ctx->ws, ctx->status_dev,
                                    (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "qfca_covariance");
    return QFCA_OK;
}

qfca_status qfca_quantize(qfca_ctx *ctx, const float *X, qfca_fmap desc, const qfca_basis *basis, int d, int B,
                          int precision, int range_mode, const float *lo_in, const float *hi_in, uint8_t *bins,
                          int pitch, float *lo_out, float *hi_out, uint32_t *ref_hist_out, float *Y_out,
                          void *stream) {
    qfca_status s = check_ctx(ctx);
    if (s) return s;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if ((s = check_fmap(ctx, X, desc))) return s;
    if (!basis || !basis->mean || !basis->V) return fail(ctx, QFCA_ERR_INVALID_ARG, "basis NULL");
    if (d < 1 || d > desc.C || d > kMaxD) return fail(ctx, QFCA_ERR_INVALID_ARG, "d = %d outside [1, min(C, %d)]", d, kMaxD);
    if (B < 2 || B > kMaxB) return fail(ctx, QFCA_ERR_INVALID_ARG, "B = %d outside [2, %d]", B, kMaxB);
    if (precision != QFCA_F32 && precision != QFCA_BF16 && precision != QFCA_FP8_E4M3)
        return fail(ctx, QFCA_ERR_INVALID_ARG, "precision %d not available", precision);
    if (range_mode != QFCA_RANGE_IMAGE && range_mode != QFCA_RANGE_FIXED)
        return fail(ctx, QFCA_ERR_INVALID_ARG, "bad range_mode %d", range_mode);
    if (range_mode == QFCA_RANGE_FIXED && (!lo_in || !hi_in))
        return fail(ctx, QFCA_ERR_INVALID_ARG, "fixed range needs lo_in and hi_in");
    if (!bins) return fail(ctx, QFCA_ERR_INVALID_ARG, "bins NULL");
    if (pitch < desc.W || pitch % 16 != 0) return fail(ctx, QFCA_ERR_INVALID_ARG, "pitch %d must be >= W and a multiple of 16", pitch);
    DeviceGuard g(ctx->device);
    HookScope hs(ctx);
    const long N = (long)desc.H * desc.W;
    const size_t o_mm = 0;
    const size_t o_y = o_mm + bytes_mmkeys(d);
    const size_t o_p = o_y + (Y_out ? 0 : align_up(sizeof(float) * d * N, 256));
    if ((s = ensure_ws(ctx, o_p + project_workspace_bytes(desc.C, N, d, 1), (cudaStream_t)stream))) return s;
    char *base = (char *)ctx->ws;
    uint32_t *mm = (uint32_t *)(base + o_mm);
    float *Y = Y_out ? Y_out : (float *)(base + o_y);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = launch_project(X, desc.layout, desc.H, desc.W, desc.C, basis->mean, basis->V, d, 1, precision, Y,
                                   mm, base + o_p, ctx->status_dev, st);
    if (e == cudaErrorNotSupported) {
        cudaGetLastError();
        return fail(ctx, QFCA_ERR_UNSUPPORTED, "projection precision %d not supported for this shape", precision);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "qfca_quantize/project");
    e = launch_quantize(Y, N, desc.H, desc.W, d, 1, B, range_mode, mm, lo_in, hi_in, bins, pitch, lo_out, hi_out,
                        ref_hist_out, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "qfca_quantize/quantize");
    return QFCA_OK;
}

qfca_status qfca_score(qfca_ctx *ctx, const uint8_t *bins, int H, int W, int pitch, int d, int B, int r,
                       const uint32_t *ref_hist, uint32_t ref_total, float *score, uint64_t *numer_out,
                       const float *lo, const float *hi, void *stream) {
    qfca_status s = check_ctx(ctx);
    if (s) return s;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (!bins || !ref_hist || !score) return fail(ctx, QFCA_ERR_INVALID_ARG, "NULL pointer");
    if (H < 1 || W < 1) return fail(ctx, QFCA_ERR_INVALID_ARG, "bad H x W");
    if (pitch < W || pitch % 16 != 0) return fail(ctx, QFCA_ERR_INVALID_ARG, "pitch %d must be >= W and a multiple of 16", pitch);
    if (((uintptr_t)bins & 15) != 0) return fail(ctx, QFCA_ERR_INVALID_ARG, "bins must be 16-byte aligned");
    if (d < 1 || d > kMaxPlanes) return fail(ctx, QFCA_ERR_INVALID_ARG, "d = %d outside [1, %d]", d, kMaxPlanes);
    if (B < 2 || B > kMaxB) return fail(ctx, QFCA_ERR_INVALID_ARG, "B = %d outside [2, %d]", B, kMaxB);
    if (r < 1 || 2 * r + 1 > 127) return fail(ctx, QFCA_ERR_INVALID_ARG, "r = %d outside [1, 63]", r);
    if (ref_total < 1) return fail(ctx, QFCA_ERR_INVALID_ARG, "ref_total must be >= 1");
    if ((lo == nullptr) != (hi == nullptr)) return fail(ctx, QFCA_ERR_INVALID_ARG, "value units need both lo and hi");
    DeviceGuard g(ctx->device);
    HookScope hs(ctx);
    const ScoreJob job{bins, H, W, pitch, r, ref_hist, ref_total, score, numer_out, lo, hi};
    if ((s = ensure_ws(ctx, score_jobs_workspace_bytes(&job, 1, d), (cudaStream_t)stream))) return s;
    // the caller's tiling (or the cost model's) with the context's CDF walk
    const ScoreTiling tl{ctx->forced.SW, ctx->forced.TH, ctx->forced.n_kg, std::max(ctx->walk_mode, 0),
                         ctx->band_run};
    cudaError_t e = launch_score_jobs(&job, 1, d, B, ctx->ws, false, ctx->status_dev, (cudaStream_t)stream, &tl,
                                      &ctx->last_tiling);
    if (e == cudaErrorNotSupported)
        return fail(ctx, QFCA_ERR_UNSUPPORTED, "B = %d with r = %d needs more shared memory than a CTA has", B, r);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "qfca_score");
    return QFCA_OK;
}

qfca_status qfca_quantize_residual(qfca_ctx *ctx, const float *X, qfca_fmap desc, const qfca_basis *basis, int dres,
                                   int B, uint8_t *bins, int pitch, float *lo_out, float *hi_out,
                                   uint32_t *ref_hist_out, float *F_out, void *stream) {
    qfca_status s = check_ctx(ctx);
    if (s) return s;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if ((s = check_fmap(ctx, X, desc))) return s;
    if (!basis || !basis->mean || (dres > 0 && !basis->V)) return fail(ctx, QFCA_ERR_INVALID_ARG, "basis NULL");
    if (dres < 0 || dres > desc.C || dres > kMaxResidual)
        return fail(ctx, QFCA_ERR_INVALID_ARG, "dres = %d outside [0, min(C, %d)]", dres, kMaxResidual);
    if (desc.C > kMaxPlanes) return fail(ctx, QFCA_ERR_INVALID_ARG, "C = %d above %d", desc.C, kMaxPlanes);
    if (B < 2 || B > kMaxB) return fail(ctx, QFCA_ERR_INVALID_ARG, "B = %d outside [2, %d]", B, kMaxB);
    if (!bins) return fail(ctx, QFCA_ERR_INVALID_ARG, "bins NULL");
    if (pitch < desc.W || pitch % 16 != 0) return fail(ctx, QFCA_ERR_INVALID_ARG, "pitch %d must be >= W and a multiple of 16", pitch);
    DeviceGuard g(ctx->device);
    HookScope hs(ctx);
    const long N = (long)desc.H * desc.W;
    const int C = desc.C;
    const size_t o_f = bytes_mmkeys(C);
    if ((s = ensure_ws(ctx, o_f + (F_out ? 0 : align_up(sizeof(float) * C * N, 256)), (cudaStream_t)stream))) return s;
    char *base = (char *)ctx->ws;
    uint32_t *mm = (uint32_t *)base;
    float *F = F_out ? F_out : (float *)(base + o_f);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = launch_residual(X, desc.layout, desc.H, desc.W, C, basis->mean, basis->V, dres, 1, F, mm, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "qfca_quantize_residual/residual");
    e = launch_quantize(F, N, desc.H, desc.W, C, 1, B, QFCA_RANGE_IMAGE, mm, nullptr, nullptr, bins, pitch, lo_out,
                        hi_out, ref_hist_out, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "qfca_quantize_residual/quantize");
    return QFCA_OK;
}

static qfca_status run_assoc(qfca_ctx *ctx, const AssocJob *jobs, int n, int d, int B, cudaStream_t st) {
    for (int i = 0; i < n; i++) {
        const AssocJob &j = jobs[i];
        if (!j.bins || !j.ref || !j.score) return fail(ctx, QFCA_ERR_INVALID_ARG, "image %d: NULL pointer", i);
        if (j.H < 1 || j.W < 1) return fail(ctx, QFCA_ERR_INVALID_ARG, "image %d: bad H x W", i);
        if (j.pitch < j.W) return fail(ctx, QFCA_ERR_INVALID_ARG, "image %d: pitch %d < W", i, j.pitch);
        if (j.r < 1) return fail(ctx, QFCA_ERR_INVALID_ARG, "image %d: r = %d < 1", i, j.r);
        if (j.Nref < 1) return fail(ctx, QFCA_ERR_INVALID_ARG, "image %d: ref_total must be >= 1", i);
        if (!assoc_shape_ok(B, j.r))
            return fail(ctx, QFCA_ERR_UNSUPPORTED, "B = %d with r = %d does not fit the association kernel", B, j.r);
        if ((j.lo == nullptr) != (j.hi == nullptr))
            return fail(ctx, QFCA_ERR_INVALID_ARG, "image %d: value units need both lo and hi", i);
    }
    if (d < 1 || d > kMaxPlanes) return fail(ctx, QFCA_ERR_INVALID_ARG, "d = %d outside [1, %d]", d, kMaxPlanes);
    if (B < 2 || B > kMaxB) return fail(ctx, QFCA_ERR_INVALID_ARG, "B = %d outside [2, %d]", B, kMaxB);
    if (!(jobs[0].sigma_s >= 0.0f && jobs[0].sigma_s <= 4.0f))
        return fail(ctx, QFCA_ERR_INVALID_ARG, "sigma_s = %g outside [0, 4]", (double)jobs[0].sigma_s);
    DeviceGuard g(ctx->device);
    HookScope hs(ctx);
    qfca_status s;
    if ((s = ensure_ws(ctx, assoc_jobs_workspace_bytes(jobs, n, d), st))) return s;
    const cudaError_t e = launch_assoc_jobs(jobs, n, d, B, ctx->ws, st);
    if (e == cudaErrorNotSupported) return fail(ctx, QFCA_ERR_UNSUPPORTED, "shape does not fit the association kernel");
    if (e != cudaSuccess) return cuda_fail(ctx, e, "qfca_score_assoc");
    return QFCA_OK;
}

qfca_status qfca_score_assoc(qfca_ctx *ctx, const uint8_t *bins, int H, int W, int pitch, int d, int B, int r,
                             const uint32_t *ref_hist, uint32_t ref_total, float sigma_s, float *score,
                             float *raw_out, float *comp_out, const float *lo, const float *hi, void *stream) {
    qfca_status s = check_ctx(ctx);
    if (s) return s;
    std::lock_guard<std::mutex> lk(ctx->mu);
    const AssocJob job{bins, H, W, pitch, r, ref_hist, ref_total, sigma_s, score, raw_out, comp_out, lo, hi};
    return run_assoc(ctx, &job, 1, d, B, (cudaStream_t)stream);
}

qfca_status qfca_score_assoc_batch(qfca_ctx *ctx, const qfca_assoc_image *imgs, int n, int d, int B,
                                   float sigma_s, void *stream) {
    qfca_status s = check_ctx(ctx);
    if (s) return s;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (!imgs || n < 1 || n > 4096) return fail(ctx, QFCA_ERR_INVALID_ARG, "n = %d outside [1, 4096]", n);
    std::vector<AssocJob> jobs(n);
    for (int i = 0; i < n; i++)
        jobs[i] = AssocJob{imgs[i].bins, imgs[i].H, imgs[i].W, imgs[i].pitch, imgs[i].r, imgs[i].ref_hist,
                           imgs[i].ref_total, sigma_s, imgs[i].score, imgs[i].raw, nullptr, imgs[i].lo, imgs[i].hi};
    return run_assoc(ctx, jobs.data(), n, d, B, (cudaStream_t)stream);
}

static qfca_status run_median(qfca_ctx *ctx, const MedianJob *jobs, int n, int d, int B, cudaStream_t st) {
    if (d < 1 || d > kMaxPlanes) return fail(ctx, QFCA_ERR_INVALID_ARG, "d = %d outside [1, %d]", d, kMaxPlanes);
    if (B < 2 || B > kMaxB) return fail(ctx, QFCA_ERR_INVALID_ARG, "B = %d outside [2, %d]", B, kMaxB);
    for (int i = 0; i < n; i++) {
        const MedianJob &j = jobs[i];
        if (!j.bins || !j.ref_out) return fail(ctx, QFCA_ERR_INVALID_ARG, "image %d: NULL pointer", i);
        if (j.r < 1) return fail(ctx, QFCA_ERR_INVALID_ARG, "image %d: r = %d < 1", i, j.r);
        if (j.H <= 2 * j.r || j.W <= 2 * j.r)
            return fail(ctx, QFCA_ERR_INVALID_ARG, "image %d: %d x %d has no full window of radius %d", i, j.H, j.W, j.r);
        if (j.pitch < j.W) return fail(ctx, QFCA_ERR_INVALID_ARG, "image %d: pitch %d < W", i, j.pitch);
        if (!median_shape_ok(B, j.r))
            return fail(ctx, QFCA_ERR_UNSUPPORTED, "B = %d with r = %d: the count table does not fit", B, j.r);
    }
    DeviceGuard g(ctx->device);
    HookScope hs(ctx);
    qfca_status s;
    if ((s = ensure_ws(ctx, median_jobs_workspace_bytes(jobs, n, d, B), st))) return s;
    const cudaError_t e = launch_median_jobs(jobs, n, d, B, ctx->ws, st);
    if (e == cudaErrorNotSupported) return fail(ctx, QFCA_ERR_UNSUPPORTED, "shape does not fit the median kernel");
    if (e != cudaSuccess) return cuda_fail(ctx, e, "qfca_median_reference");
    return QFCA_OK;
}

qfca_status qfca_median_reference(qfca_ctx *ctx, const uint8_t *bins, int H, int W, int pitch, int d, int B,
                                  int r, uint32_t *ref_out, void *stream) {
    qfca_status s = check_ctx(ctx);
    if (s) return s;
    std::lock_guard<std::mutex> lk(ctx->mu);
    const MedianJob job{bins, H, W, pitch, r, ref_out};
    return run_median(ctx, &job, 1, d, B, (cudaStream_t)stream);
}

qfca_status qfca_metrics(qfca_ctx *ctx, const float *scores, const uint8_t *masks, int nimg, int H, int W, int border,
                         double fpr_limit, double *out, void *stream) {
    qfca_status s = check_ctx(ctx);
    if (s) return s;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (!scores || !masks || !out) return fail(ctx, QFCA_ERR_INVALID_ARG, "scores / masks / out NULL");
    if (nimg < 1 || nimg > 4096) return fail(ctx, QFCA_ERR_INVALID_ARG, "nimg = %d outside [1, 4096]", nimg);
    if (H < 1 || W < 1 || border < 0 || 2 * border >= H || 2 * border >= W)
        return fail(ctx, QFCA_ERR_INVALID_ARG, "H x W = %d x %d with border %d leaves no pixel", H, W, border);
    if (!(fpr_limit > 0.0 && fpr_limit <= 1.0))
        return fail(ctx, QFCA_ERR_INVALID_ARG, "fpr_limit = %g outside (0, 1]", fpr_limit);
    const long M = (long)nimg * (H - 2 * border) * (W - 2 * border);
    if (M > metrics_max_pixels())
        return fail(ctx, QFCA_ERR_UNSUPPORTED, "%ld kept pixels above the %ld one call ranks", M, metrics_max_pixels());
    DeviceGuard g(ctx->device);
    HookScope hs(ctx);
    if ((s = ensure_ws(ctx, metrics_workspace_bytes(nimg, H, W, border), (cudaStream_t)stream))) return s;
    const cudaError_t e = launch_metrics(scores, masks, nimg, H, W, border, fpr_limit, out, ctx->ws, ctx->status_dev,
                                         (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "qfca_metrics");
    return QFCA_OK;
}

qfca_status qfca_median_reference_batch(qfca_ctx *ctx, const qfca_median_image *imgs, int n, int d, int B,
                                        void *stream) {
    qfca_status s = check_ctx(ctx);
    if (s) return s;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (!imgs || n < 1 || n > 4096) return fail(ctx, QFCA_ERR_INVALID_ARG, "n = %d outside [1, 4096]", n);
    std::vector<MedianJob> jobs(n);
    for (int i = 0; i < n; i++)
        jobs[i] = MedianJob{imgs[i].bins, imgs[i].H, imgs[i].W, imgs[i].pitch, imgs[i].r, imgs[i].ref_out};
    return run_median(ctx, jobs.data(), n, d, B, (cudaStream_t)stream);
}

qfca_status qfca_batch_run_plus(qfca_ctx *ctx, const float *X, int nimg, qfca_fmap desc, int dres, int B, int r,
                                float *scores, const qfca_batch_outputs *extra, void *stream) {
    qfca_status s = check_ctx(ctx);
    if (s) return s;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if ((s = check_fmap(ctx, X, desc))) return s;
    if (nimg < 1 || nimg > 4096) return fail(ctx, QFCA_ERR_INVALID_ARG, "nimg = %d outside [1, 4096]", nimg);
    if (!scores) return fail(ctx, QFCA_ERR_INVALID_ARG, "scores NULL");
    if (dres < 1 || dres > desc.C || dres > kMaxResidual)
        return fail(ctx, QFCA_ERR_INVALID_ARG, "dres = %d outside [1, min(C, %d)]", dres, kMaxResidual);
    if (desc.C > kMaxPlanes) return fail(ctx, QFCA_ERR_INVALID_ARG, "C = %d above %d", desc.C, kMaxPlanes);
    if (B < 2 || B > kMaxB) return fail(ctx, QFCA_ERR_INVALID_ARG, "B = %d outside [2, %d]", B, kMaxB);
    if (r < 1 || 2 * r + 1 > 127) return fail(ctx, QFCA_ERR_INVALID_ARG, "r = %d outside [1, 63]", r);
    if (extra && extra->bins && (extra->pitch < desc.W || extra->pitch % 16 != 0))
        return fail(ctx, QFCA_ERR_INVALID_ARG, "extra->pitch %d must be >= W and a multiple of 16", extra->pitch);
    if (extra && extra->bins && ((uintptr_t)extra->bins & 15) != 0)
        return fail(ctx, QFCA_ERR_INVALID_ARG, "extra->bins must be 16-byte aligned");
    DeviceGuard g(ctx->device);
    HookScope hs(ctx);
    const long N = (long)desc.H * desc.W;
    const int C = desc.C;
    const int pitch = (extra && extra->bins) ? extra->pitch : (desc.W + 15) / 16 * 16;
    // workspace: [fit | basis | residual features | keys | bins | hist | lo/hi | score]
    size_t o = 0;
    auto take = [&](size_t bytes) { const size_t at = o; o = align_up(o + bytes, 256); return at; };
    const size_t o_fit = take(fit_workspace_bytes(C, N, dres, nimg));
    const size_t o_mean = take(sizeof(double) * (size_t)C * nimg);
    const size_t o_V = take(sizeof(double) * (size_t)C * dres * nimg);
    const size_t o_ev = take(sizeof(double) * (size_t)dres * nimg);
    const size_t o_F = take(sizeof(float) * (size_t)C * N * nimg);
    const size_t o_mm = take(sizeof(uint32_t) * 2 * (size_t)C * kKeyStride * nimg);
    const size_t o_bins = take((size_t)C * desc.H * pitch * nimg);
    const size_t o_hist = take(sizeof(uint32_t) * (size_t)C * B * nimg);
    const size_t o_lohi = take(sizeof(float) * 2 * (size_t)C * nimg);
    std::vector<ScoreJob> jobs((size_t)nimg);
    for (int i = 0; i < nimg; i++) jobs[i] = ScoreJob{nullptr, desc.H, desc.W, pitch, r, nullptr, (uint32_t)N, nullptr, nullptr};
    const size_t o_sc = take(score_jobs_workspace_bytes(jobs.data(), nimg, C));
    if ((s = ensure_ws(ctx, o, (cudaStream_t)stream))) return s;
    char *b = (char *)ctx->ws;
    double *mean = (extra && extra->mean) ? extra->mean : (double *)(b + o_mean);
    double *V = (extra && extra->V) ? extra->V : (double *)(b + o_V);
    double *ev = (extra && extra->eigvals) ? extra->eigvals : (double *)(b + o_ev);
    uint8_t *bins = (extra && extra->bins) ? extra->bins : (uint8_t *)(b + o_bins);
    uint32_t *hist = (extra && extra->ref_hist) ? extra->ref_hist : (uint32_t *)(b + o_hist);
    float *lo = (extra && extra->lo) ? extra->lo : (float *)(b + o_lohi);
    float *hi = (extra && extra->hi) ? extra->hi : (float *)(b + o_lohi) + (size_t)C * nimg;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = launch_fit(X, desc.layout, desc.H, desc.W, C, dres, nimg, mean, V, ev, b + o_fit, ctx->status_dev, st,
                               ctx->eig_tol);
    if (e == cudaErrorNotSupported) return fail(ctx, QFCA_ERR_UNSUPPORTED, "eigensolver shape C=%d d=%d", C, dres);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "qfca_batch_run_plus/fit");
    float *F = (float *)(b + o_F);
    uint32_t *mm = (uint32_t *)(b + o_mm);
    e = launch_residual(X, desc.layout, desc.H, desc.W, C, mean, V, dres, nimg, F, mm, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "qfca_batch_run_plus/residual");
    e = launch_quantize(F, N, desc.H, desc.W, C, nimg, B, QFCA_RANGE_IMAGE, mm, nullptr, nullptr, bins, pitch, lo, hi,
                        hist, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "qfca_batch_run_plus/quantize");
    for (int i = 0; i < nimg; i++) {
        jobs[i].bins = bins + (size_t)i * C * desc.H * pitch;
        jobs[i].ref = hist + (size_t)i * C * B;
        jobs[i].score = scores + (size_t)i * N;
    }
    return run_score(ctx, jobs.data(), nimg, C, B, b + o_sc, st, "qfca_batch_run_plus/score");
}

// qfca_batch_run, and (mean_in, V_in given) qfca_batch_run_basis: the fit is
// skipped and the given bases are used.
static qfca_status batch_run_impl(qfca_ctx *ctx, const float *X, int nimg, qfca_fmap desc, int d, int B, int r,
                                  int precision, float *scores, const qfca_batch_outputs *extra, void *stream,
                                  const double *mean_in, const double *V_in) {
    qfca_status s = check_ctx(ctx);
    if (s) return s;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if ((s = check_fmap(ctx, X, desc))) return s;
    if (nimg < 1 || nimg > 4096) return fail(ctx, QFCA_ERR_INVALID_ARG, "nimg = %d outside [1, 4096]", nimg);
    if (!scores) return fail(ctx, QFCA_ERR_INVALID_ARG, "scores NULL");
    if (d < 1 || d > desc.C || d > kMaxD) return fail(ctx, QFCA_ERR_INVALID_ARG, "d = %d outside [1, min(C, %d)]", d, kMaxD);
    if (B < 2 || B > kMaxB) return fail(ctx, QFCA_ERR_INVALID_ARG, "B = %d outside [2, %d]", B, kMaxB);
    if (r < 1 || 2 * r + 1 > 127) return fail(ctx, QFCA_ERR_INVALID_ARG, "r = %d outside [1, 63]", r);
    if (precision != QFCA_F32 && precision != QFCA_BF16 && precision != QFCA_FP8_E4M3)
        return fail(ctx, QFCA_ERR_INVALID_ARG, "precision %d not available", precision);
    const int pitch_min = (desc.W + 15) / 16 * 16;
    if (extra && extra->bins && (extra->pitch < desc.W || extra->pitch % 16 != 0))
        return fail(ctx, QFCA_ERR_INVALID_ARG, "extra->pitch %d must be >= W and a multiple of 16", extra->pitch);
    if (extra && extra->bins && ((uintptr_t)extra->bins & 15) != 0)
        return fail(ctx, QFCA_ERR_INVALID_ARG, "extra->bins must be 16-byte aligned");
    DeviceGuard g(ctx->device);
    HookScope hs(ctx);
    const long N = (long)desc.H * desc.W;
    const int C = desc.C;
    const int pitch = (extra && extra->bins) ? extra->pitch : pitch_min;
    // workspace: [fit | basis | Y | keys | project | bins | hist | lo/hi | score]
    size_t o = 0;
    auto take = [&](size_t bytes) { const size_t at = o; o = align_up(o + bytes, 256); return at; };
    const bool fit = mean_in == nullptr;
    const size_t o_fit = take(fit ? fit_workspace_bytes(C, N, d, nimg) : 0);
    const size_t o_mean = take(sizeof(double) * (size_t)C * nimg);
    const size_t o_V = take(sizeof(double) * (size_t)C * d * nimg);
    const size_t o_ev = take(sizeof(double) * (size_t)d * nimg);
    const size_t o_Y = take(sizeof(float) * (size_t)d * N * nimg);
    const size_t o_mm = take(sizeof(uint32_t) * 2 * (size_t)d * kKeyStride * nimg);
    const size_t o_pj = take(project_workspace_bytes(C, N, d, nimg));
    const size_t o_bins = take((size_t)d * desc.H * pitch * nimg);
    const size_t o_hist = take(sizeof(uint32_t) * (size_t)d * B * nimg);
    const size_t o_lohi = take(sizeof(float) * 2 * (size_t)d * nimg);
    std::vector<ScoreJob> jobs((size_t)nimg);
    for (int i = 0; i < nimg; i++) jobs[i] = ScoreJob{nullptr, desc.H, desc.W, pitch, r, nullptr, (uint32_t)N, nullptr, nullptr};
    const size_t o_sc = take(score_jobs_workspace_bytes(jobs.data(), nimg, d));
    if ((s = ensure_ws(ctx, o, (cudaStream_t)stream))) return s;
    char *b = (char *)ctx->ws;
    const double *mean = mean_in ? mean_in : (extra && extra->mean) ? extra->mean : (double *)(b + o_mean);
    const double *V = V_in ? V_in : (extra && extra->V) ? extra->V : (double *)(b + o_V);
    uint8_t *bins = (extra && extra->bins) ? extra->bins : (uint8_t *)(b + o_bins);
    uint32_t *hist = (extra && extra->ref_hist) ? extra->ref_hist : (uint32_t *)(b + o_hist);
    float *lo = (extra && extra->lo) ? extra->lo : (float *)(b + o_lohi);
    float *hi = (extra && extra->hi) ? extra->hi : (float *)(b + o_lohi) + (size_t)d * nimg;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (fit) {
        double *ev = (extra && extra->eigvals) ? extra->eigvals : (double *)(b + o_ev);
        e = launch_fit(X, desc.layout, desc.H, desc.W, C, d, nimg, const_cast<double *>(mean),
                       const_cast<double *>(V), ev, b + o_fit, ctx->status_dev, st, ctx->eig_tol);
        if (e == cudaErrorNotSupported) return fail(ctx, QFCA_ERR_UNSUPPORTED, "eigensolver shape C=%d d=%d", C, d);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "qfca_batch_run/fit");
    }
    float *Y = (float *)(b + o_Y);
    uint32_t *mm = (uint32_t *)(b + o_mm);
    e = run_projection(ctx, shape_key("batch", nimg, C, d, {N, (long)precision, (long)desc.layout}), C, d, st,
                       [&] {
                           return launch_project(X, desc.layout, desc.H, desc.W, C, mean, V, d, nimg, precision, Y,
                                                 mm, b + o_pj, ctx->status_dev, st);
                       });
    if (e == cudaErrorNotSupported) return fail(ctx, QFCA_ERR_UNSUPPORTED, "projection precision %d", precision);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "qfca_batch_run/project");
    e = launch_quantize(Y, N, desc.H, desc.W, d, nimg, B, QFCA_RANGE_IMAGE, mm, nullptr, nullptr, bins, pitch, lo, hi,
                        hist, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "qfca_batch_run/quantize");
    for (int i = 0; i < nimg; i++) {
        jobs[i].bins = bins + (size_t)i * d * desc.H * pitch;
        jobs[i].ref = hist + (size_t)i * d * B;
        jobs[i].score = scores + (size_t)i * N;
    }
    return run_score(ctx, jobs.data(), nimg, d, B, b + o_sc, st, "qfca_batch_run/score");
}

qfca_status qfca_batch_run(qfca_ctx *ctx, const float *X, int nimg, qfca_fmap desc, int d, int B, int r,
                           int precision, float *scores, const qfca_batch_outputs *extra, void *stream) {
    return batch_run_impl(ctx, X, nimg, desc, d, B, r, precision, scores, extra, stream, nullptr, nullptr);
}

qfca_status qfca_batch_run_host(qfca_ctx *ctx, const float *X_host, int nimg, qfca_fmap desc, int d, int B, int r,
                                int precision, float *scores_host, void *stream) {
    qfca_status s = check_ctx(ctx);
    if (s) return s;
    cudaStream_t st = (cudaStream_t)stream;
    size_t o_s = 0, sb = 0;
    char *io = nullptr;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        if (!X_host || !scores_host) return fail(ctx, QFCA_ERR_INVALID_ARG, "X_host / scores_host NULL");
        if (nimg < 1 || nimg > 4096) return fail(ctx, QFCA_ERR_INVALID_ARG, "nimg = %d outside [1, 4096]", nimg);
        if (desc.H < 1 || desc.W < 1 || desc.C < 1 || (long)desc.H * desc.W > (1L << 23) || desc.C > kMaxC)
            return fail(ctx, QFCA_ERR_INVALID_ARG, "bad shape %d x %d x %d", desc.C, desc.H, desc.W);
        const size_t xb = sizeof(float) * (size_t)nimg * desc.C * desc.H * desc.W;
        sb = sizeof(float) * (size_t)nimg * desc.H * desc.W;
        o_s = align_up(xb, 256);
        DeviceGuard g(ctx->device);
        if (o_s + sb > ctx->io_bytes) {  // grows like the workspace: never during stream capture
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            if (st && cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
                return fail(ctx, QFCA_ERR_INVALID_ARG,
                            "the staging buffer must grow to %zu bytes during stream capture: run the call once "
                            "before capturing", o_s + sb);
            if (ctx->io) {
                cudaError_t e = cudaFree(ctx->io);
                ctx->io = nullptr;
                ctx->io_bytes = 0;
                if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaFree(staging)");
            }
            void *p = nullptr;
            const size_t sz = align_up(o_s + sb, 1 << 20);
            cudaError_t e = cudaMalloc(&p, sz);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return fail(ctx, QFCA_ERR_OOM, "staging of %zu bytes: %s", sz, cudaGetErrorString(e));
            }
            ctx->io = p;
            ctx->io_bytes = sz;
        }
        io = (char *)ctx->io;
        cudaError_t e = cudaMemcpyAsync(io, X_host, xb, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "qfca_batch_run_host/H2D");
    }
    s = batch_run_impl(ctx, (const float *)io, nimg, desc, d, B, r, precision, (float *)(io + o_s), nullptr, stream,
                       nullptr, nullptr);
    if (s) return s;
    cudaError_t e = cudaMemcpyAsync(scores_host, io + o_s, sb, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) {
        std::lock_guard<std::mutex> lk(ctx->mu);
        return cuda_fail(ctx, e, "qfca_batch_run_host/D2H");
    }
    return QFCA_OK;
}

qfca_status qfca_batch_run_basis(qfca_ctx *ctx, const float *X, int nimg, qfca_fmap desc, const double *mean,
                                 const double *V, int d, int B, int r, int precision, float *scores,
                                 const qfca_batch_outputs *extra, void *stream) {
    if (!mean || !V) return fail(ctx, QFCA_ERR_INVALID_ARG, "mean / V NULL");
    return batch_run_impl(ctx, X, nimg, desc, d, B, r, precision, scores, extra, stream, mean, V);
}

qfca_status qfca_score_batch(qfca_ctx *ctx, const qfca_image *imgs, int n, int C, int layout, int d, int B,
                             int precision, void *stream) {
    qfca_status s = check_ctx(ctx);
    if (s) return s;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (!imgs) return fail(ctx, QFCA_ERR_INVALID_ARG, "imgs is NULL");
    if (n < 1 || n > 4096) return fail(ctx, QFCA_ERR_INVALID_ARG, "n = %d outside [1, 4096]", n);
    if (layout != QFCA_NCHW && layout != QFCA_NHWC) return fail(ctx, QFCA_ERR_INVALID_ARG, "bad layout %d", layout);
    if (C < 2 || C > kMaxC) return fail(ctx, QFCA_ERR_UNSUPPORTED, "C = %d outside [2, %d]", C, kMaxC);
    if (d < 1 || d > C || d > kMaxD) return fail(ctx, QFCA_ERR_INVALID_ARG, "d = %d outside [1, min(C, %d)]", d, kMaxD);
    if (B < 2 || B > kMaxB) return fail(ctx, QFCA_ERR_INVALID_ARG, "B = %d outside [2, %d]", B, kMaxB);
    if (precision != QFCA_F32 && precision != QFCA_BF16 && precision != QFCA_FP8_E4M3)
        return fail(ctx, QFCA_ERR_INVALID_ARG, "precision %d not available", precision);
    for (int i = 0; i < n; i++) {
        const qfca_image &im = imgs[i];
        if (!im.X || !im.score) return fail(ctx, QFCA_ERR_INVALID_ARG, "image %d: NULL pointer", i);
        if (im.H < 1 || im.W < 1 || (long)im.H * im.W < 2)
            return fail(ctx, QFCA_ERR_INVALID_ARG, "image %d: bad H x W = %d x %d", i, im.H, im.W);
        if ((long)im.H * im.W > (1L << 23)) return fail(ctx, QFCA_ERR_UNSUPPORTED, "image %d: H*W > 2^23", i);
        if (im.r < 1 || 2 * im.r + 1 > 127) return fail(ctx, QFCA_ERR_INVALID_ARG, "image %d: r = %d outside [1, 63]", i, im.r);
        if (!score_shape_ok(B, im.r))
            return fail(ctx, QFCA_ERR_UNSUPPORTED, "image %d: B = %d with r = %d does not fit shared memory", i, B, im.r);
    }
    DeviceGuard g(ctx->device);
    HookScope hs(ctx);
    cudaStream_t st = (cudaStream_t)stream;
    // workspace: [fit | mean | V | ev | prep | keys | per image: Y, bins, hist, lo/hi | score]
    size_t o = 0;
    auto take = [&](size_t bytes) { const size_t at = o; o = align_up(o + bytes, 256); return at; };
    const size_t o_fit = take(fit_workspace_bytes(C, 1, d, n));
    const size_t o_mean = take(sizeof(double) * (size_t)C * n);
    const size_t o_V = take(sizeof(double) * (size_t)C * d * n);
    const size_t o_ev = take(sizeof(double) * (size_t)d * n);
    long maxN = 0;
    for (int i = 0; i < n; i++) maxN = std::max(maxN, (long)imgs[i].H * imgs[i].W);
    const size_t o_pj = take(std::max(project_bf16_workspace_bytes(C, maxN, d, n), project_workspace_bytes(C, maxN, d, 1)));
    const size_t o_mm = take(bytes_mmkeys(d) * (size_t)n);
    std::vector<size_t> o_Y(n), o_bins(n), o_hist(n), o_lohi(n);
    std::vector<int> pitch(n);
    for (int i = 0; i < n; i++) {
        const long N = (long)imgs[i].H * imgs[i].W;
        pitch[i] = (imgs[i].W + 15) / 16 * 16;
        o_Y[i] = take(sizeof(float) * (size_t)d * N);
        o_bins[i] = take((size_t)d * imgs[i].H * pitch[i]);
        o_hist[i] = take(sizeof(uint32_t) * (size_t)d * B);
        o_lohi[i] = take(sizeof(float) * 2 * (size_t)d);
    }
    std::vector<ScoreJob> sjobs(n);
    for (int i = 0; i < n; i++)
        sjobs[i] = ScoreJob{nullptr, imgs[i].H, imgs[i].W, pitch[i], imgs[i].r, nullptr,
                            (uint32_t)((long)imgs[i].H * imgs[i].W), imgs[i].score, nullptr};
    const size_t o_sc = take(score_jobs_workspace_bytes(sjobs.data(), n, d));
    if ((s = ensure_ws(ctx, o, (cudaStream_t)stream))) return s;
    char *b = (char *)ctx->ws;
    double *mean = (double *)(b + o_mean), *V = (double *)(b + o_V), *ev = (double *)(b + o_ev);
    uint32_t *mm = (uint32_t *)(b + o_mm);
    const size_t mm_stride = bytes_mmkeys(d) / sizeof(uint32_t);

    // fit: one launch per stage for the table
    std::vector<FitJob> fjobs(n);
    for (int i = 0; i < n; i++) fjobs[i] = FitJob{imgs[i].X, (long)imgs[i].H * imgs[i].W};
    cudaError_t e = launch_fit_jobs(fjobs.data(), n, layout, C, d, mean, V, ev, b + o_fit, ctx->status_dev, st,
                                    ctx->eig_tol);
    if (e == cudaErrorNotSupported) return fail(ctx, QFCA_ERR_UNSUPPORTED, "eigensolver shape C=%d d=%d", C, d);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "qfca_score_batch/fit");
    // projection: the TMA-fed table kernel when every image allows it, else one call per image
    bool tma = precision == QFCA_BF16;
    for (int i = 0; i < n && tma; i++) tma = project_tma_ok(imgs[i].X, (long)imgs[i].H * imgs[i].W, layout);
    if (mm_stride != (size_t)2 * d * kKeyStride) return fail(ctx, QFCA_ERR_UNSUPPORTED, "key layout");
    if (tma) {
        std::vector<long> sizes;
        for (int i = 0; i < n; i++) sizes.push_back((long)imgs[i].H * imgs[i].W);
        e = run_projection(ctx, shape_key("table", n, C, d, sizes), C, d, st, [&] {
            float *mean32 = nullptr;
            void *Vt = nullptr;
            int Cp = 0, DT = 0;
            cudaError_t r = launch_prep_bf16(mean, V, C, d, n, b + o_pj, &mean32, &Vt, &Cp, &DT, st);
            if (r == cudaSuccess) r = launch_init_keys(mm, d, n, st);
            std::vector<ProjJob> pjobs(n);
            for (int i = 0; i < n; i++)
                pjobs[i] = ProjJob{imgs[i].X, (long)imgs[i].H * imgs[i].W, mean32 + (size_t)i * Cp,
                                   (const char *)Vt + sizeof(uint16_t) * (size_t)i * DT * Cp, (float *)(b + o_Y[i]),
                                   mm + (size_t)i * mm_stride};
            if (r == cudaSuccess) r = launch_project_tma(pjobs.data(), n, C, d, false, ctx->status_dev, st);
            return r;
        });
    } else {
        for (int i = 0; i < n && e == cudaSuccess; i++)
            e = launch_project(imgs[i].X, layout, imgs[i].H, imgs[i].W, C, mean + (size_t)i * C, V + (size_t)i * C * d, d,
                               1, precision, (float *)(b + o_Y[i]), mm + (size_t)i * mm_stride, b + o_pj,
                               ctx->status_dev, st);
    }
    if (e == cudaErrorNotSupported) return fail(ctx, QFCA_ERR_UNSUPPORTED, "projection shape C=%d d=%d", C, d);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "qfca_score_batch/project");
    // quantisation: image-wide ranges, each image's own reference histogram
    std::vector<QuantJob> qjobs(n);
    for (int i = 0; i < n; i++) {
        float *lo = (float *)(b + o_lohi[i]);
        qjobs[i] = QuantJob{(const float *)(b + o_Y[i]), imgs[i].H, imgs[i].W, mm + (size_t)i * mm_stride, nullptr,
                            nullptr, (uint8_t *)(b + o_bins[i]), pitch[i], lo, lo + d, (uint32_t *)(b + o_hist[i])};
    }
    e = launch_quantize_jobs(qjobs.data(), n, d, B, true, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "qfca_score_batch/quantize");
    for (int i = 0; i < n; i++) {
        sjobs[i].bins = (const uint8_t *)(b + o_bins[i]);
        sjobs[i].ref = (const uint32_t *)(b + o_hist[i]);
    }
    return run_score(ctx, sjobs.data(), n, d, B, b + o_sc, st, "qfca_score_batch/score");
}

qfca_status qfca_set_autotune(qfca_ctx *ctx, int mode) {
    if (!ctx || (mode != 0 && mode != 1)) return QFCA_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->autotune = mode;
    return QFCA_OK;
}

qfca_status qfca_set_tiling(qfca_ctx *ctx, int strip_width, int band_height, int component_groups) {
    if (!ctx) return QFCA_ERR_INVALID_ARG;
    if (strip_width == 0) {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->forced = ScoreTiling{0, 0, 0};
        return QFCA_OK;
    }
    if (!(strip_width == 64 || strip_width == 128) || band_height < 1 || band_height > 64 || component_groups < 1)
        return fail(ctx, QFCA_ERR_INVALID_ARG, "tiling %d x %d x %d", strip_width, band_height, component_groups);
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->forced = ScoreTiling{strip_width, band_height, component_groups};
    return QFCA_OK;
}

qfca_status qfca_set_cdf_walk(qfca_ctx *ctx, int walk) {
    if (!ctx) return QFCA_ERR_INVALID_ARG;
    if (walk < -1 || walk > 1) return fail(ctx, QFCA_ERR_INVALID_ARG, "CDF walk %d outside [-1, 1]", walk);
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->walk_mode = walk;
    return QFCA_OK;
}

qfca_status qfca_set_band_run(qfca_ctx *ctx, int bands) {
    if (!ctx) return QFCA_ERR_INVALID_ARG;
    if (bands < 0 || bands > 4096) return fail(ctx, QFCA_ERR_INVALID_ARG, "band run %d outside [0, 4096]", bands);
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->band_run = bands;
    return QFCA_OK;
}

qfca_status qfca_last_band_run(qfca_ctx *ctx, int *bands) {
    if (!ctx || !bands) return QFCA_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    *bands = ctx->last_tiling.bands;
    return QFCA_OK;
}

qfca_status qfca_last_cdf_walk(qfca_ctx *ctx, int *walk) {
    if (!ctx || !walk) return QFCA_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    *walk = ctx->last_tiling.walk;
    return QFCA_OK;
}

qfca_status qfca_last_tiling(qfca_ctx *ctx, int *strip_width, int *band_height, int *component_groups) {
    if (!ctx || !strip_width || !band_height || !component_groups) return QFCA_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    *strip_width = ctx->last_tiling.SW;
    *band_height = ctx->last_tiling.TH;
    *component_groups = ctx->last_tiling.n_kg;
    return QFCA_OK;
}

qfca_status qfca_last_projection_tiling(qfca_ctx *ctx, int *stages, int *operand_buffers) {
    if (!ctx || !stages || !operand_buffers) return QFCA_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    *stages = ctx->last_proj.stages;
    *operand_buffers = ctx->last_proj.na;
    return QFCA_OK;
}

qfca_status qfca_device_status(qfca_ctx *ctx, int *out) {
    if (!ctx || !out) return QFCA_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(out, ctx->status_dev, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(ctx->status_dev, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "qfca_device_status");
    return *out ? QFCA_ERR_TIMEOUT : QFCA_OK;
}

qfca_status qfca_set_eig_tolerance(qfca_ctx *ctx, double tol) {
    if (!ctx || !(tol >= 0.0)) return QFCA_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->eig_tol = (float)tol;
    return QFCA_OK;
}

qfca_status qfca_eig_redo_count(qfca_ctx *ctx, uint64_t *out) {
    if (!ctx || !out) return QFCA_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    int v = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&v, ctx->status_dev + kRedoCountSlot, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(ctx->status_dev + kRedoCountSlot, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "qfca_eig_redo_count");
    *out = (uint64_t)v;
    return QFCA_OK;
}

qfca_status qfca_launch_count(qfca_ctx *ctx, uint64_t *out) {
    if (!ctx || !out) return QFCA_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    *out = ctx->tracer.launches;
    return QFCA_OK;
}

qfca_status qfca_trace_start(qfca_ctx *ctx, const char *filter) {
    if (!ctx) return QFCA_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    ctx->tracer.reset();
    ctx->tracer.filter = filter ? filter : "";
    ctx->tracer.active = true;
    return QFCA_OK;
}

qfca_status qfca_trace_stop(qfca_ctx *ctx) {
    if (!ctx) return QFCA_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->tracer.active = false;
    return QFCA_OK;
}

qfca_status qfca_trace_get(qfca_ctx *ctx, int i, char *name_out, double *total_ms, uint64_t *launches) {
    if (!ctx) return QFCA_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx->mu);
    DeviceGuard g(ctx->device);
    cudaError_t e = ctx->tracer.aggregate();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "qfca_trace_get");
    if (i < 0 || (size_t)i >= ctx->tracer.agg_name.size()) return QFCA_ERR_INVALID_ARG;
    if (name_out) {
        strncpy(name_out, ctx->tracer.agg_name[i].c_str(), 63);
        name_out[63] = 0;
    }
    if (total_ms) *total_ms = ctx->tracer.agg_ms[i];
    if (launches) *launches = ctx->tracer.agg_n[i];
    return QFCA_OK;
}

}  // extern "C"
