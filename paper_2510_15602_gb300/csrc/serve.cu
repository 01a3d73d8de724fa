// serve.cu -- the serving session of include/qfca.h: resident per-class PCA
// bases, fixed quantisation ranges and reference histograms (the per-texture
// references of arXiv 2510.15602, Sec. 4), a request queue, and a scheduler
// thread doing continuous batching.
//
// Scheduler (one host thread per session):
//   - requests wait in FIFO order; a batch takes requests from the head while
//     they fit max_batch and one contiguous block of the device arena (first
//     fit over a free list), so admission follows free device memory;
//   - a batch runs on a free stream of the session (up to `streams` batches
//     in flight): optional host-to-device copies, one table-driven launch per
//     stage (projection with each request's class basis, quantisation with the
//     class's fixed range, window EMD against the class reference, component
//     mean), optional device-to-host copies, then a stream host callback;
//   - the callback (a CUDA runtime thread, no CUDA calls) stamps the requests
//     done and wakes pollers and the scheduler; the scheduler then returns the
//     batch's arena block and stream and drops its class references.
// A request's arithmetic does not depend on its batch: each image keeps its
// own tiles, its own class operands and exact integer window stages.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "arena.cuh"
#include "internal.cuh"

namespace qfca {

namespace {

struct ClassRec {
    double *mean = nullptr, *V = nullptr;  // FP64 basis (FP32 path, unaligned inputs)
    float *mean32 = nullptr;               // prepared BF16 operands: mean32 [Cp], Vt [DT][Cp]
    void *Vt = nullptr;
    void *prep = nullptr;                  // one allocation holding mean32 and Vt
    float *lo = nullptr, *hi = nullptr;    // fixed range [d] (one allocation)
    uint32_t *ref = nullptr;               // [d][B]
    uint32_t ref_total = 0;
    ~ClassRec() {
        cudaFree(mean);
        cudaFree(V);
        cudaFree(prep);
        cudaFree(lo);
        cudaFree(ref);
    }
};

struct Pending {
    uint64_t ticket;
    qfca_request req;
    std::shared_ptr<ClassRec> cls;
    double t_submit;
};

struct Batch;

}  // namespace

struct ServeState {
    qfca_serve_config cfg{};
    int device = 0;
    int *status_dev = nullptr;
    int Cp = 0, DT = 0;
    char *arena_base = nullptr;
    Arena arena;
    std::vector<cudaStream_t> streams;
    std::vector<char> stream_busy;
    std::map<int, std::shared_ptr<ClassRec>> classes;
    std::deque<Pending> queue;
    std::unordered_map<uint64_t, qfca_result> results;  // submitted, not yet polled
    std::unordered_map<uint64_t, char> done;
    std::vector<std::unique_ptr<Batch>> inflight;
    uint64_t next_ticket = 1;
    uint64_t next_batch = 1;
    std::mutex m;
    std::condition_variable cv_sched, cv_done;
    bool stop = false;
    std::thread th;
    std::chrono::steady_clock::time_point t0;

    double now_us() const {
        return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

struct Batch {
    ServeState *S = nullptr;
    int stream = 0;
    size_t off = 0, bytes = 0;
    std::vector<Pending> reqs;
    double t_start = 0.0;
    bool finished = false;
};

int pitch_of(int W) { return (W + 15) / 16 * 16; }

// Device bytes one request occupies inside a batch block.
size_t request_bytes(const ServeState &S, const qfca_request &r) {
    const qfca_serve_config &c = S.cfg;
    const long N = (long)r.H * r.W;
    size_t b = 0;
    if (r.flags & QFCA_REQ_HOST_INPUT) b += align_up(sizeof(float) * (size_t)c.C * N, 256);
    b += align_up(sizeof(float) * (size_t)c.d * N, 256);                  // Y
    b += align_up((size_t)c.d * r.H * pitch_of(r.W), 256);                // bins
    if (r.flags & QFCA_REQ_HOST_OUTPUT) b += align_up(sizeof(float) * (size_t)N, 256);
    b += align_up(sizeof(uint32_t) * 2 * c.d * kKeyStride, 256);          // min/max keys
    return b;
}

// Per-batch bytes beyond the requests: the projection's operand scratch.
size_t batch_extra_bytes(const ServeState &S, long maxN) {
    return align_up(project_workspace_bytes(S.cfg.C, maxN, S.cfg.d, 1), 256) + 512;
}

void CUDART_CB batch_done(void *arg) {
    Batch *b = static_cast<Batch *>(arg);
    ServeState *S = b->S;
    {
        std::lock_guard<std::mutex> lk(S->m);
        const double t = S->now_us();
        for (const Pending &p : b->reqs) {
            auto it = S->results.find(p.ticket);
            if (it != S->results.end()) {
                it->second.t_done_us = t;
                it->second.status = QFCA_OK;
                S->done[p.ticket] = 1;
            }
        }
        b->finished = true;
    }
    S->cv_done.notify_all();
    S->cv_sched.notify_one();
}

// Enqueue one batch on its stream (scheduler thread, lock not held).
cudaError_t launch_batch(ServeState *S, Batch *b) {
    const qfca_serve_config &c = S->cfg;
    cudaStream_t st = S->streams[b->stream];
    const int n = (int)b->reqs.size();
    char *base = S->arena_base + b->off;
    long maxN = 0;
    for (const Pending &p : b->reqs) maxN = std::max(maxN, (long)p.req.H * p.req.W);
    size_t o = 0;
    auto take = [&](size_t bytes) { char *at = base + o; o += align_up(bytes, 256); return at; };
    char *prep = take(project_workspace_bytes(c.C, maxN, c.d, 1));
    uint32_t *keys = (uint32_t *)take(sizeof(uint32_t) * 2 * c.d * kKeyStride * (size_t)n);
    std::vector<const float *> X(n);
    std::vector<float *> Y(n), sc(n);
    std::vector<uint8_t *> bins(n);
    std::vector<ScoreJob> sj(n);
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < n && e == cudaSuccess; i++) {
        const qfca_request &r = b->reqs[i].req;
        const long N = (long)r.H * r.W;
        X[i] = r.X;
        if (r.flags & QFCA_REQ_HOST_INPUT) {
            float *xd = (float *)take(sizeof(float) * (size_t)c.C * N);
            e = cudaMemcpyAsync(xd, r.X, sizeof(float) * (size_t)c.C * N, cudaMemcpyHostToDevice, st);
            X[i] = xd;
        }
        Y[i] = (float *)take(sizeof(float) * (size_t)c.d * N);
        bins[i] = (uint8_t *)take((size_t)c.d * r.H * pitch_of(r.W));
        sc[i] = (r.flags & QFCA_REQ_HOST_OUTPUT) ? (float *)take(sizeof(float) * (size_t)N) : r.score;
        const ClassRec &cl = *b->reqs[i].cls;
        sj[i] = ScoreJob{bins[i], r.H, r.W, pitch_of(r.W), r.r, cl.ref, cl.ref_total, sc[i], nullptr};
    }
    if (e != cudaSuccess) return e;
    // projection: the TMA-fed table kernel when every image allows it
    bool tma = c.precision == QFCA_BF16;
    for (int i = 0; i < n && tma; i++) tma = project_tma_ok(X[i], (long)b->reqs[i].req.H * b->reqs[i].req.W, QFCA_NCHW);
    if (tma) {
        e = launch_init_keys(keys, c.d, n, st);
        // the class's fixed range is known, so the projection's epilogue writes the bins itself
        std::vector<ProjJob> pj(n);
        for (int i = 0; i < n; i++) {
            const ClassRec &cl = *b->reqs[i].cls;
            const qfca_request &r = b->reqs[i].req;
            pj[i] = ProjJob{X[i], (long)r.H * r.W, cl.mean32, cl.Vt, Y[i], keys + (size_t)i * 2 * c.d * kKeyStride};
            pj[i].qlo = cl.lo, pj[i].qhi = cl.hi, pj[i].bins = bins[i];
            pj[i].W = r.W, pj[i].pitch = pitch_of(r.W), pj[i].B = c.B;
        }
        if (e == cudaSuccess) e = launch_project_tma(pj.data(), n, c.C, c.d, false, S->status_dev, st);
    } else {
        for (int i = 0; i < n && e == cudaSuccess; i++) {
            const qfca_request &r = b->reqs[i].req;
            const ClassRec &cl = *b->reqs[i].cls;
            e = launch_project(X[i], QFCA_NCHW, r.H, r.W, c.C, cl.mean, cl.V, c.d, 1, c.precision, Y[i],
                               keys + (size_t)i * 2 * c.d * kKeyStride, prep, S->status_dev, st);
        }
    }
    if (e != cudaSuccess) return e;
    if (!tma) {
        // quantisation with the class's fixed range; the class histogram is the reference
        std::vector<QuantJob> qj(n);
        for (int i = 0; i < n; i++) {
            const qfca_request &r = b->reqs[i].req;
            const ClassRec &cl = *b->reqs[i].cls;
            qj[i] = QuantJob{Y[i], r.H, r.W, nullptr, cl.lo, cl.hi, bins[i], pitch_of(r.W), nullptr, nullptr, nullptr};
        }
        e = launch_quantize_jobs(qj.data(), n, c.d, c.B, false, st);
        if (e != cudaSuccess) return e;
    }
    char *score_ws = base + o;
    e = launch_score_jobs(sj.data(), n, c.d, c.B, score_ws, false, S->status_dev, st, nullptr, nullptr);
    if (e != cudaSuccess) return e;
    for (int i = 0; i < n && e == cudaSuccess; i++) {
        const qfca_request &r = b->reqs[i].req;
        if (r.flags & QFCA_REQ_HOST_OUTPUT)
            e = cudaMemcpyAsync(r.score, sc[i], sizeof(float) * (size_t)r.H * r.W, cudaMemcpyDeviceToHost, st);
    }
    if (e != cudaSuccess) return e;
    return cudaLaunchHostFunc(st, batch_done, b);
}

size_t batch_bytes(const ServeState &S, const std::vector<Pending> &reqs) {
    long maxN = 0;
    size_t b = 0;
    std::vector<ScoreJob> sj;
    for (const Pending &p : reqs) {
        maxN = std::max(maxN, (long)p.req.H * p.req.W);
        b += request_bytes(S, p.req);
        sj.push_back(ScoreJob{nullptr, p.req.H, p.req.W, pitch_of(p.req.W), p.req.r, nullptr, 1, nullptr, nullptr});
    }
    return b + batch_extra_bytes(S, maxN) + score_jobs_workspace_bytes(sj.data(), (int)sj.size(), S.cfg.d);
}

void scheduler(ServeState *S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->m);
    for (;;) {
        // reap finished batches
        for (size_t i = 0; i < S->inflight.size();) {
            Batch *b = S->inflight[i].get();
            if (b->finished) {
                S->arena.release(b->off, b->bytes);
                S->stream_busy[b->stream] = 0;
                S->inflight.erase(S->inflight.begin() + (long)i);
            } else {
                i++;
            }
        }
        // launch batches while a stream is free and the head of the queue fits
        for (;;) {
            int sidx = -1;
            for (size_t k = 0; k < S->streams.size(); k++)
                if (!S->stream_busy[k]) { sidx = (int)k; break; }
            if (sidx < 0 || S->queue.empty()) break;
            std::vector<Pending> take;
            size_t bytes = 0;
            const size_t room = S->arena.largest();
            for (const Pending &p : S->queue) {
                if ((int)take.size() >= S->cfg.max_batch) break;
                take.push_back(p);
                const size_t need = batch_bytes(*S, take);
                if (need > room) {
                    take.pop_back();
                    break;
                }
                bytes = need;
            }
            if (take.empty()) break;  // the head waits for memory
            size_t off = 0;
            if (!S->arena.alloc(bytes, &off)) break;
            for (size_t k = 0; k < take.size(); k++) S->queue.pop_front();
            auto b = std::make_unique<Batch>();
            b->S = S, b->stream = sidx, b->off = off, b->bytes = bytes, b->reqs = std::move(take);
            b->t_start = S->now_us();
            const uint64_t seq = S->next_batch++;
            for (const Pending &p : b->reqs) {
                auto it = S->results.find(p.ticket);
                if (it != S->results.end()) {
                    it->second.t_start_us = b->t_start;
                    it->second.batch_size = (int)b->reqs.size();
                    it->second.stream = sidx;
                    it->second.batch_seq = seq;
                }
            }
            S->stream_busy[sidx] = 1;
            Batch *raw = b.get();
            S->inflight.push_back(std::move(b));
            lk.unlock();
            const cudaError_t e = launch_batch(S, raw);
            lk.lock();
            if (e != cudaSuccess) {
                cudaGetLastError();
                for (const Pending &p : raw->reqs) {
                    auto it = S->results.find(p.ticket);
                    if (it != S->results.end()) {
                        it->second.status = QFCA_ERR_CUDA;
                        it->second.t_done_us = S->now_us();
                        S->done[p.ticket] = 1;
                    }
                }
                // the stream may still hold copies or kernels of this batch: keep its block until they end
                lk.unlock();
                cudaStreamSynchronize(S->streams[sidx]);
                cudaGetLastError();
                lk.lock();
                raw->finished = true;
                S->cv_done.notify_all();
            }
        }
        if (S->stop && S->queue.empty() && S->inflight.empty()) break;
        S->cv_sched.wait_for(lk, std::chrono::milliseconds(50));
    }
}

}  // namespace

}  // namespace qfca

using namespace qfca;

extern "C" qfca_status qfca_serve_start(qfca_ctx *ctx, const qfca_serve_config *cfg) {
    if (!ctx || !cfg) return QFCA_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx_mutex(ctx));
    if (ctx_sticky(ctx)) return ctx_set_error(ctx, QFCA_ERR_CUDA, "context has a sticky CUDA error");
    if (ctx_serve(ctx)) return ctx_set_error(ctx, QFCA_ERR_INVALID_ARG, "a serving session is already running");
    const qfca_serve_config c = *cfg;
    if (c.C < 2 || c.C > kMaxC || c.d < 1 || c.d > c.C || c.d > kMaxD || c.B < 2 || c.B > kMaxB)
        return ctx_set_error(ctx, QFCA_ERR_INVALID_ARG, "serve: bad C, d or B");
    if (c.precision != QFCA_F32 && c.precision != QFCA_BF16)
        return ctx_set_error(ctx, QFCA_ERR_UNSUPPORTED, "serve: precision must be QFCA_F32 or QFCA_BF16");
    if (c.max_batch < 1 || c.max_batch > kMaxBatch || c.streams < 1 || c.streams > 8 || c.max_queue < 1 ||
        c.arena_bytes < (1u << 20))
        return ctx_set_error(ctx, QFCA_ERR_INVALID_ARG, "serve: bad max_batch, streams, max_queue or arena_bytes");
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(ctx_device(ctx));
    auto S = std::make_unique<ServeState>();
    S->cfg = c;
    S->device = ctx_device(ctx);
    S->status_dev = ctx_status_dev(ctx);
    S->t0 = std::chrono::steady_clock::now();
    cudaError_t e = cudaMalloc(&S->arena_base, c.arena_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (prev >= 0) cudaSetDevice(prev);
        return ctx_set_error(ctx, QFCA_ERR_OOM, "serve: arena of " + std::to_string(c.arena_bytes) + " bytes");
    }
    S->arena.reset(c.arena_bytes);
    for (int i = 0; i < c.streams && e == cudaSuccess; i++) {
        cudaStream_t s = nullptr;
        e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
        if (e == cudaSuccess) S->streams.push_back(s), S->stream_busy.push_back(0);
    }
    if (e != cudaSuccess) {
        for (cudaStream_t s : S->streams) cudaStreamDestroy(s);
        cudaFree(S->arena_base);
        if (prev >= 0) cudaSetDevice(prev);
        return ctx_set_error(ctx, QFCA_ERR_CUDA, std::string("serve: ") + cudaGetErrorString(e));
    }
    S->Cp = (c.C + 63) / 64 * 64;
    S->DT = c.d <= 16 ? 16 : (c.d <= 32 ? 32 : 64);
    ServeState *raw = S.release();
    raw->th = std::thread(scheduler, raw);
    ctx_serve(ctx) = raw;
    if (prev >= 0) cudaSetDevice(prev);
    return QFCA_OK;
}

extern "C" qfca_status qfca_register_class(qfca_ctx *ctx, int class_id, const double *mean, const double *V,
                                           const float *lo, const float *hi, const uint32_t *ref_hist,
                                           uint32_t ref_total) {
    if (!ctx) return QFCA_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(ctx_mutex(ctx));
    ServeState *S = ctx_serve(ctx);
    if (!S) return ctx_set_error(ctx, QFCA_ERR_INVALID_ARG, "register_class: no serving session");
    if (!mean || !V || !lo || !hi || !ref_hist || ref_total < 1)
        return ctx_set_error(ctx, QFCA_ERR_INVALID_ARG, "register_class: NULL pointer or empty reference");
    const qfca_serve_config &c = S->cfg;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(S->device);
    auto cl = std::make_shared<ClassRec>();
    cl->ref_total = ref_total;
    cudaError_t e = cudaMalloc(&cl->mean, sizeof(double) * c.C);
    if (e == cudaSuccess) e = cudaMalloc(&cl->V, sizeof(double) * (size_t)c.C * c.d);
    if (e == cudaSuccess) e = cudaMalloc(&cl->lo, sizeof(float) * 2 * c.d);
    if (e == cudaSuccess) e = cudaMalloc(&cl->ref, sizeof(uint32_t) * (size_t)c.d * c.B);
    if (e == cudaSuccess) e = cudaMalloc(&cl->prep, project_bf16_workspace_bytes(c.C, 1, c.d, 1));
    cudaStream_t st = nullptr;
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) {
        cl->hi = cl->lo + c.d;
        e = cudaMemcpyAsync(cl->mean, mean, sizeof(double) * c.C, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(cl->V, V, sizeof(double) * (size_t)c.C * c.d, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(cl->lo, lo, sizeof(float) * c.d, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(cl->hi, hi, sizeof(float) * c.d, cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(cl->ref, ref_hist, sizeof(uint32_t) * (size_t)c.d * c.B, cudaMemcpyDeviceToDevice, st);
        int Cp = 0, DT = 0;
        if (e == cudaSuccess) e = launch_prep_bf16(cl->mean, cl->V, c.C, c.d, 1, cl->prep, &cl->mean32, &cl->Vt, &Cp, &DT, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (st) cudaStreamDestroy(st);
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return ctx_set_error(ctx, QFCA_ERR_CUDA, std::string("register_class: ") + cudaGetErrorString(e));
    }
    std::lock_guard<std::mutex> sl(S->m);
    S->classes[class_id] = cl;
    return QFCA_OK;
}

extern "C" qfca_status qfca_submit(qfca_ctx *ctx, const qfca_request *req, uint64_t *ticket) {
    if (!ctx || !req || !ticket) return QFCA_ERR_INVALID_ARG;
    ServeState *S;
    {
        std::lock_guard<std::mutex> lk(ctx_mutex(ctx));
        S = ctx_serve(ctx);
    }
    if (!S) return QFCA_ERR_INVALID_ARG;
    const qfca_request &r = *req;
    if (!r.X || !r.score || r.H < 1 || r.W < 1 || (long)r.H * r.W < 2 || (long)r.H * r.W > (1L << 23) || r.r < 1 ||
        2 * r.r + 1 > 127 || (r.flags & ~(QFCA_REQ_HOST_INPUT | QFCA_REQ_HOST_OUTPUT)))
        return QFCA_ERR_INVALID_ARG;
    if (!score_shape_ok(S->cfg.B, r.r)) return QFCA_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(S->m);
    if (S->stop) return QFCA_ERR_INVALID_ARG;
    auto it = S->classes.find(r.class_id);
    if (it == S->classes.end()) return QFCA_ERR_INVALID_ARG;
    const Pending probe{0, r, it->second, 0.0};
    if (batch_bytes(*S, std::vector<Pending>{probe}) > S->arena.size) return QFCA_ERR_UNSUPPORTED;
    if ((int)S->queue.size() >= S->cfg.max_queue) return QFCA_ERR_BUSY;
    const uint64_t t = S->next_ticket++;
    Pending p{t, r, it->second, S->now_us()};
    qfca_result res{};
    res.status = QFCA_PENDING;
    res.t_submit_us = p.t_submit;
    S->results[t] = res;
    S->queue.push_back(std::move(p));
    *ticket = t;
    S->cv_sched.notify_one();
    return QFCA_OK;
}

extern "C" qfca_status qfca_poll(qfca_ctx *ctx, uint64_t ticket, int timeout_us, qfca_result *out) {
    if (!ctx || !out) return QFCA_ERR_INVALID_ARG;
    ServeState *S;
    {
        std::lock_guard<std::mutex> lk(ctx_mutex(ctx));
        S = ctx_serve(ctx);
    }
    if (!S) return QFCA_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->m);
    if (!S->results.count(ticket)) return QFCA_ERR_INVALID_ARG;
    auto is_done = [&] { return S->done.count(ticket) != 0; };
    if (!is_done() && timeout_us > 0)
        S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), is_done);
    if (!is_done()) return QFCA_PENDING;
    *out = S->results[ticket];
    S->results.erase(ticket);
    S->done.erase(ticket);
    return QFCA_OK;
}

extern "C" qfca_status qfca_serve_stop(qfca_ctx *ctx) {
    if (!ctx) return QFCA_ERR_INVALID_ARG;
    ServeState *S;
    {
        std::lock_guard<std::mutex> lk(ctx_mutex(ctx));
        S = ctx_serve(ctx);
        ctx_serve(ctx) = nullptr;
    }
    if (!S) return QFCA_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(S->m);
        S->stop = true;
    }
    S->cv_sched.notify_all();
    if (S->th.joinable()) S->th.join();
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(S->device);
    for (cudaStream_t s : S->streams) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
    }
    cudaFree(S->arena_base);
    S->classes.clear();
    if (prev >= 0) cudaSetDevice(prev);
    delete S;
    return QFCA_OK;
}
