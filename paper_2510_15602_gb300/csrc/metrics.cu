// metrics.cu -- the evaluation of arXiv 2510.15602, Sec. 4.2, on the GPU:
// pixel AUROC, F1 at the optimal threshold, the per-region overlap (PRO) curve
// integrated to a false-positive-rate limit (AUPRO), and the image-level AUROC
// of the maximum pixel score, each after discarding a border of the maps.
//
// Thresholds are every distinct score value (a pixel is predicted anomalous
// when its score is >= the threshold), so the curves are exact:
//   1. every kept pixel becomes one 64-bit word (the order-inverted key of its
//      score, then its index) and the words are sorted ascending by a bitonic
//      network: scores descending, ties grouped (their order inside a run of
//      equal scores does not change any metric);
//   2. anomalous regions are the 8-connected components of the cropped masks,
//      found by a lock-free union-find (one pass of unions over each pixel's
//      left, upper-left, upper and upper-right neighbours, then flattening);
//      an anomalous pixel weighs 1 / (number of regions x its region's size);
//   3. inclusive prefix sums over the sorted order give, at the end of every
//      run of equal scores, the true positives TP and the predicted count (F1 =
//      2 TP / (predicted + positives)), the false-positive rate and the PRO
//      value; the Mann-Whitney statistic (ties one half) is summed exactly in
//      integers per run, AUPRO by trapezoids up to the limit with linear
//      interpolation at it;
//   4. the image-level AUROC compares the maxima of the cropped maps of the
//      images with and without anomalous pixels, pair by pair.
// Integer results are exact; FP64 sums use a fixed reduction order, so the
// results are deterministic.  Every retry loop is bounded and reports through
// the status word.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>

#include "internal.cuh"

namespace qfca {
namespace {

constexpr int kTile = 2048;       // elements of a shared-memory bitonic tile (and of a scan block)
constexpr int kTileThreads = 1024;

struct MetCounters {
    unsigned long long u2;   // 2 U of the Mann-Whitney statistic (exact)
    unsigned long long f1b;  // bits of the largest F1 (non-negative doubles order like their bits)
    unsigned int n_pos, n_reg;
};

__host__ __device__ inline long next_pow2(long v) {
    long p = kTile;
    while (p < v) p <<= 1;
    return p;
}

// ---------------------------------------------------------------- 1. keys, masks, components

// keys[p] = (inverted score key) << 32 | p for the M kept pixels (and all-ones past M);
// parent[p] = p for anomalous pixels, -1 otherwise; counts the anomalous pixels.
__global__ void k_met_init(const float *__restrict__ scores, const uint8_t *__restrict__ masks, int H, int W,
                           int border, long M, long P, unsigned long long *__restrict__ keys, int *__restrict__ parent,
                           MetCounters *cnt) {
    const int h = H - 2 * border, w = W - 2 * border;
    const long hw = (long)h * w;
    unsigned pos = 0;
    for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < P; p += (long)gridDim.x * blockDim.x) {
        if (p >= M) {
            keys[p] = ~0ull;
            continue;
        }
        const long img = p / hw, rem = p - img * hw;
        const int y = (int)(rem / w) + border, x = (int)(rem % w) + border;
        const long src = (img * H + y) * (long)W + x;
        // -0 and +0 are one score: adding +0 maps -0 to +0 (round to nearest) and leaves every
        // other value as it is, so equal scores share one key
        const uint32_t key = ~f2key(__fadd_rn(scores[src], 0.0f));  // ascending key order = descending score
        keys[p] = (unsigned long long)key << 32 | (unsigned long long)p;
        const bool m = masks[src] != 0;
        parent[p] = m ? (int)p : -1;
        pos += m;
    }
    for (int o = 16; o > 0; o >>= 1) pos += __shfl_down_sync(0xffffffffu, pos, o);
    if ((threadIdx.x & 31) == 0 && pos) atomicAdd(&cnt->n_pos, pos);
}

__device__ int uf_find(volatile int *parent, int x, int *status) {
    for (int it = 0; it < (1 << 24); it++) {
        const int q = parent[x];
        if (q == x) return x;
        x = q;
    }
    atomicOr(status, kStatusMetricsLimit);
    return x;
}

// Link the two roots, the larger under the smaller; a link succeeds only while its target is still a root.
__device__ void uf_unite(int *parent, int a, int b, int *status) {
    for (int it = 0; it < (1 << 20); it++) {
        a = uf_find(parent, a, status);
        b = uf_find(parent, b, status);
        if (a == b) return;
        if (a > b) {
            const int t = a;
            a = b;
            b = t;
        }
        if (atomicCAS(&parent[b], b, a) == b) return;
    }
    atomicOr(status, kStatusMetricsLimit);
}

__global__ void k_met_union(int *parent, int h, int w, long M, int *status) {
    const long hw = (long)h * w;
    for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < M; p += (long)gridDim.x * blockDim.x) {
        if (parent[p] < 0) continue;
        const long img0 = p - p % hw;
        const int y = (int)((p - img0) / w), x = (int)((p - img0) % w);
        const int dx[4] = {-1, -1, 0, 1}, dy[4] = {0, -1, -1, -1};
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const int yy = y + dy[k], xx = x + dx[k];
            if (yy < 0 || xx < 0 || xx >= w) continue;
            const long q = img0 + (long)yy * w + xx;
            if (((volatile int *)parent)[q] >= 0) uf_unite(parent, (int)p, (int)q, status);
        }
    }
}

// parent[p] = its root (an ancestor, so concurrent finds stay valid); region sizes at the roots; region count.
__global__ void k_met_flatten(int *parent, long M, unsigned *__restrict__ rsize, MetCounters *cnt, int *status) {
    unsigned roots = 0;
    for (long p = blockIdx.x * (long)blockDim.x + threadIdx.x; p < M; p += (long)gridDim.x * blockDim.x) {
        if (((volatile int *)parent)[p] < 0) continue;
        const int r = uf_find(parent, (int)p, status);
        parent[p] = r;
        atomicAdd(&rsize[r], 1u);
        roots += r == (int)p;
    }
    for (int o = 16; o > 0; o >>= 1) roots += __shfl_down_sync(0xffffffffu, roots, o);
    if ((threadIdx.x & 31) == 0 && roots) atomicAdd(&cnt->n_reg, roots);
}

// ---------------------------------------------------------------- 2. bitonic sort (ascending)

__device__ __forceinline__ void cmp_swap(unsigned long long &a, unsigned long long &b, bool asc) {
    if ((a > b) == asc) {
        const unsigned long long t = a;
        a = b;
        b = t;
    }
}

// Every stage j <= jmax of merge size k (k = 0: all merge sizes up to kTile) inside one tile of kTile
// words in shared memory; the direction of element i is ascending when (i & k) == 0 (global index i).
__global__ void __launch_bounds__(kTileThreads) k_bitonic_tile(unsigned long long *keys, long k_fixed) {
    __shared__ unsigned long long s[kTile];
    const long base = (long)blockIdx.x * kTile;
    for (int i = threadIdx.x; i < kTile; i += kTileThreads) s[i] = keys[base + i];
    __syncthreads();
    const long k0 = k_fixed ? k_fixed : 2, k1 = k_fixed ? k_fixed : kTile;
    for (long k = k0; k <= k1; k <<= 1) {
        for (int j = (int)(k_fixed ? kTile / 2 : k / 2); j > 0; j >>= 1) {
            const int t = threadIdx.x;
            const int i0 = (t / j) * 2 * j + t % j, i1 = i0 + j;
            const bool asc = ((base + i0) & k) == 0;
            unsigned long long a = s[i0], b = s[i1];
            cmp_swap(a, b, asc);
            s[i0] = a;
            s[i1] = b;
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < kTile; i += kTileThreads) keys[base + i] = s[i];
}

// One stage (merge size k, stride j >= kTile) over the whole array: one thread per pair.
__global__ void k_bitonic_global(unsigned long long *keys, long P, long k, long j) {
    const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (t >= P / 2) return;
    const long i0 = (t / j) * 2 * j + t % j, i1 = i0 + j;
    unsigned long long a = keys[i0], b = keys[i1];
    const bool asc = (i0 & k) == 0;
    if ((a > b) == asc) {
        keys[i0] = b;
        keys[i1] = a;
    }
}

// ---------------------------------------------------------------- 3. sorted-order arrays and scans

// For sorted position i: the anomalous indicator and the PRO weight of its pixel.
__global__ void k_met_gather(const unsigned long long *__restrict__ keys, const int *__restrict__ parent,
                             const unsigned *__restrict__ rsize, const MetCounters *cnt, long M, int *__restrict__ sp,
                             double *__restrict__ sw) {
    const double nreg = (double)cnt->n_reg;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < M; i += (long)gridDim.x * blockDim.x) {
        const long p = (long)(keys[i] & 0xffffffffull);
        const int r = parent[p];
        sp[i] = r >= 0;
        sw[i] = r >= 0 ? 1.0 / (nreg * (double)rsize[r]) : 0.0;
    }
}

struct SumOp {
    template <class T>
    __device__ T operator()(T a, T b) const { return a + b; }
};
struct MaxOp {
    template <class T>
    __device__ T operator()(T a, T b) const { return a > b ? a : b; }
};

// Inclusive scan of one block's kTile elements in place (Hillis-Steele in shared memory, a fixed
// order); the block's total to tot[block].
template <class T, class Op>
__global__ void __launch_bounds__(kTileThreads) k_scan_block(T *v, long M, T *tot, T ident) {
    __shared__ T s[2][kTile];
    const long base = (long)blockIdx.x * kTile;
    for (int i = threadIdx.x; i < kTile; i += kTileThreads) s[0][i] = base + i < M ? v[base + i] : ident;
    __syncthreads();
    int cur = 0;
    for (int o = 1; o < kTile; o <<= 1) {
        for (int i = threadIdx.x; i < kTile; i += kTileThreads)
            s[cur ^ 1][i] = i >= o ? Op()(s[cur][i - o], s[cur][i]) : s[cur][i];
        __syncthreads();
        cur ^= 1;
    }
    for (int i = threadIdx.x; i < kTile; i += kTileThreads)
        if (base + i < M) v[base + i] = s[cur][i];
    if (threadIdx.x == 0) tot[blockIdx.x] = s[cur][kTile - 1];
}

// Adds the scanned totals of the blocks before each block (the totals themselves scanned by one block).
template <class T, class Op>
__global__ void k_scan_add(T *v, long M, const T *tot_scanned) {
    const long b = blockIdx.x;
    if (b == 0) return;
    const T add = tot_scanned[b - 1];
    for (long i = b * kTile + threadIdx.x; i < min(M, (b + 1) * kTile); i += blockDim.x) v[i] = Op()(add, v[i]);
}

// run starts: rs[i] = i if position i begins a run of equal scores, else 0 (a max-scan then gives each
// position its run's start)
__global__ void k_met_starts(const unsigned long long *__restrict__ keys, long M, int *__restrict__ rs) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < M; i += (long)gridDim.x * blockDim.x)
        rs[i] = (i == 0 || (keys[i] >> 32) != (keys[i - 1] >> 32)) ? (int)i : 0;
}

// ---------------------------------------------------------------- 4. per-run terms

// At every run end i (run start s): F1, the Mann-Whitney terms and the AUPRO trapezoid between the previous
// run end (s - 1, or the curve's (0, 0) start) and i.  Per-block area sums in a fixed order.
__global__ void __launch_bounds__(256) k_met_runs(const unsigned long long *__restrict__ keys, long M,
                                                  const int *__restrict__ tp, const double *__restrict__ wp,
                                                  const int *__restrict__ rstart, MetCounters *cnt, double limit,
                                                  double *__restrict__ area_part) {
    __shared__ double red[256];
    const long npos = cnt->n_pos, nneg = M - npos;
    double area = 0.0;
    unsigned long long u2 = 0, f1b = 0;
    const long i = blockIdx.x * (long)blockDim.x + threadIdx.x;
    if (i < M && (i == M - 1 || (keys[i + 1] >> 32) != (keys[i] >> 32))) {
        const long s = rstart[i];
        const long tpi = tp[i], tps = s > 0 ? tp[s - 1] : 0;
        const long fni = (i + 1) - tpi, fns = s - tps;  // negatives up to i / before the run
        // F1 at threshold = this run's score
        if (npos > 0) {
            const double f1 = 2.0 * (double)tpi / ((double)(i + 1) + (double)npos);
            f1b = (unsigned long long)__double_as_longlong(f1);
        }
        // Mann-Whitney: each anomalous pixel of the run beats the negatives below it, ties one half (times 2)
        const unsigned long long pg = (unsigned long long)(tpi - tps), ng = (unsigned long long)(fni - fns);
        u2 = 2ull * pg * (unsigned long long)(nneg - fni) + pg * ng;
        // PRO curve point and its predecessor
        if (nneg > 0) {
            const double fi = fmin((double)fni / (double)nneg, 1.0), fp = fmin((double)fns / (double)nneg, 1.0);
            const double pi = wp[i], pp = s > 0 ? wp[s - 1] : 0.0;
            if (fi <= limit) {
                area = 0.5 * (pi + pp) * (fi - fp);
            } else if (fp < limit) {
                const double pl = pp + (pi - pp) * (limit - fp) / (fi - fp);
                area = 0.5 * (pl + pp) * (limit - fp);
            }
        }
    }
    if (u2) atomicAdd(&cnt->u2, u2);
    if (f1b) atomicMax(&cnt->f1b, f1b);
    red[threadIdx.x] = area;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) area_part[blockIdx.x] = red[0];
}

// ---------------------------------------------------------------- 5. image level and the results

// One block per image: the maximum of the cropped map, and whether the full mask has an anomalous pixel.
__global__ void __launch_bounds__(256) k_met_image(const float *__restrict__ scores, const uint8_t *__restrict__ masks,
                                                   int H, int W, int border, float *__restrict__ imax,
                                                   int *__restrict__ ilab) {
    __shared__ float smax[256];
    __shared__ int sany[256];
    const long img = blockIdx.x;
    const float *s = scores + img * (long)H * W;
    const uint8_t *m = masks + img * (long)H * W;
    float mx = -INFINITY;
    int any = 0;
    for (long q = threadIdx.x; q < (long)H * W; q += blockDim.x) {
        const int y = (int)(q / W), x = (int)(q % W);
        if (y >= border && y < H - border && x >= border && x < W - border) mx = fmaxf(mx, s[q]);
        any |= m[q] != 0;
    }
    smax[threadIdx.x] = mx;
    sany[threadIdx.x] = any;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            smax[threadIdx.x] = fmaxf(smax[threadIdx.x], smax[threadIdx.x + o]);
            sany[threadIdx.x] |= sany[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        imax[img] = smax[0];
        ilab[img] = sany[0];
    }
}

// One block: the image-level AUROC by pair counting (ties one half), the area's fixed-order sum, and the
// four results: pixel AUROC, F1 max, AUPRO, image AUROC (NaN where a class is empty).
__global__ void __launch_bounds__(256) k_met_final(const float *__restrict__ imax, const int *__restrict__ ilab, int n,
                                                   const double *__restrict__ area_part, long nparts, long M,
                                                   const MetCounters *cnt, double limit, double *__restrict__ out) {
    __shared__ unsigned long long su[256];
    __shared__ double sa[256];
    unsigned long long u = 0;
    for (long e = threadIdx.x; e < (long)n * n; e += blockDim.x) {
        const int a = (int)(e / n), b = (int)(e % n);
        if (ilab[a] && !ilab[b]) u += imax[a] > imax[b] ? 2ull : (imax[a] == imax[b] ? 1ull : 0ull);
    }
    double area = 0.0;
    for (long e = threadIdx.x; e < nparts; e += blockDim.x) area += area_part[e];  // fixed per-thread order
    su[threadIdx.x] = u;
    sa[threadIdx.x] = area;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            su[threadIdx.x] += su[threadIdx.x + o];
            sa[threadIdx.x] += sa[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double nan = __longlong_as_double(0x7ff8000000000000ll);
        const long npos = cnt->n_pos, nneg = M - npos;
        out[0] = (npos > 0 && nneg > 0) ? (double)cnt->u2 / (2.0 * (double)npos * (double)nneg) : nan;
        out[1] = npos > 0 ? __longlong_as_double((long long)cnt->f1b) : nan;
        out[2] = (nneg > 0 && cnt->n_reg > 0 && M > 0) ? sa[0] / limit : nan;
        long ip = 0;
        for (int a = 0; a < n; a++) ip += ilab[a] != 0;
        out[3] = (ip > 0 && ip < n) ? (double)su[0] / (2.0 * (double)ip * (double)(n - ip)) : nan;
    }
}

struct MetPlan {
    long M, P, nblk;
    size_t keys, parent, rsize, sp, sw, rs, tot_i, tot_d, area, imax, ilab, cnt, total;
};

MetPlan met_plan(int nimg, int H, int W, int border) {
    MetPlan m{};
    m.M = (long)nimg * (H - 2 * border) * (W - 2 * border);
    m.P = next_pow2(m.M);
    m.nblk = (m.M + kTile - 1) / kTile;
    size_t o = 0;
    auto take = [&](size_t b) { const size_t at = o; o = align_up(o + b, 256); return at; };
    m.keys = take(sizeof(unsigned long long) * (size_t)m.P);
    m.parent = take(sizeof(int) * (size_t)m.M);
    m.rsize = take(sizeof(unsigned) * (size_t)m.M);
    m.sp = take(sizeof(int) * (size_t)m.M);
    m.sw = take(sizeof(double) * (size_t)m.M);
    m.rs = take(sizeof(int) * (size_t)m.M);
    m.tot_i = take(sizeof(int) * (size_t)(kTile + 1));
    m.tot_d = take(sizeof(double) * (size_t)(kTile + 1));
    m.area = take(sizeof(double) * (size_t)((m.M + 255) / 256 + 1));
    m.imax = take(sizeof(float) * (size_t)nimg);
    m.ilab = take(sizeof(int) * (size_t)nimg);
    m.cnt = take(sizeof(MetCounters));
    m.total = o;
    return m;
}

template <class T, class Op>
cudaError_t scan(T *v, long M, long nblk, T *tot, T ident, cudaStream_t st) {
    QFCA_LAUNCH("k_scan_block", st, (k_scan_block<T, Op><<<(unsigned)nblk, kTileThreads, 0, st>>>(v, M, tot, ident)));
    if (nblk > 1) {
        // the block totals (at most kTile of them) scanned by one block, in place; its own total goes past them
        QFCA_LAUNCH("k_scan_block", st, (k_scan_block<T, Op><<<1, kTileThreads, 0, st>>>(tot, nblk, tot + kTile, ident)));
        QFCA_LAUNCH("k_scan_add", st, (k_scan_add<T, Op><<<(unsigned)nblk, 256, 0, st>>>(v, M, tot)));
    }
    return cudaGetLastError();
}

}  // namespace

long metrics_max_pixels() { return (long)kTile * kTile; }

size_t metrics_workspace_bytes(int nimg, int H, int W, int border) { return met_plan(nimg, H, W, border).total; }

cudaError_t launch_metrics(const float *scores, const uint8_t *masks, int nimg, int H, int W, int border,
                           double fpr_limit, double *out, void *ws, int *status, cudaStream_t st) {
    const MetPlan m = met_plan(nimg, H, W, border);
    if (m.M > metrics_max_pixels()) return cudaErrorNotSupported;
    char *b = (char *)ws;
    unsigned long long *keys = (unsigned long long *)(b + m.keys);
    int *parent = (int *)(b + m.parent), *sp = (int *)(b + m.sp), *rs = (int *)(b + m.rs);
    unsigned *rsize = (unsigned *)(b + m.rsize);
    double *sw = (double *)(b + m.sw), *area = (double *)(b + m.area);
    MetCounters *cnt = (MetCounters *)(b + m.cnt);
    float *imax = (float *)(b + m.imax);
    int *ilab = (int *)(b + m.ilab);
    const int h = H - 2 * border, w = W - 2 * border;
    cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(MetCounters), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(rsize, 0, sizeof(unsigned) * (size_t)m.M, st);
    if (e != cudaSuccess) return e;
    const unsigned g = (unsigned)std::min<long>((m.P + 255) / 256, 4096);
    QFCA_LAUNCH("k_met_init", st, (k_met_init<<<g, 256, 0, st>>>(scores, masks, H, W, border, m.M, m.P, keys, parent, cnt)));
    const unsigned gm = (unsigned)std::max<long>(1, std::min<long>((m.M + 255) / 256, 4096));
    QFCA_LAUNCH("k_met_union", st, (k_met_union<<<gm, 256, 0, st>>>(parent, h, w, m.M, status)));
    QFCA_LAUNCH("k_met_flatten", st, (k_met_flatten<<<gm, 256, 0, st>>>(parent, m.M, rsize, cnt, status)));
    // bitonic sort of the P words
    const unsigned tiles = (unsigned)(m.P / kTile);
    QFCA_LAUNCH("k_bitonic_tile", st, (k_bitonic_tile<<<tiles, kTileThreads, 0, st>>>(keys, 0)));
    for (long k = 2L * kTile; k <= m.P; k <<= 1) {
        for (long j = k / 2; j >= kTile; j >>= 1)
            QFCA_LAUNCH("k_bitonic_global", st,
                        (k_bitonic_global<<<(unsigned)((m.P / 2 + 255) / 256), 256, 0, st>>>(keys, m.P, k, j)));
        QFCA_LAUNCH("k_bitonic_tile", st, (k_bitonic_tile<<<tiles, kTileThreads, 0, st>>>(keys, k)));
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (m.M > 0) {
        QFCA_LAUNCH("k_met_gather", st, (k_met_gather<<<gm, 256, 0, st>>>(keys, parent, rsize, cnt, m.M, sp, sw)));
        QFCA_LAUNCH("k_met_starts", st, (k_met_starts<<<gm, 256, 0, st>>>(keys, m.M, rs)));
        if ((e = scan<int, SumOp>(sp, m.M, m.nblk, (int *)(b + m.tot_i), 0, st)) != cudaSuccess) return e;
        if ((e = scan<double, SumOp>(sw, m.M, m.nblk, (double *)(b + m.tot_d), 0.0, st)) != cudaSuccess) return e;
        if ((e = scan<int, MaxOp>(rs, m.M, m.nblk, (int *)(b + m.tot_i), 0, st)) != cudaSuccess) return e;
        QFCA_LAUNCH("k_met_runs", st,
                    (k_met_runs<<<(unsigned)((m.M + 255) / 256), 256, 0, st>>>(keys, m.M, sp, sw, rs, cnt, fpr_limit, area)));
    }
    QFCA_LAUNCH("k_met_image", st, (k_met_image<<<(unsigned)nimg, 256, 0, st>>>(scores, masks, H, W, border, imax, ilab)));
    QFCA_LAUNCH("k_met_final", st,
                (k_met_final<<<1, 256, 0, st>>>(imax, ilab, nimg, area, m.M > 0 ? (m.M + 255) / 256 : 0, m.M, cnt,
                                                 fpr_limit, out)));
    return cudaGetLastError();
}

}  // namespace qfca
