// project_tc.cu -- BF16 principal-component projection on the 5th-generation
// tensor cores (tcgen05), FP32 accumulation in tensor memory (arXiv 2510.15602,
// Sec. 3.3: Y = (X - mean) V).
//
// GEMM view: Y[p][j] = sum_c A[p][c] * Bt[j][c] with A = bf16(X - mean)
// (M = 128 pixels per tile, K = channels) and Bt = bf16(V^T) (N = DT >= d
// components, zero padded).  Both operands are K-major in shared memory with
// the 128-byte swizzle; one K-chunk is 64 channels (one 128-B row per pixel).
//
// Per CTA (128 threads, persistent over pixel tiles):
//   - Bt for all K stays resident in shared memory;
//   - all threads stream the tile's FP32 features from HBM (coalesced along
//     pixels for NCHW), subtract the mean, convert to BF16 and write them in
//     the swizzled layout;  fence.proxy.async + barrier;
//   - one thread issues the K/16 tcgen05.mma (128 x DT x 16) and a
//     tcgen05.commit to an mbarrier;  all threads wait on it (bounded);
//   - each warp reads its 32 accumulator lanes (tcgen05.ld 32x32b), writes
//     Y[j][p] coalesced and reduces the per-component min/max.
// A wait that runs out sets bit 0 of the device status word, waits once more
// (bounded) for the CTA's MMAs, frees the tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "internal.cuh"
#include "tc.cuh"

namespace qfca {
namespace {

constexpr int kM = 128;
constexpr int kKc = 64;
constexpr int kThreads = 128;
constexpr uint32_t kWaitTries = 1u << 26;

struct TcShape {
    int Cp, DT, nk;
    size_t a_bytes, b_bytes, smem;
};

TcShape tc_shape(int C, int d) {
    TcShape s;
    s.DT = d <= 16 ? 16 : (d <= 32 ? 32 : 64);
    s.Cp = (C + kKc - 1) / kKc * kKc;
    s.nk = s.Cp / kKc;
    s.a_bytes = (size_t)s.nk * kM * 128;
    s.b_bytes = (size_t)s.nk * s.DT * 128;
    s.smem = 1024 + s.a_bytes + s.b_bytes + 64 + 8 * 64;
    return s;
}

// Per image (grid.y): mean32[c] (c < Cp, zero padded) and Vt[j][c] = bf16(V[c][j]) (DT x Cp, zero padded).
__global__ void k_prep_bf16(const double *__restrict__ mean, const double *__restrict__ V, int C, int d, int Cp,
                            int DT, float *__restrict__ mean32, __nv_bfloat16 *__restrict__ Vt) {
    const long img = blockIdx.y;
    mean += img * C;
    V += img * C * d;
    mean32 += img * Cp;
    Vt += img * DT * Cp;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < DT * Cp; e += gridDim.x * blockDim.x) {
        const int j = e / Cp, c = e % Cp;
        const float v = (j < d && c < C) ? (float)V[(long)c * d + j] : 0.0f;
        Vt[e] = __float2bfloat16_rn(v);
        if (j == 0) mean32[c] = c < C ? (float)mean[c] : 0.0f;
    }
}

// FP8 (e4m3) operands of one basis per CTA (grid.x = image):
//   s_c = 2^floor(log2(448 / (max_p |x_cp| + |mean_c|)))   (|(x - mean) s_c| <= 448, no saturation)
//   B'_jc = V_cj / s_c * t_j,  t_j = 2^floor(log2(448 / max_c |V_cj / s_c|))
//   hi = e4m3(B'), lo = e4m3(B' - hi)   (round to nearest even)
// so (x - mean) V = sum_c [(x - mean) s_c] (hi + lo)_jc / t_j up to the e4m3
// roundings.  amax holds max |x| per channel as float bits.
__global__ void __launch_bounds__(256) k_prep_fp8(const double *__restrict__ mean, const double *__restrict__ V,
                                                  const unsigned *__restrict__ amax, int C, int d, int Cp, int DT,
                                                  float *__restrict__ mean32, float *__restrict__ scale,
                                                  float *__restrict__ colscale, uint8_t *__restrict__ Vt8) {
    const long img = blockIdx.x;
    mean += img * C;
    V += img * C * d;
    amax += img * C;
    mean32 += img * Cp;
    scale += img * Cp;
    colscale += img * DT;
    Vt8 += img * 2 * DT * Cp;
    __shared__ float s_sc[512];
    __shared__ float s_t[64];
    for (int c = threadIdx.x; c < Cp; c += blockDim.x) {
        float sc = 1.0f;
        if (c < C) {
            const double bound = (double)__uint_as_float(amax[c]) + fabs(mean[c]);
            if (bound > 0.0) sc = (float)exp2(floor(log2(448.0 / bound)));
        }
        s_sc[c] = sc;
        scale[c] = sc;
        mean32[c] = c < C ? (float)mean[c] : 0.0f;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < DT; j += blockDim.x) {
        double m = 0.0;
        if (j < d)
            for (int c = 0; c < C; c++) m = fmax(m, fabs(V[(long)c * d + j]) / (double)s_sc[c]);
        const float t = m > 0.0 ? (float)exp2(floor(log2(448.0 / m))) : 1.0f;
        s_t[j] = t;
        colscale[j] = 1.0f / t;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < DT * Cp; e += blockDim.x) {
        const int j = e / Cp, c = e % Cp;
        const float b = (j < d && c < C) ? (float)(V[(long)c * d + j] / (double)s_sc[c] * (double)s_t[j]) : 0.0f;
        const __nv_fp8_e4m3 hi(b);
        const __nv_fp8_e4m3 lo(b - (float)hi);
        Vt8[e] = hi.__x;
        Vt8[(long)DT * Cp + e] = lo.__x;
    }
}

__device__ __forceinline__ uint32_t swz_off(int row, int chunk16) {
    // byte offset of 16-B chunk `chunk16` (0..7) of row `row` in a 128-B-swizzled K-major tile
    return (uint32_t)(row * 128 + ((chunk16 ^ (row & 7)) << 4));
}

template <int DT>
__global__ void __launch_bounds__(kThreads) k_project_bf16(const float *__restrict__ X, int layout, int C, int Cp,
                                                          long N, const float *__restrict__ mean32,
                                                          const __nv_bfloat16 *__restrict__ Vt, int d,
                                                          float *__restrict__ Y, uint32_t *__restrict__ mm_keys,
                                                          int *__restrict__ status, long tiles_per_img, int nimg) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = tc::align_smem<1024>(smem_raw);
    const int nk = Cp / kKc;
    uint8_t *As = smem;
    uint8_t *Bs = smem + (size_t)nk * kM * 128;
    uint64_t *bar = (uint64_t *)(Bs + (size_t)nk * DT * 128);
    uint32_t *tmem_slot = (uint32_t *)(bar + 1);
    uint32_t *kmin = tmem_slot + 1;  // [DT]
    uint32_t *kmax = kmin + DT;      // [DT]
    constexpr uint32_t kCols = DT < 32 ? 32 : DT;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        tc::tmem_alloc(tmem_slot, kCols);
        tc::tmem_relinquish();
    }
    if (tid == 0) {
        tc::mbar_init(bar, 1);
        tc::fence_mbar_init();
    }
    if (tid < DT) { kmin[tid] = 0xffffffffu; kmax[tid] = 0u; }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const uint32_t idesc = tc::idesc_bf16_f32(kM, DT);
    const uint32_t a_base = tc::smem_u32(As), b_base = tc::smem_u32(Bs);
    uint32_t phase = 0;
    bool failed = false;
    int cur = -1;  // image whose Bt is resident and whose min/max kmin/kmax hold
    const long n_tiles = tiles_per_img * nimg;

    for (long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int img = (int)(tile / tiles_per_img);
        if (img != cur) {
            if (cur >= 0) {  // flush the previous image's min/max, then reset
                __syncthreads();
                if (tid < d) {
                    atomicMin(&mm_keys[((long)cur * 2 * d + tid) * kKeyStride], kmin[tid]);
                    atomicMax(&mm_keys[((long)cur * 2 * d + d + tid) * kKeyStride], kmax[tid]);
                }
                __syncthreads();
                if (tid < DT) { kmin[tid] = 0xffffffffu; kmax[tid] = 0u; }
            }
            // resident Bt of this image: DT rows x Cp channels, 16-B chunks of 8 channels
            // (the MMAs that read the previous Bt completed before the last epilogue)
            const __nv_bfloat16 *Vi = Vt + (long)img * DT * Cp;
            for (int e = tid; e < DT * (Cp / 8); e += kThreads) {
                const int j = e / (Cp / 8), c8 = e % (Cp / 8);
                const int kc = c8 >> 3, g = c8 & 7;
                const uint4 v = *reinterpret_cast<const uint4 *>(Vi + (long)j * Cp + c8 * 8);
                *reinterpret_cast<uint4 *>(Bs + (size_t)kc * DT * 128 + swz_off(j, g)) = v;
            }
            cur = img;
        }
        const float *Xi = X + (long)img * C * N;
        const float *mui = mean32 + (long)img * Cp;
        const long p0 = (tile - (long)img * tiles_per_img) * kM;
        const int m = tid;
        const long p = p0 + m;
        const bool pv = p < N;
        // ---- stage A: 128 pixels x Cp channels, centred, BF16, swizzled
        for (int kc = 0; kc < nk; kc++) {
            float v[kKc];
            if (layout == QFCA_NCHW) {
#pragma unroll
                for (int i = 0; i < kKc; i++) {
                    const int c = kc * kKc + i;
                    v[i] = (pv && c < C) ? __ldg(Xi + (long)c * N + p) : 0.0f;
                }
            } else {
#pragma unroll
                for (int i = 0; i < kKc; i++) {
                    const int c = kc * kKc + i;
                    v[i] = (pv && c < C) ? __ldg(Xi + p * C + c) : 0.0f;
                }
            }
#pragma unroll
            for (int g = 0; g < 8; g++) {
                uint4 pk;
                const float *mu = mui + kc * kKc + g * 8;
                pk.x = tc::pack_bf16x2(v[g * 8 + 0] - mu[0], v[g * 8 + 1] - mu[1]);
                pk.y = tc::pack_bf16x2(v[g * 8 + 2] - mu[2], v[g * 8 + 3] - mu[3]);
                pk.z = tc::pack_bf16x2(v[g * 8 + 4] - mu[4], v[g * 8 + 5] - mu[5]);
                pk.w = tc::pack_bf16x2(v[g * 8 + 6] - mu[6], v[g * 8 + 7] - mu[7]);
                if (!pv) pk = make_uint4(0, 0, 0, 0);
                *reinterpret_cast<uint4 *>(As + (size_t)kc * kM * 128 + swz_off(m, g)) = pk;
            }
        }
        tc::fence_proxy_async_smem();
        tc::tc_fence_before();
        __syncthreads();
        // ---- MMA: one thread issues K/16 instructions, then commits to the mbarrier
        if (tid == 0) {
            tc::tc_fence_after();
            for (int s = 0; s < nk * 4; s++) {
                const int kc = s >> 2, ks = s & 3;
                const uint64_t ad = tc::sdesc_kmajor_sw128(a_base + kc * kM * 128 + ks * 32);
                const uint64_t bd = tc::sdesc_kmajor_sw128(b_base + kc * DT * 128 + ks * 32);
                tc::mma_bf16_ss(tmem, ad, bd, idesc, s > 0 ? 1u : 0u);
            }
            tc::mma_commit(bar);
        }
        const bool ok = tc::mbar_wait(bar, phase, kWaitTries);
        phase ^= 1u;
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        tc::tc_fence_after();
        // ---- epilogue: lanes 32*warp.. of the accumulator -> registers
        float acc[DT];
#pragma unroll
        for (int j0 = 0; j0 < DT; j0 += 16) {
            uint32_t r[16];
            tc::tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)j0, r);
            tc::tmem_wait_ld();
#pragma unroll
            for (int i = 0; i < 16; i++) acc[j0 + i] = __uint_as_float(r[i]);
        }
        const long pe = p0 + 32 * warp + lane;
        const bool valid = pe < N;
        float *Yi = Y + (long)img * d * N;
#pragma unroll
        for (int j = 0; j < DT; j++) {
            if (j >= d) break;
            if (valid) Yi[(long)j * N + pe] = acc[j];
            float mn = valid ? acc[j] : __int_as_float(0x7f800000);
            float mx = valid ? acc[j] : -__int_as_float(0x7f800000);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
                mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            }
            if (lane == 0) {
                atomicMin(&kmin[j], f2key(mn));
                atomicMax(&kmax[j], f2key(mx));
            }
        }
        tc::tc_fence_before();
    }
    if (failed) {
        if (tid == 0) atomicOr(status, 1);
        tc::mbar_wait(bar, phase ^ 1u, kWaitTries);  // let the CTA's MMAs drain (bounded)
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(tmem, kCols);
    }
    if (!failed && cur >= 0 && tid < d) {
        atomicMin(&mm_keys[((long)cur * 2 * d + tid) * kKeyStride], kmin[tid]);
        atomicMax(&mm_keys[((long)cur * 2 * d + d + tid) * kKeyStride], kmax[tid]);
    }
}

template <int DT>
cudaError_t launch_dt(const float *X, int layout, int C, const TcShape &sh, long N, int nimg, const float *mean32,
                      const __nv_bfloat16 *Vt, int d, float *Y, uint32_t *mm_keys, int *status, cudaStream_t st) {
    static DeviceOnce attrs;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaError_t e = device_once(attrs, dev, [] {
        cudaError_t r = cudaFuncSetAttribute(k_project_bf16<DT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             227 * 1024);
        if (r == cudaSuccess)
            r = cudaFuncSetAttribute(k_project_bf16<DT>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     cudaSharedmemCarveoutMaxShared);
        return r;
    });
    if (e != cudaSuccess) return e;
    int per_sm = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_project_bf16<DT>, kThreads, sh.smem);
    if (e != cudaSuccess) return e;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (per_sm < 1) return cudaErrorNotSupported;
    const int max_blocks = per_sm * sms;
    const long tiles = (N + kM - 1) / kM;
    const long n_tiles = tiles * nimg;
    const int grid = (int)(n_tiles < max_blocks ? n_tiles : max_blocks);
    QFCA_LAUNCH("k_project_bf16", st,
                k_project_bf16<DT><<<grid, kThreads, sh.smem, st>>>(X, layout, C, sh.Cp, N, mean32, Vt, d, Y,
                                                                    mm_keys, status, tiles, nimg));
    return cudaGetLastError();
}

}  // namespace

size_t project_fp8_workspace_bytes(int C, int d, int nimg) {
    const int Cp = (C + 127) / 128 * 128, DT = d <= 16 ? 16 : (d <= 32 ? 32 : 64);
    return (align_up(sizeof(float) * 2 * Cp, 256) + align_up(sizeof(float) * DT, 256) +
            align_up((size_t)2 * DT * Cp, 256) + align_up(sizeof(unsigned) * C, 256)) * nimg + 256;
}

// FP8 projection of nimg same-shaped NCHW images (TMA path only).
cudaError_t launch_project_fp8(const float *X, int layout, long N, int C, const double *mean, const double *V, int d,
                               int nimg, float *Y, uint32_t *mm_keys, void *ws, int *status, cudaStream_t st) {
    if (!project_tma_ok(X, N, layout) || C > 512) return cudaErrorNotSupported;
    const int Cp = (C + 127) / 128 * 128, DT = d <= 16 ? 16 : (d <= 32 ? 32 : 64);
    char *b = (char *)ws;
    float *mean32 = (float *)b;
    b += align_up(sizeof(float) * Cp * nimg, 256);
    float *scale = (float *)b;
    b += align_up(sizeof(float) * Cp * nimg, 256);
    float *colscale = (float *)b;
    b += align_up(sizeof(float) * DT * nimg, 256);
    uint8_t *Vt8 = (uint8_t *)b;
    b += align_up((size_t)2 * DT * Cp * nimg, 256);
    unsigned *amax = (unsigned *)b;
    std::vector<FitJob> fj(nimg);
    for (int i = 0; i < nimg; i++) fj[i] = FitJob{X + (long)i * C * N, N};
    cudaError_t e = launch_chan_absmax_jobs(fj.data(), nimg, layout, C, amax, st);
    if (e != cudaSuccess) return e;
    QFCA_LAUNCH("k_prep_fp8", st,
                k_prep_fp8<<<nimg, 256, 0, st>>>(mean, V, amax, C, d, Cp, DT, mean32, scale, colscale, Vt8));
    std::vector<ProjJob> jobs(nimg);
    for (int i = 0; i < nimg; i++) {
        jobs[i] = ProjJob{X + (long)i * C * N, N, mean32 + (size_t)i * Cp, Vt8 + (size_t)i * 2 * DT * Cp,
                          Y + (size_t)i * d * N, mm_keys + (size_t)i * 2 * d * kKeyStride};
        jobs[i].scale = scale + (size_t)i * Cp;
        jobs[i].colscale = colscale + (size_t)i * DT;
    }
    return launch_project_tma(jobs.data(), nimg, C, d, true, status, st);
}

size_t project_bf16_workspace_bytes(int C, long N, int d, int nimg) {
    (void)N;
    const TcShape s = tc_shape(C, d);
    return align_up(sizeof(float) * s.Cp * nimg, 256) + align_up(sizeof(__nv_bfloat16) * (size_t)s.DT * s.Cp * nimg, 256) +
           256;
}

// Prepared BF16 operands of n bases (packed mean [n][C], V [n][C][d]): mean32
// [n][Cp] and Vt [n][DT][Cp] at the start of ws (project_bf16_workspace_bytes).
cudaError_t launch_prep_bf16(const double *mean, const double *V, int C, int d, int n, void *ws, float **mean32_out,
                             void **Vt_out, int *Cp_out, int *DT_out, cudaStream_t st) {
    const TcShape sh = tc_shape(C, d);
    float *mean32 = (float *)ws;
    __nv_bfloat16 *Vt = (__nv_bfloat16 *)((char *)ws + align_up(sizeof(float) * sh.Cp * n, 256));
    QFCA_LAUNCH("k_prep_bf16", st,
                k_prep_bf16<<<dim3((sh.DT * sh.Cp + 255) / 256, n), 256, 0, st>>>(mean, V, C, d, sh.Cp, sh.DT, mean32,
                                                                                  Vt));
    *mean32_out = mean32;
    *Vt_out = Vt;
    *Cp_out = sh.Cp;
    *DT_out = sh.DT;
    return cudaGetLastError();
}

cudaError_t launch_project_bf16(const float *X, int layout, int H, int W, int C, const double *mean,
                                const double *V, int d, int nimg, float *Y, uint32_t *mm_keys, void *ws,
                                int *status, cudaStream_t st) {
    const long N = (long)H * W;
    const TcShape sh = tc_shape(C, d);
    if (sh.smem > 227 * 1024) return cudaErrorNotSupported;
    float *mean32 = (float *)ws;
    __nv_bfloat16 *Vt = (__nv_bfloat16 *)((char *)ws + align_up(sizeof(float) * sh.Cp * nimg, 256));
    QFCA_LAUNCH("k_prep_bf16", st,
                k_prep_bf16<<<dim3((sh.DT * sh.Cp + 255) / 256, nimg), 256, 0, st>>>(mean, V, C, d, sh.Cp, sh.DT,
                                                                                     mean32, Vt));
    if (project_tma_ok(X, N, layout)) {
        // NCHW with 16-B aligned rows: the TMA-fed pipeline
        ProjJob jobs[kMaxBatch];
        for (int i0 = 0; i0 < nimg; i0 += kMaxBatch) {
            const int m = nimg - i0 < kMaxBatch ? nimg - i0 : kMaxBatch;
            for (int i = 0; i < m; i++) {
                const long img = i0 + i;
                jobs[i] = ProjJob{X + img * C * N, N, mean32 + img * sh.Cp, Vt + img * sh.DT * sh.Cp, Y + img * d * N,
                                  mm_keys + img * 2 * d * kKeyStride};
            }
            cudaError_t e = launch_project_tma(jobs, m, C, d, false, status, st);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    switch (sh.DT) {
        case 16: return launch_dt<16>(X, layout, C, sh, N, nimg, mean32, Vt, d, Y, mm_keys, status, st);
        case 32: return launch_dt<32>(X, layout, C, sh, N, nimg, mean32, Vt, d, Y, mm_keys, status, st);
        default: return launch_dt<64>(X, layout, C, sh, N, nimg, mean32, Vt, d, Y, mm_keys, status, st);
    }
}

}  // namespace qfca
