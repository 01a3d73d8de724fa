// fit.cu -- single-image PCA fit (arXiv 2510.15602, Sec. 3.3) on the GPU:
// the mean and covariance of the C channels over the H*W pixels (exact
// integer-sliced Gram on the tensor cores, gram.cu) followed by the top-d
// eigenpairs of the covariance (eig32.cu: FP32 reduction and eigenvectors with
// one float-float Newton correction; eig.cu: the float-float cluster solver for
// the matrices that fail its residual check, and for larger shapes).
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.cuh"

namespace qfca {

namespace {

struct FitLayout {
    size_t off_gram, off_cov, off_covff, off_eig, total;
};

FitLayout fit_layout(int C, long N, int d, int nimg) {
    FitLayout L{};
    size_t o = 0;
    L.off_gram = o;
    o = align_up(o + gram_workspace_bytes(C, N, nimg), 256);
    L.off_cov = o;
    o = align_up(o + sizeof(double) * (size_t)C * C * nimg, 256);
    L.off_covff = o;
    o = align_up(o + 2 * sizeof(float) * (size_t)C * C * nimg, 256);
    L.off_eig = o;
    o = align_up(o + eig_workspace_bytes(C, d, nimg), 256);
    L.total = o;
    return L;
}

}  // namespace

size_t fit_workspace_bytes(int C, long N, int d, int nimg) { return fit_layout(C, N, d, nimg).total; }

cudaError_t launch_fit_jobs(const FitJob *jobs, int n, int layout, int C, int d, double *mean, double *V,
                            double *eigvals, void *ws, int *status, cudaStream_t st, float eig_tol) {
    const FitLayout L = fit_layout(C, 1, d, n);
    char *base = (char *)ws;
    double *cov = (double *)(base + L.off_cov);
    void *cov_ff = base + L.off_covff;
    cudaError_t e = launch_gram_cov_jobs(jobs, n, layout, C, mean, cov, cov_ff, base + L.off_gram, status, st);
    if (e != cudaSuccess) return e;
    return launch_eig(cov_ff, C, d, n, V, eigvals, base + L.off_eig, status, st, eig_tol);
}

cudaError_t launch_fit(const float *X, int layout, int H, int W, int C, int d, int nimg, double *mean, double *V,
                       double *eigvals, void *ws, int *status, cudaStream_t st, float eig_tol) {
    const long N = (long)H * W;
    const FitLayout L = fit_layout(C, N, d, nimg);
    char *base = (char *)ws;
    double *cov = (double *)(base + L.off_cov);
    void *cov_ff = base + L.off_covff;
    cudaError_t e = launch_gram_cov(X, layout, C, N, nimg, mean, cov, cov_ff, base + L.off_gram, status, st);
    if (e != cudaSuccess) return e;
    return launch_eig(cov_ff, C, d, nimg, V, eigvals, base + L.off_eig, status, st, eig_tol);
}

}  // namespace qfca
