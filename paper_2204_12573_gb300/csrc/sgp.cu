// Mapping a sparse GP onto the quadratic forms of the hot path (Sec. V-B,
// "Mapped Sparse GP"; Eq. 1 and Eq. 2), on the device in FP64:
//
//   beta  = sig2 * D_S^T diag(alpha) D_S                (Eq. 1 reordered)
//   gamma = sig2 * I - sig2^2 * D_S^T K_SS^{-1} D_S     (Eq. 2 reordered)
//
// with D_S the n_S normalized descriptor rows of the sparse set (full ABI
// layout, d columns), alpha the mean weights and K_SS the sparse-set kernel
// matrix.  K_SS^{-1} is applied through its Cholesky factor L (K_SS = L L^T):
// X = L^{-1} D_S, so D_S^T K_SS^{-1} D_S = X^T X, a symmetric product with no
// explicit inverse.  Kernels: a blocked right-looking Cholesky (panels of
// kNb columns), a blocked forward substitution for X, and one tiled
// weighted symmetric product for both beta and gamma.  This runs once per
// model, not per step; FP64 throughout (GB300's FP64 rate is low, but the
// mapping is a few milliseconds for thousands of sparse points).
#include <vector>

#include "internal.cuh"

namespace flr {
namespace {

constexpr int kNb = 32;   // panel width of the Cholesky and of the substitution
constexpr int kTile = 32; // output tile of the symmetric product

// C = diag * I + coef * sum_s w_s X[s][a] X[s][b]   (a, b < d; X row-major with
// leading dimension ld; w may be nullptr for w = 1).  One 32x32 tile of C per
// block, 256 threads, four outputs per thread.
__global__ void k_weighted_syrk(const double *X, int n, int d, int ld, const double *w, double diag, double coef,
                                double *C)
{
    __shared__ double xa[kTile][kTile + 1], xb[kTile][kTile + 1];
    const int a0 = blockIdx.y * kTile, b0 = blockIdx.x * kTile;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8 threads
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int s0 = 0; s0 < n; s0 += kTile) {
        for (int r = ty; r < kTile; r += 8) {
            const int s = s0 + r;
            const double ws = (s < n) ? (w ? w[s] : 1.0) : 0.0;
            xa[r][tx] = (s < n && a0 + tx < d) ? ws * X[(size_t)s * ld + a0 + tx] : 0.0;
            xb[r][tx] = (s < n && b0 + tx < d) ? X[(size_t)s * ld + b0 + tx] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int r = 0; r < kTile; ++r) {
            const double vb = xb[r][tx];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] += xa[r][ty + 8 * q] * vb;
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int a = a0 + ty + 8 * q, b = b0 + tx;
        if (a < d && b < d) C[(size_t)a * d + b] = coef * acc[q] + (a == b ? diag : 0.0);
    }
}

// Factor the kNb x kNb diagonal block at (k0, k0) of the lower triangle of
// A (n x n, row-major) in place: one block, the block staged in shared
// memory, column by column.  A pivot that is not positive sets *bad.
__global__ void k_potrf_diag(double *A, int n, int k0, int *bad)
{
    __shared__ double s[kNb][kNb + 1];
    const int m = min(kNb, n - k0);
    for (int t = threadIdx.x; t < kNb * kNb; t += blockDim.x) {
        const int r = t / kNb, c = t % kNb;
        s[r][c] = (r < m && c < m) ? A[(size_t)(k0 + r) * n + k0 + c] : 0.0;
    }
    __syncthreads();
    for (int j = 0; j < m; ++j) {
        if (threadIdx.x == 0) {
            const double p = s[j][j];
            if (!(p > 0.0)) {
                atomicExch(bad, 1);
                s[j][j] = 1.0;
            } else {
                s[j][j] = sqrt(p);
            }
        }
        __syncthreads();
        const double piv = s[j][j];
        for (int r = j + 1 + threadIdx.x; r < m; r += blockDim.x) s[r][j] /= piv;
        __syncthreads();
        // trailing update of the block (lower triangle)
        for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
            const int r = t / m, c = t % m;
            if (r > j && c > j && c <= r) s[r][c] -= s[r][j] * s[c][j];
        }
        __syncthreads();
    }
    for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
        const int r = t / m, c = t % m;
        if (c <= r) A[(size_t)(k0 + r) * n + k0 + c] = s[r][c];
    }
}

// Panel below the diagonal block: L[i][k0..k0+m) = A[i][k0..k0+m) L_kk^{-T}
// for i >= k0 + m.  One thread per row, forward substitution against the
// factored diagonal block (staged in shared memory).
__global__ void k_trsm_panel(double *A, int n, int k0)
{
    __shared__ double L[kNb][kNb + 1];
    const int m = min(kNb, n - k0);
    for (int t = threadIdx.x; t < kNb * kNb; t += blockDim.x) {
        const int r = t / kNb, c = t % kNb;
        L[r][c] = (r < m && c <= r) ? A[(size_t)(k0 + r) * n + k0 + c] : 0.0;
    }
    __syncthreads();
    const int i = k0 + m + blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double x[kNb];
    double *row = A + (size_t)i * n + k0;
#pragma unroll
    for (int c = 0; c < kNb; ++c) {
        if (c < m) {
            double v = row[c];
            for (int q = 0; q < c; ++q) v -= x[q] * L[c][q];
            x[c] = v / L[c][c];
        } else {
            x[c] = 0.0;
        }
    }
#pragma unroll
    for (int c = 0; c < kNb; ++c)
        if (c < m) row[c] = x[c];
}

// Trailing update of the lower triangle: A[i][j] -= sum_{t<m} L[i][k0+t] L[j][k0+t]
// for j <= i, both >= k1 = k0 + m.  32x32 tiles, tiles above the diagonal skip.
__global__ void k_syrk_trailing(double *A, int n, int k0, int m)
{
    const int k1 = k0 + m;
    const int ti = blockIdx.y * kTile, tj = blockIdx.x * kTile;
    if (tj > ti) return;
    __shared__ double li[kTile][kNb + 1], lj[kTile][kNb + 1];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int r = ty; r < kTile; r += 8) {
        const int i = k1 + ti + r, j = k1 + tj + r;
        li[r][tx] = (i < n && tx < m) ? A[(size_t)i * n + k0 + tx] : 0.0;
        lj[r][tx] = (j < n && tx < m) ? A[(size_t)j * n + k0 + tx] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int r = ty + 8 * q;
        const int i = k1 + ti + r, j = k1 + tj + tx;
        if (i < n && j <= i) {
            double v = 0.0;
#pragma unroll 8
            for (int t = 0; t < kNb; ++t) v += li[r][t] * lj[tx][t];
            A[(size_t)i * n + j] -= v;
        }
    }
}

// Forward substitution on a block of kNb rows of X (n x d): rows k0..k0+m of
// X := L_kk^{-1} X_k, one thread per column.
__global__ void k_trsv_block(const double *L, int n, double *X, int d, int k0)
{
    __shared__ double Ls[kNb][kNb + 1];
    const int m = min(kNb, n - k0);
    for (int t = threadIdx.x; t < kNb * kNb; t += blockDim.x) {
        const int r = t / kNb, c = t % kNb;
        Ls[r][c] = (r < m && c <= r) ? L[(size_t)(k0 + r) * n + k0 + c] : 0.0;
    }
    __syncthreads();
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= d) return;
    double x[kNb];
#pragma unroll
    for (int r = 0; r < kNb; ++r) {
        if (r < m) {
            double v = X[(size_t)(k0 + r) * d + col];
            for (int q = 0; q < r; ++q) v -= Ls[r][q] * x[q];
            x[r] = v / Ls[r][r];
        } else {
            x[r] = 0.0;
        }
    }
#pragma unroll
    for (int r = 0; r < kNb; ++r)
        if (r < m) X[(size_t)(k0 + r) * d + col] = x[r];
}

// X[i][:] -= L[i][k0..k0+m) X[k0..k0+m)[:] for rows i >= k0 + m: one thread
// per (row, column), the block's rows of X staged per 32 columns.
__global__ void k_trsv_update(const double *L, int n, double *X, int d, int k0, int m)
{
    __shared__ double xs[kNb][kTile + 1], ls[kTile][kNb + 1];
    const int k1 = k0 + m;
    const int r0 = k1 + blockIdx.y * kTile, c0 = blockIdx.x * kTile;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int r = ty; r < kNb; r += 8) xs[r][tx] = (r < m && c0 + tx < d) ? X[(size_t)(k0 + r) * d + c0 + tx] : 0.0;
    for (int r = ty; r < kTile; r += 8) {
        const int i = r0 + r;
        ls[r][tx] = (i < n && tx < m) ? L[(size_t)i * n + k0 + tx] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int r = ty + 8 * q;
        const int i = r0 + r, col = c0 + tx;
        if (i < n && col < d) {
            double v = 0.0;
#pragma unroll 8
            for (int t = 0; t < kNb; ++t) v += ls[r][t] * xs[t][tx];
            X[(size_t)i * d + col] -= v;
        }
    }
}

int launch_syrk(const double *X, int n, int d, int ld, const double *w, double diag, double coef, double *C,
                cudaStream_t st)
{
    const dim3 grid((d + kTile - 1) / kTile, (d + kTile - 1) / kTile);
    k_weighted_syrk<<<grid, 256, 0, st>>>(X, n, d, ld, w, diag, coef, C);
    return cuda_fail(cudaGetLastError(), "sparse-GP symmetric product");
}

}  // namespace
}  // namespace flr

extern "C" int flr_map_sgp(flr_ctx *c, int32_t species, int32_t n_sparse, const double *d_sparse,
                           const double *alpha, const double *k_ss, double sig2, double *beta_out,
                           double *gamma_out, flr_stream_t stream)
{
    using namespace flr;
    if (!c || species < 0 || species >= kSpecies || n_sparse < 1 || !d_sparse || !alpha || !k_ss ||
        !(sig2 > 0.0)) {
        set_error("flr_map_sgp: invalid argument (species in range, n_sparse >= 1, device arrays, sig2 > 0)");
        return FLR_EINVAL;
    }
    cudaSetDevice(c->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int d = c->dims.d_full;
    const int n = n_sparse;
    double *L = nullptr, *X = nullptr, *beta = nullptr, *gamma = nullptr;
    int *bad = nullptr;
    cudaError_t e = cudaMalloc(&L, sizeof(double) * n * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&X, sizeof(double) * n * (size_t)d);
    if (e == cudaSuccess) e = cudaMalloc(&beta, sizeof(double) * d * (size_t)d);
    if (e == cudaSuccess) e = cudaMalloc(&gamma, sizeof(double) * d * (size_t)d);
    if (e == cudaSuccess) e = cudaMalloc(&bad, sizeof(int));
    auto release = [&]() {
        cudaFree(L);
        cudaFree(X);
        cudaFree(beta);
        cudaFree(gamma);
        cudaFree(bad);
    };
    if (e != cudaSuccess) {
        release();
        return cuda_fail(e, "flr_map_sgp workspace");
    }
    int s = cuda_fail(cudaMemcpyAsync(L, k_ss, sizeof(double) * n * (size_t)n, cudaMemcpyDeviceToDevice, st), "K_SS");
    if (s == FLR_OK) s = cuda_fail(cudaMemcpyAsync(X, d_sparse, sizeof(double) * n * (size_t)d, cudaMemcpyDeviceToDevice, st), "D_S");
    if (s == FLR_OK) s = cuda_fail(cudaMemsetAsync(bad, 0, sizeof(int), st), "flag");
    // beta = sig2 D_S^T diag(alpha) D_S
    if (s == FLR_OK) s = launch_syrk(d_sparse, n, d, d, alpha, 0.0, sig2, beta, st);
    // K_SS = L L^T (lower, in place), panel by panel
    for (int k0 = 0; k0 < n && s == FLR_OK; k0 += kNb) {
        const int m = std::min(kNb, n - k0);
        k_potrf_diag<<<1, 256, 0, st>>>(L, n, k0, bad);
        const int rest = n - k0 - m;
        if (rest > 0) {
            k_trsm_panel<<<(rest + 127) / 128, 128, 0, st>>>(L, n, k0);
            const int nt = (rest + kTile - 1) / kTile;
            k_syrk_trailing<<<dim3(nt, nt), 256, 0, st>>>(L, n, k0, m);
        }
        s = cuda_fail(cudaGetLastError(), "Cholesky of K_SS");
    }
    // X = L^{-1} D_S
    for (int k0 = 0; k0 < n && s == FLR_OK; k0 += kNb) {
        const int m = std::min(kNb, n - k0);
        k_trsv_block<<<(d + 127) / 128, 128, 0, st>>>(L, n, X, d, k0);
        const int rest = n - k0 - m;
        if (rest > 0)
            k_trsv_update<<<dim3((d + kTile - 1) / kTile, (rest + kTile - 1) / kTile), 256, 0, st>>>(L, n, X, d, k0, m);
        s = cuda_fail(cudaGetLastError(), "substitution with L");
    }
    // gamma = sig2 I - sig2^2 X^T X
    if (s == FLR_OK) s = launch_syrk(X, n, d, d, nullptr, sig2, -sig2 * sig2, gamma, st);
    int badh = 0;
    std::vector<double> bh((size_t)d * d), gh((size_t)d * d);
    if (s == FLR_OK) s = cuda_fail(cudaMemcpyAsync(&badh, bad, sizeof(int), cudaMemcpyDeviceToHost, st), "flag");
    if (s == FLR_OK) s = cuda_fail(cudaMemcpyAsync(bh.data(), beta, sizeof(double) * bh.size(), cudaMemcpyDeviceToHost, st), "beta");
    if (s == FLR_OK) s = cuda_fail(cudaMemcpyAsync(gh.data(), gamma, sizeof(double) * gh.size(), cudaMemcpyDeviceToHost, st), "gamma");
    if (s == FLR_OK && beta_out)
        s = cuda_fail(cudaMemcpyAsync(beta_out, beta, sizeof(double) * bh.size(), cudaMemcpyDeviceToDevice, st), "beta out");
    if (s == FLR_OK && gamma_out)
        s = cuda_fail(cudaMemcpyAsync(gamma_out, gamma, sizeof(double) * gh.size(), cudaMemcpyDeviceToDevice, st), "gamma out");
    if (s == FLR_OK) s = cuda_fail(cudaStreamSynchronize(st), "flr_map_sgp");
    release();
    if (s != FLR_OK) return s;
    if (badh) {
        set_error("flr_map_sgp: K_SS is not positive definite (Cholesky pivot <= 0)");
        return FLR_EINVAL;
    }
    return flr_set_model(c, species, bh.data(), gh.data());
}
