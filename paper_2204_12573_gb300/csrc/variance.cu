// FP64 re-evaluation of the variance V = d^T Sigma d (Eq. 2) for the atoms
// whose FP32 quadratic form cancelled.
//
// The quadratic-form epilogue accumulates, beside V = sum_k d_k (Sigma d)_k,
// the sum of the terms' magnitudes; an atom whose V is below 1/32 of it has
// lost most of its FP32 digits to cancellation (an ill-conditioned Sigma with
// d near its small-eigenvalue directions, where V is small but the terms are
// not) and is queued.  Here one warp per queued atom forms
//   u_c = sum_k d_k Sigma_kc,   V = sum_c d_c u_c
// in FP64 from the atom's FP32 descriptor row and an FP64 copy of the class
// block of Sigma (lanes over c, so every row of Sigma is read coalesced), and
// overwrites the atom's V and sigma.  FP64 is slow on this GPU, which is
// why only the queued atoms take this path.
#include "internal.cuh"

namespace flr {
namespace {

struct VarArgs {
    const int32_t *list;
    const int *count;
    int cap;
    const int32_t *group, *row;
    const float *D32[2];
    int kp32[2], K[2];
    const double *S64[kGroups];
    float *variance, *sigma;
};

__global__ void __launch_bounds__(256) k_variance_fp64(VarArgs a)
{
    __shared__ double sd[8][544];   // the atom's descriptor row in FP64 (K <= 544)
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int m = min(*a.count, a.cap);
    for (int q = blockIdx.x * 8 + w; q < m; q += gridDim.x * 8) {
        const int i = a.list[q];
        const int g = a.group[i], reg = group_region(g), K = a.K[reg];
        const float *d = a.D32[reg] + (size_t)a.row[i] * a.kp32[reg];
        for (int k = lane; k < K; k += 32) sd[w][k] = (double)d[k];
        __syncwarp();
        const double *S = a.S64[g];
        double v = 0.0;
        for (int c = lane; c < K; c += 32) {
            double u = 0.0;
            for (int k = 0; k < K; ++k) u = fma(sd[w][k], S[(size_t)k * K + c], u);
            v = fma(sd[w][c], u, v);
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) {
            if (a.variance) a.variance[i] = (float)v;
            if (a.sigma) a.sigma[i] = (float)sqrt(fmax(v, 0.0));
        }
        __syncwarp();
    }
}

}  // namespace

int launch_variance_fp64(flr_ctx *ctx, const flr_nbrlist *nl, flr_outputs *out, cudaStream_t st)
{
    if (nl->n == 0 || (!out->variance && !out->sigma)) return FLR_OK;
    VarArgs a;
    a.list = ctx->ref_list;
    a.count = ctx->ref_count;
    a.cap = ctx->ws_n;
    a.group = nl->group;
    a.row = nl->row;
    for (int r = 0; r < 2; ++r) {
        a.D32[r] = ctx->D32[r];
        a.kp32[r] = ctx->dims.kp32[r];
        a.K[r] = ctx->dims.K[r];
    }
    for (int g = 0; g < kGroups; ++g) a.S64[g] = ctx->S64[g];
    a.variance = out->variance;
    a.sigma = out->sigma;
    // the queue length is known only on the device: a fixed grid walks it
    k_variance_fp64<<<ctx->num_sms, 256, 0, st>>>(a);
    count_launch(ctx);
    return cuda_fail(cudaGetLastError(), "FP64 variance");
}

}  // namespace flr
