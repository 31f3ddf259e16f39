// Backward pass of the energy with respect to the model (Eq. 1):
//   L = sum_i u_i E_i,  E_i = d_i^T beta_{s_i} d_i
//   dL/dbeta_s = sum_{i of species s} u_i d_i d_i^T
// accumulated block by block: each compaction group contributes the outer
// products of its compact descriptor rows to the rows and columns of the
// full d x d matrix that its class uses.  One CTA owns a 32 x 32 tile of a
// group's block and walks all of the group's rows in order; groups are
// launched one after another, so every element is summed in a fixed order.
// (dL/dpositions reuses the force kernel with the weights u applied to g.)
#include "internal.cuh"

namespace flr {
namespace {

constexpr int kT = 32;

struct DbetaArgs {
    const float *D32;          // region rows [row][kp32]
    int kp32, K;
    const int32_t *atom_of_row;
    const float *u;            // [n] weights
    const GroupTab *gtab;
    int g;
    const int32_t *idx;        // compact -> full index (nullptr: identity)
    int d_full;
    float *out;                // [d_full][d_full] of the group's central species
};

__global__ void __launch_bounds__(256) k_dbeta_block(DbetaArgs a)
{
    __shared__ float sp[kT][kT + 1], sq[kT][kT + 1];
    const int tiles = (a.K + kT - 1) / kT;
    const int tp = blockIdx.x / tiles, tq = blockIdx.x % tiles;
    const int p0 = tp * kT, q0 = tq * kT;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8 threads, 4 outputs each
    const int off = a.gtab->off[a.g], cnt = a.gtab->count[a.g];
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int r0 = 0; r0 < cnt; r0 += kT) {
        // stage 32 rows: weighted columns p0.. and plain columns q0..
        for (int k = threadIdx.x; k < kT * kT; k += blockDim.x) {
            const int rr = k / kT, c = k % kT;
            const int row = off + r0 + rr;
            float vp = 0.f, vq = 0.f;
            if (r0 + rr < cnt) {
                const float *dr = a.D32 + (size_t)row * a.kp32;
                const float w = a.u[a.atom_of_row[row]];
                if (p0 + c < a.K) vp = w * dr[p0 + c];
                if (q0 + c < a.K) vq = dr[q0 + c];
            }
            sp[rr][c] = vp;
            sq[rr][c] = vq;
        }
        __syncthreads();
#pragma unroll 8
        for (int rr = 0; rr < kT; ++rr) {
            const float b = sq[rr][tx];
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[k] += sp[rr][ty + 8 * k] * b;
        }
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int p = p0 + ty + 8 * k, q = q0 + tx;
        if (p < a.K && q < a.K) {
            const int fp = a.idx ? a.idx[p] : p, fq = a.idx ? a.idx[q] : q;
            a.out[(size_t)fp * a.d_full + fq] += acc[k];
        }
    }
}

}  // namespace

int launch_dbeta(flr_ctx *ctx, const flr_nbrlist *nl, const float *u, float *grad_beta, cudaStream_t st)
{
    const Dims &D = ctx->dims;
    cudaError_t e = cudaMemsetAsync(grad_beta, 0, sizeof(float) * (size_t)kSpecies * D.d_full * D.d_full, st);
    if (e != cudaSuccess) return cuda_fail(e, "clear dL/dbeta");
    for (int g = 0; g < kGroups; ++g) {
        const int reg = group_region(g), cls = group_cls(g);
        DbetaArgs a;
        a.D32 = ctx->D32[reg];
        a.kp32 = D.kp32[reg];
        a.K = D.K[reg];
        a.atom_of_row = nl->atom_of_row + (size_t)reg * nl->n_cap;
        a.u = u;
        a.gtab = nl->gtab;
        a.g = g;
        a.idx = cls == 0 ? nullptr : ctx->tab_single + (size_t)D.d_single * cls;
        a.d_full = D.d_full;
        a.out = grad_beta + (size_t)group_species(g) * D.d_full * D.d_full;
        const int tiles = (a.K + kT - 1) / kT;
        k_dbeta_block<<<tiles * tiles, 256, 0, st>>>(a);
        count_launch(ctx);
    }
    return cuda_fail(cudaGetLastError(), "dL/dbeta");
}

}  // namespace flr
