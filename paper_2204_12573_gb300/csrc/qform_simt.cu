// Quadratic-form products on the FP32 SIMT pipes (the plain path).
//
// For every compaction group g the rows of D_g (normalized descriptors of
// that group's atoms, one per row) are multiplied by the group's stacked
// model block, P_g = D_g [beta_g | Sigma_g] (Eq. 1 and Eq. 2 evaluated for a
// tile of atoms at once instead of one matrix-vector product per atom).
// Both operands are stored K-major: D_g[m][k] and Wt_g[n][k] = W_g[k][n]
// (beta and Sigma are symmetric).  Persistent CTAs walk a device-side tile
// table, so the launch needs no host knowledge of the group sizes.
#include "internal.cuh"

namespace flr {
namespace {

constexpr int BM = 128, BN = 144, BK = 16;
constexpr int kThreads = 256;

struct SimtArgs {
    const float *D32[2];
    int kp32[2], K[2];
    const float *W32[kGroups];
    float *P[2];
    const GroupTab *gtab;
};

__global__ void __launch_bounds__(kThreads) k_qform_simt(SimtArgs a)
{
    __shared__ __align__(16) float As[2][BK][BM + 4];
    __shared__ __align__(16) float Bs[2][BK][BN + 4];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const GroupTab &T = *a.gtab;
    const int total = T.tiles_simt[kGroups];
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        int g = 0;
        while (g < kGroups - 1 && t >= T.tiles_simt[g + 1]) ++g;
        const int reg = group_region(g);
        const int K = a.K[reg], kp = a.kp32[reg], N2 = 2 * K;
        const int ntn = (N2 + BN - 1) / BN;
        const int local = t - T.tiles_simt[g];
        const int mt = local / ntn, nt = local % ntn;
        const int r0 = T.off[g] + mt * BM, rend = T.off[g] + T.count[g];
        const int c0 = nt * BN;
        const float *Dg = a.D32[reg];
        const float *Wg = a.W32[g];

        float acc[8][9];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 9; ++j) acc[i][j] = 0.f;

        // register staging of the next K slice
        float4 ra[2];
        float4 rb[3];
        auto load_slice = [&](int k0) {
            // A: 128 rows x 16 k -> each thread 2 float4 (row = tid/2, k = (tid&1)*8 + 0/4)
            const int row = r0 + (tid >> 1);
            const int kk = k0 + (tid & 1) * 8;
#pragma unroll
            for (int h = 0; h < 2; ++h)
                ra[h] = row < rend ? *reinterpret_cast<const float4 *>(Dg + (size_t)row * kp + kk + 4 * h)
                                   : make_float4(0.f, 0.f, 0.f, 0.f);
            // B: 144 cols x 16 k = 576 float4 -> each thread up to 3
#pragma unroll
            for (int h = 0; h < 3; ++h) {
                const int idx = tid + h * kThreads;
                const int col = idx >> 2, kq = idx & 3;
                const int c = c0 + col;
                rb[h] = (idx < BN * 4 && c < N2)
                            ? *reinterpret_cast<const float4 *>(Wg + (size_t)c * kp + k0 + 4 * kq)
                            : make_float4(0.f, 0.f, 0.f, 0.f);
            }
        };
        auto store_slice = [&](int buf) {
            const int row = tid >> 1;
            const int kk = (tid & 1) * 8;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                As[buf][kk + 4 * h + 0][row] = ra[h].x;
                As[buf][kk + 4 * h + 1][row] = ra[h].y;
                As[buf][kk + 4 * h + 2][row] = ra[h].z;
                As[buf][kk + 4 * h + 3][row] = ra[h].w;
            }
#pragma unroll
            for (int h = 0; h < 3; ++h) {
                const int idx = tid + h * kThreads;
                if (idx < BN * 4) {
                    const int col = idx >> 2, kq = idx & 3;
                    Bs[buf][4 * kq + 0][col] = rb[h].x;
                    Bs[buf][4 * kq + 1][col] = rb[h].y;
                    Bs[buf][4 * kq + 2][col] = rb[h].z;
                    Bs[buf][4 * kq + 3][col] = rb[h].w;
                }
            }
        };

        const int nks = kp / BK;
        load_slice(0);
        store_slice(0);
        __syncthreads();
        for (int ks = 0; ks < nks; ++ks) {
            const int buf = ks & 1;
            if (ks + 1 < nks) load_slice((ks + 1) * BK);
#pragma unroll
            for (int k = 0; k < BK; ++k) {
                const float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][k][ty * 8]);
                const float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][k][ty * 8 + 4]);
                const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                float bv[9];
#pragma unroll
                for (int j = 0; j < 9; ++j) bv[j] = Bs[buf][k][tx + 16 * j];
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 9; ++j) acc[i][j] += av[i] * bv[j];
            }
            if (ks + 1 < nks) store_slice(buf ^ 1);
            __syncthreads();
        }
        float *Pg = a.P[reg];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int row = r0 + ty * 8 + i;
            if (row < rend) {
#pragma unroll
                for (int j = 0; j < 9; ++j) {
                    const int c = c0 + tx + 16 * j;
                    if (c < N2) Pg[(size_t)row * N2 + c] = acc[i][j];
                }
            }
        }
    }
}

// Epilogue of the SIMT path, one warp per atom: E = d . P_beta, V = d . P_Sigma,
// sigma = sqrt(V), g = (2/||B||)(P_beta - E d)  (the tensor-core kernel does
// this in its own epilogue).
struct EpiArgs {
    const int32_t *group, *row;
    const float *norm;
    const float *D32[2];
    int kp32[2], K[2];
    const float *P[2];
    float *G[2];
    float *energy, *variance, *sigma;
    int var_factored[kGroups];   // 1: P_Sigma holds L^T d, V = |L^T d|^2
    int refine;                  // queue atoms whose V cancelled for the FP64 variance
    float v_small[kGroups];      // ... or is below this (kVarSmallFP32 x |Sigma_c|_2)
    int32_t *ref_list;
    int *ref_count;
    int ref_cap;
    int n;
};

__global__ void __launch_bounds__(256) k_qform_epilogue(EpiArgs a)
{
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * 8;
    for (int i = blockIdx.x * 8 + (threadIdx.x >> 5); i < a.n; i += warps) {
        const int g = a.group[i];
        if (g < 0) continue;
        const int reg = group_region(g), K = a.K[reg], r = a.row[i];
        const float4 *d4 = reinterpret_cast<const float4 *>(a.D32[reg] + (size_t)r * a.kp32[reg]);
        const float4 *p4 = reinterpret_cast<const float4 *>(a.P[reg] + (size_t)r * (2 * K));
        float E = 0.f, V = 0.f, Va = 0.f;
        const bool fact = a.var_factored[g] != 0;
        for (int o = lane; 4 * o < K; o += 32) {
            const float4 d = d4[o], pb = p4[o], ps = p4[K / 4 + o];
            E += d.x * pb.x + d.y * pb.y + d.z * pb.z + d.w * pb.w;
            const float4 t = fact ? make_float4(ps.x * ps.x, ps.y * ps.y, ps.z * ps.z, ps.w * ps.w)
                                  : make_float4(d.x * ps.x, d.y * ps.y, d.z * ps.z, d.w * ps.w);
            V += t.x + t.y + t.z + t.w;
            Va += fabsf(t.x) + fabsf(t.y) + fabsf(t.z) + fabsf(t.w);
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            E += __shfl_xor_sync(0xffffffffu, E, o);
            V += __shfl_xor_sync(0xffffffffu, V, o);
            Va += __shfl_xor_sync(0xffffffffu, Va, o);
        }
        const float nrm = a.norm[i];
        const float s2 = nrm > 0.f ? 2.f / nrm : 0.f;
        float4 *g4 = reinterpret_cast<float4 *>(a.G[reg] + (size_t)r * K);
        for (int o = lane; 4 * o < K; o += 32) {
            const float4 d = d4[o], pb = p4[o];
            g4[o] = make_float4(s2 * (pb.x - E * d.x), s2 * (pb.y - E * d.y), s2 * (pb.z - E * d.z),
                                s2 * (pb.w - E * d.w));
        }
        if (lane == 0) {
            a.energy[i] = E;
            if (a.variance) a.variance[i] = V;
            if (a.sigma) a.sigma[i] = sqrtf(fmaxf(V, 0.f));
            if (a.refine && !fact && (V * kVarCancel < Va || V < a.v_small[g])) {
                const int q = atomicAdd(a.ref_count, 1);
                if (q < a.ref_cap) a.ref_list[q] = i;
            }
        }
    }
}

}  // namespace

int launch_qform_simt(flr_ctx *ctx, const flr_nbrlist *nl, flr_outputs *out, cudaStream_t st)
{
    SimtArgs a;
    for (int r = 0; r < 2; ++r) {
        a.D32[r] = ctx->D32[r];
        a.kp32[r] = ctx->dims.kp32[r];
        a.K[r] = ctx->dims.K[r];
        a.P[r] = ctx->P[r];
    }
    for (int g = 0; g < kGroups; ++g) a.W32[g] = ctx->W32[g];
    a.gtab = nl->gtab;
    k_qform_simt<<<ctx->num_sms * 2, kThreads, 0, st>>>(a);
    EpiArgs e;
    e.group = nl->group;
    e.row = nl->row;
    e.norm = ctx->norm;
    for (int r = 0; r < 2; ++r) {
        e.D32[r] = ctx->D32[r];
        e.kp32[r] = ctx->dims.kp32[r];
        e.K[r] = ctx->dims.K[r];
        e.P[r] = ctx->P[r];
        e.G[r] = ctx->G[r];
    }
    e.energy = out->energy;
    e.variance = out->variance;
    e.sigma = out->sigma;
    e.n = nl->n;
    for (int g = 0; g < kGroups; ++g) e.var_factored[g] = ctx->var_factored[g];
    e.refine = ctx->var_mode == FLR_VAR_AUTO;
    for (int g = 0; g < kGroups; ++g) e.v_small[g] = kVarSmallFP32 * ctx->sigma_norm[g];
    e.ref_list = ctx->ref_list;
    e.ref_count = ctx->ref_count;
    e.ref_cap = ctx->ws_n;
    k_qform_epilogue<<<persistent_grid(k_qform_epilogue, 256, ctx->num_sms, (nl->n + 7) / 8), 256, 0, st>>>(e);
    count_launch(ctx, 2);
    return cuda_fail(cudaGetLastError(), "FP32 quadratic-form GEMM");
}

}  // namespace flr
