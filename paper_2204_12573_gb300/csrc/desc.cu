// Per-atom normalized ACE-B2 descriptor (Sec. V-B "Local structure
// descriptors" and "Acceleration of heterogeneous multi-element system").
//
// One warp per atom.  Lanes first take the neighbour-list entries 32 at a
// time (coalesced row loads), evaluate the basis of the pairs inside r_cut
// and stage it in shared memory; then every lane owns 8 coefficients of A
// (radial index n = lane / 4, four harmonics, both neighbour species) and
// accumulates them over the staged pairs, so no cross-lane reduction of A is
// needed.  B2 = sum_m A_a A_b is contracted for the atom's compaction class
// only (both species blocks, or the one block its neighbours occupy),
// normalized, and written as one row of the class's GEMM operand (FP32, and
// for the 3xBF16 path also BF16 hi and lo parts).
#include "basis.cuh"
#include "internal.cuh"

namespace flr {
namespace {

constexpr int kAStride = 17;   // padded channel stride of A in shared memory

struct DescArgs {
    const float4 *pos;
    const int32_t *species;
    const int32_t *entries, *count, *group, *row;
    int max_nbr, n;
    CellArg cell;
    float rcut;
    const int32_t *tab[2];     // compact index -> (a, b, l)
    int K[2], kp32[2], kp64[2];
    float *A;                  // [n][2N*16]
    float *norm;               // [n]
    float *D32[2];
    __nv_bfloat16 *Dhi[2], *Dlo[2];
    int bf16;                  // also write BF16 hi/lo rows
};

template <int N>
struct DescSmem {
    float Rf[kWarpsDesc][32][N];
    float Y[kWarpsDesc][32][16];
    int sp[kWarpsDesc][32];
    float A[kWarpsDesc][2 * N * kAStride];
};

template <int N>
__global__ void __launch_bounds__(kWarpsDesc * 32) k_desc(DescArgs a)
{
    constexpr int KF = (2 * N) * (2 * N + 1) / 2 * 4;   // full descriptor dimension
    constexpr int NK = (KF + 31) / 32;
    __shared__ __align__(16) DescSmem<N> sm;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // persistent warps: a fixed grid walks the atoms
    for (int i = blockIdx.x * kWarpsDesc + w; i < a.n; i += gridDim.x * kWarpsDesc) {
    const int g = a.group[i];
    if (g < 0) {
        if (lane == 0) a.norm[i] = 0.f;
        continue;
    }
    const int cls = group_cls(g);
    const int reg = group_region(g);
    const float4 pi = a.pos[i];
    const int cnt = a.count[i];
    const int32_t *rowp = a.entries + (size_t)i * a.max_nbr;
    const float rc = a.rcut, rc2 = rc * rc;

    const int my_n = lane >> 2, quad = lane & 3;
    float acc0[4] = {0.f, 0.f, 0.f, 0.f}, acc1[4] = {0.f, 0.f, 0.f, 0.f};

    for (int base = 0; base < cnt; base += 32) {
        const int q = base + lane;
        bool ok = false;
        float3 r = make_float3(0.f, 0.f, 0.f);
        float d2 = 0.f;
        int sj = 0;
        if (q < cnt) {
            int j, sx, sy, sz;
            decode_entry(rowp[q], j, sx, sy, sz);
            const float4 pj = a.pos[j];
            r = pair_vector(pi, pj, sx, sy, sz, a.cell);
            d2 = r.x * r.x + r.y * r.y + r.z * r.z;
            ok = d2 < rc2;
            sj = a.species[j];
        }
        const unsigned m = __ballot_sync(0xffffffffu, ok);
        const int slot = __popc(m & ((1u << lane) - 1u));
        if (ok) {
            const float rr = sqrtf(d2);
            const float inv = 1.f / rr;
            float Rf[N], dummy[N];
            radial<N, false>(rr, rc, Rf, dummy);
            float Y[16];
            real_ylm(r.x * inv, r.y * inv, r.z * inv, Y);
#pragma unroll
            for (int n = 0; n < N; ++n) sm.Rf[w][slot][n] = Rf[n];
#pragma unroll
            for (int k = 0; k < 16; k += 4)
                *reinterpret_cast<float4 *>(&sm.Y[w][slot][k]) = make_float4(Y[k], Y[k + 1], Y[k + 2], Y[k + 3]);
            sm.sp[w][slot] = sj;
        }
        __syncwarp();
        const int nv = __popc(m);
        if (my_n < N) {
            for (int p = 0; p < nv; ++p) {
                const float rf = sm.Rf[w][p][my_n];
                const float4 y = *reinterpret_cast<const float4 *>(&sm.Y[w][p][4 * quad]);
                if (sm.sp[w][p] == 0) {
                    acc0[0] += rf * y.x; acc0[1] += rf * y.y; acc0[2] += rf * y.z; acc0[3] += rf * y.w;
                } else {
                    acc1[0] += rf * y.x; acc1[1] += rf * y.y; acc1[2] += rf * y.z; acc1[3] += rf * y.w;
                }
            }
        }
        __syncwarp();
    }

    // A to shared memory (padded) and to global memory (blocks in use only)
    float *sA = sm.A[w];
    if (my_n < N) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            sA[my_n * kAStride + 4 * quad + k] = acc0[k];
            sA[(N + my_n) * kAStride + 4 * quad + k] = acc1[k];
        }
        float *Ag = a.A + (size_t)i * (2 * N * 16);
        if (cls != 2)
            *reinterpret_cast<float4 *>(Ag + my_n * 16 + 4 * quad) = make_float4(acc0[0], acc0[1], acc0[2], acc0[3]);
        if (cls != 1)
            *reinterpret_cast<float4 *>(Ag + (N + my_n) * 16 + 4 * quad) =
                make_float4(acc1[0], acc1[1], acc1[2], acc1[3]);
    }
    __syncwarp();

    // B2 for the compaction class
    const int K = a.K[reg];
    const int32_t *tab = a.tab[reg];
    const int choff = cls == 0 ? 0 : (cls - 1) * N;
    float b[NK];
    float ss = 0.f;
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        const int o = lane + 32 * k;
        float v = 0.f;
        if (o < K) {
            const int t = __ldg(tab + o);
            const int ca = choff + (t & 255), cb = choff + ((t >> 8) & 255), l = t >> 16;
            const float *pa = sA + ca * kAStride + l * l, *pb = sA + cb * kAStride + l * l;
            for (int mm = 0; mm < 2 * l + 1; ++mm) v += pa[mm] * pb[mm];
        }
        b[k] = v;
        ss += v * v;
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    const float nrm = sqrtf(ss);
    const float inv = nrm > 0.f ? 1.f / nrm : 0.f;
    if (lane == 0) a.norm[i] = nrm;

    const int r = a.row[i];
    float *d32 = a.D32[reg] + (size_t)r * a.kp32[reg];
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        const int o = lane + 32 * k;
        if (o < a.kp32[reg]) d32[o] = o < K ? b[k] * inv : 0.f;
    }
    for (int o = NK * 32 + lane; o < a.kp32[reg]; o += 32) d32[o] = 0.f;
    if (a.bf16) {
        __nv_bfloat16 *dh = a.Dhi[reg] + (size_t)r * a.kp64[reg];
        __nv_bfloat16 *dl = a.Dlo[reg] + (size_t)r * a.kp64[reg];
#pragma unroll
        for (int k = 0; k < NK; ++k) {
            const int o = lane + 32 * k;
            if (o < a.kp64[reg]) {
                const float v = o < K ? b[k] * inv : 0.f;
                const __nv_bfloat16 hi = __float2bfloat16_rn(v);
                dh[o] = hi;
                dl[o] = __float2bfloat16_rn(v - __bfloat162float(hi));
            }
        }
        for (int o = NK * 32 + lane; o < a.kp64[reg]; o += 32) {
            dh[o] = __float2bfloat16_rn(0.f);
            dl[o] = __float2bfloat16_rn(0.f);
        }
    }
    __syncwarp();
    }  // atoms
}

// Scatter compact rows back to the full layout (for flr_compute_descriptors).
struct ExpandArgs {
    const int32_t *group, *row;
    const float *D32[2];
    int kp32[2], K[2];
    const int32_t *map_single[2];   // compact single-block index -> full index, per block t
    int n, d_full;
    float *out;
};

__global__ void k_expand(ExpandArgs a)
{
    const int i = blockIdx.x;
    if (i >= a.n) return;
    const int g = a.group[i];
    float *o = a.out + (size_t)i * a.d_full;
    for (int k = threadIdx.x; k < a.d_full; k += blockDim.x) o[k] = 0.f;
    __syncthreads();
    if (g < 0) return;
    const int reg = group_region(g), cls = group_cls(g);
    const float *src = a.D32[reg] + (size_t)a.row[i] * a.kp32[reg];
    for (int k = threadIdx.x; k < a.K[reg]; k += blockDim.x) {
        const int dst = cls == 0 ? k : __ldg(a.map_single[cls - 1] + k);
        o[dst] = src[k];
    }
}

}  // namespace

int launch_desc(flr_ctx *ctx, const flr_nbrlist *nl, const float4 *pos, const int *species, int n,
                cudaStream_t st)
{
    DescArgs a;
    a.pos = pos;
    a.species = species;
    a.entries = nl->entries;
    a.count = nl->count;
    a.group = nl->group;
    a.row = nl->row;
    a.max_nbr = nl->max_nbr;
    a.n = n;
    for (int c = 0; c < 9; ++c) a.cell.c[c] = nl->plan.cell[c];
    a.rcut = (float)ctx->p.r_cut;
    a.tab[0] = ctx->tab_full;
    a.tab[1] = ctx->tab_single;
    for (int r = 0; r < 2; ++r) {
        a.K[r] = ctx->dims.K[r];
        a.kp32[r] = ctx->dims.kp32[r];
        a.kp64[r] = ctx->dims.kp64[r];
        a.D32[r] = ctx->D32[r];
        a.Dhi[r] = ctx->Dhi[r];
        a.Dlo[r] = ctx->Dlo[r];
    }
    a.A = ctx->A;
    a.norm = ctx->norm;
    a.bf16 = ctx->p.precision == FLR_PREC_BF16X3;
    if (ctx->dims.N == 8) {
        const int grid = persistent_grid(k_desc<8>, kWarpsDesc * 32, ctx->num_sms, (n + kWarpsDesc - 1) / kWarpsDesc);
        k_desc<8><<<grid, kWarpsDesc * 32, 0, st>>>(a);
    } else {
        const int grid = persistent_grid(k_desc<7>, kWarpsDesc * 32, ctx->num_sms, (n + kWarpsDesc - 1) / kWarpsDesc);
        k_desc<7><<<grid, kWarpsDesc * 32, 0, st>>>(a);
    }
    count_launch(ctx);
    return cuda_fail(cudaGetLastError(), "descriptor kernel");
}

int launch_expand_desc(flr_ctx *ctx, const flr_nbrlist *nl, int n, float *d_hat, float *norm,
                       cudaStream_t st)
{
    ExpandArgs a;
    a.group = nl->group;
    a.row = nl->row;
    for (int r = 0; r < 2; ++r) {
        a.D32[r] = ctx->D32[r];
        a.kp32[r] = ctx->dims.kp32[r];
        a.K[r] = ctx->dims.K[r];
    }
    // the single-block index maps live after the two packed tables
    a.map_single[0] = ctx->tab_single + ctx->dims.d_single;
    a.map_single[1] = ctx->tab_single + 2 * ctx->dims.d_single;
    a.n = n;
    a.d_full = ctx->dims.d_full;
    a.out = d_hat;
    if (n > 0) k_expand<<<n, 128, 0, st>>>(a);
    count_launch(ctx);
    if (norm && n > 0) {
        cudaError_t e = cudaMemcpyAsync(norm, ctx->norm, sizeof(float) * n, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "copy norm");
    }
    return cuda_fail(cudaGetLastError(), "expand descriptors");
}

}  // namespace flr
