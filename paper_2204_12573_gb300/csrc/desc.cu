// Per-atom normalized ACE-B2 descriptor kernel (Sec. V-B "Local structure
// descriptors" and "Acceleration of heterogeneous multi-element system").
//
// Persistent warps take atoms from a work counter; each atom's descriptor is
// computed by desc_atom (desc_dev.cuh), normalized, and written as one row of
// its compaction class's quadratic-form operand (FP32, and for the 3xBF16
// path also BF16 hi and lo parts, for TF32 a copy rounded to nearest TF32).
#include "desc_dev.cuh"

namespace flr {
namespace {

template <int N>
__global__ void __launch_bounds__(kWarpsDesc * 32, 5) k_desc(DescArgs a)
{
    constexpr int C = 2 * N;
    constexpr int NPF = C * (C + 1) / 2;          // channel pairs of the full descriptor
    constexpr int NPS = N * (N + 1) / 2;          // channel pairs of a one-species block
    constexpr int MAXP = (NPF + 31) / 32;
    __shared__ DescWarp<N> sm[kWarpsDesc];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    DescWarp<N> &dw = sm[w];
    const int n_take = desc_count(a);
    // persistent warps taking chunks of the atom sequence dynamically; each
    // atom's scalars and first 64 list entries are loaded one atom ahead
    WarpChunksT<8> wc;   // 8-atom chunks: measured 0.5 % faster than 16 here
    wc.init(a.sched, n_take, lane);
    int p = wc.pos();
    const int i_end = a.order ? 0x7fffffff : a.n;
    int i = p < n_take ? (a.order ? __ldg(a.order + p) : p) : i_end;
    DescPre cur = desc_preload(a, i, i_end, lane);
    int p2 = n_take, i2 = i_end;
    DescPre nxt;
    for (; p < n_take; p = p2, i = i2, cur = nxt, wc.advance(lane)) {
        p2 = wc.peek();
        i2 = p2 < n_take ? (a.order ? __ldg(a.order + p2) : p2) : i_end;
        nxt = desc_preload(a, i2, i_end, lane);
        const int g = cur.g;
        if (g < 0) {
            if (lane == 0) a.norm[i] = 0.f;
            continue;
        }
        float4 b0;   // channel pair `lane` of B2, kept in registers
        const float nrm = desc_atom<N, DescWarp<N>, true>(a, dw, lane, cur, i, &b0);
        const float inv = nrm > 0.f ? 1.f / nrm : 0.f;
        const int cls = group_cls(g), reg = group_region(g);
        const int npairs = cls == 0 ? NPF : NPS;
        const float4 *sB = dw.st.b.B;
        const int r = cur.row;
        float *d32 = (a.skip_d32_one && reg == 1) ? nullptr : a.D32[reg] + (size_t)r * a.kp32[reg];
        __nv_bfloat16 *dh = a.bf16 ? a.Dhi[reg] + (size_t)r * a.kp64[reg] : nullptr;
        __nv_bfloat16 *dl = a.bf16 ? a.Dlo[reg] + (size_t)r * a.kp64[reg] : nullptr;
        float *dt = a.Dtf[reg] ? a.Dtf[reg] + (size_t)r * a.kp32[reg] : nullptr;
#pragma unroll
        for (int k = 0; k < MAXP; ++k) {
            const int t = lane + 32 * k;
            if (t < npairs) {
                const float4 bb = k == 0 ? b0 : sB[t];
                const float4 v = make_float4(bb.x * inv, bb.y * inv, bb.z * inv, bb.w * inv);
                if (d32) *reinterpret_cast<float4 *>(d32 + 4 * t) = v;
                if (dt)
                    *reinterpret_cast<uint4 *>(dt + 4 * t) =
                        make_uint4(tf32_round_bits(__float_as_uint(v.x)), tf32_round_bits(__float_as_uint(v.y)),
                                   tf32_round_bits(__float_as_uint(v.z)), tf32_round_bits(__float_as_uint(v.w)));
                if (dh) {
                    // hi = RN(v), lo = RN(v - hi), two values per conversion
                    const __nv_bfloat162 hi01 = __floats2bfloat162_rn(v.x, v.y);
                    const __nv_bfloat162 hi23 = __floats2bfloat162_rn(v.z, v.w);
                    const float2 f01 = __bfloat1622float2(hi01), f23 = __bfloat1622float2(hi23);
                    const __nv_bfloat162 lo01 = __floats2bfloat162_rn(v.x - f01.x, v.y - f01.y);
                    const __nv_bfloat162 lo23 = __floats2bfloat162_rn(v.z - f23.x, v.w - f23.y);
                    uint2 hv, lv;
                    hv.x = *reinterpret_cast<const uint32_t *>(&hi01); hv.y = *reinterpret_cast<const uint32_t *>(&hi23);
                    lv.x = *reinterpret_cast<const uint32_t *>(&lo01); lv.y = *reinterpret_cast<const uint32_t *>(&lo23);
                    *reinterpret_cast<uint2 *>(dh + 4 * t) = hv;
                    *reinterpret_cast<uint2 *>(dl + 4 * t) = lv;
                }
            }
        }
        // columns K.. of the rows are zero from allocation on and never written
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
                cudaStream_t st, const int32_t *order, const int *n_dev0, const int *n_dev1, bool skip_d32_one)
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
    a.cells.shift = nl->shift_d;
    a.cells.struct_of = nl->n_structs > 1 ? nl->struct_of : nullptr;
    a.rcut = (float)ctx->p.r_cut;
    a.two_over_rc = (float)(2.0 / ctx->p.r_cut);
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
    a.skip_d32_one = skip_d32_one && a.bf16 ? 1 : 0;
    for (int r = 0; r < 2; ++r) a.Dtf[r] = nullptr;
    if (ctx->p.precision == FLR_PREC_TF32) {
        // rows rounded to nearest TF32 for the tensor-core A operand, allocated
        // (and their padding zeroed) on first use at this workspace size
        if (!ctx->Dtf[0]) {
            for (int r = 0; r < 2; ++r) {
                const size_t bytes = sizeof(float) * (size_t)ctx->ws_n * ctx->dims.kp32[r];
                cudaError_t e = cudaMalloc(&ctx->Dtf[r], bytes);
                if (e == cudaSuccess) e = cudaMemset(ctx->Dtf[r], 0, bytes);
                if (e != cudaSuccess) return cuda_fail(e, "workspace TF32 rows");
            }
            ctx->maps_n = -1;   // the A maps of the tensor-core kernel point at these rows
        }
        for (int r = 0; r < 2; ++r) a.Dtf[r] = ctx->Dtf[r];
    }
    a.pair_rec = nl->pair_rec;
    a.pair_cnt = nl->pair_cnt;
    a.order = order;
    a.n_dev[0] = n_dev0;
    a.n_dev[1] = n_dev1;
    a.sched = ctx->sched;
    if (n <= 0) return FLR_OK;
    {
        const cudaError_t e = cudaMemsetAsync(ctx->sched, 0, sizeof(int), st);
        if (e != cudaSuccess) return cuda_fail(e, "descriptor work counter");
    }
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
