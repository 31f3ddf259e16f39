// Per-atom normalized ACE-B2 descriptor (Sec. V-B "Local structure
// descriptors" and "Acceleration of heterogeneous multi-element system").
//
// One warp per atom (persistent warps).  Lanes take the neighbour-list
// entries 32 at a time (coalesced row loads) and compact the pairs inside
// r_cut into a per-warp queue, so the basis is evaluated only for those
// pairs with the lanes full; then every lane owns 8 coefficients of A
// (radial index n = lane / 4, four harmonics, both neighbour species) and
// accumulates them over the queued pairs, so no cross-lane reduction of A is
// needed.  B2 = sum_m A_a A_b is contracted for the atom's compaction class
// only (both species blocks, or the one block its neighbours occupy), one
// radial-channel pair (all four l) per lane from float4 rows of A,
// normalized, and written as one row of the class's GEMM operand (FP32, and
// for the 3xBF16 path also BF16 hi and lo parts).
#include "basis.cuh"
#include "internal.cuh"

namespace flr {
namespace {

constexpr int kAStride = 20;   // padded channel stride of A in shared memory (conflict-free float4 rows)

struct DescArgs {
    const float4 *pos;
    const int32_t *species;
    const int32_t *entries, *count, *group, *row;
    int max_nbr, n;
    Cells cells;               // per-structure image shifts
    float rcut;
    const int32_t *tab[2];     // compact index -> (a, b, l)
    int K[2], kp32[2], kp64[2];
    float *A;                  // [n][2N*16]
    float *norm;               // [n]
    float *D32[2];
    __nv_bfloat16 *Dhi[2], *Dlo[2];
    int bf16;                  // also write BF16 hi/lo rows
    float *Dtf[2];             // also write rows rounded to nearest TF32 (TF32 precision), or nullptr
    float4 *pair_rec;          // [n][max_nbr] out: pairs inside r_cut (r_ij, j | s_j << 25)
    int32_t *pair_cnt;         // [n] out: their number
    const int32_t *order;      // order in which atoms are taken (nullptr: by index)
    int *sched;                // work counter, zero at launch
};

constexpr int kYStride = 20;   // padded row of staged harmonics (conflict-free float4 stores)

// Per warp, the staged basis of a batch of pairs and, once the pairs are
// done, the rows of A and the unnormalized B2 (kept here between the norm
// reduction and the scaled stores instead of in registers) share one region.
template <int N>
union __align__(16) DescStage {
    struct {
        float Y[32][kYStride];           // harmonics of up to 32 staged pairs
        float Rf[N][33];                 // their radial values, pair index fastest
    } p;
    struct {
        float A[2 * N * kAStride];
        float4 B[(2 * N) * (2 * N + 1) / 2];   // unnormalized B2 of the class's channel pairs
    } b;
};

template <int N>
struct DescSmem {
    float4 rec[kWarpsDesc][64];          // compacted pairs inside r_cut: r_ij, species of j
    DescStage<N> st[kWarpsDesc];
};

// Basis of up to 32 staged pairs (lane p evaluates pair p), then the lanes
// that own A coefficients accumulate over them.  The basis is stored with the
// pairs of a species-0 neighbour first (each species keeps list order, so
// every accumulator sums in the same order as an unsorted pass), so the
// accumulation picks the accumulator by a warp-uniform index test instead of
// loading each pair's species.
template <int N>
__device__ __forceinline__ void desc_batch(DescSmem<N> &sm, int w, int lane, int m, float rc, float acc0[4],
                                           float acc1[4])
{
    float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
    if (lane < m) r = sm.rec[w][lane];
    const bool s1 = lane < m && __float_as_int(r.w) != 0;
    const unsigned b1 = __ballot_sync(0xffffffffu, s1);
    const int n0 = m - __popc(b1);
    if (lane < m) {
        const int below1 = __popc(b1 & ((1u << lane) - 1u));
        const int slot = s1 ? n0 + below1 : lane - below1;
        const float d2 = r.x * r.x + r.y * r.y + r.z * r.z;
        const float rr = sqrtf(d2), inv = 1.f / rr;
        float Rf[N], dummy[N];
        radial<N, false>(rr, rc, Rf, dummy);
        float Y[16];
        real_ylm(r.x * inv, r.y * inv, r.z * inv, Y);
#pragma unroll
        for (int n = 0; n < N; ++n) sm.st[w].p.Rf[n][slot] = Rf[n];
#pragma unroll
        for (int k = 0; k < 16; k += 4)
            *reinterpret_cast<float4 *>(&sm.st[w].p.Y[slot][k]) = make_float4(Y[k], Y[k + 1], Y[k + 2], Y[k + 3]);
    }
    __syncwarp();
    const int my_n = lane >> 2, quad = lane & 3;
    if (my_n < N) {
#pragma unroll 4
        for (int p = 0; p < m; ++p) {
            const float rf = sm.st[w].p.Rf[my_n][p];
            const float4 y = *reinterpret_cast<const float4 *>(&sm.st[w].p.Y[p][4 * quad]);
            if (p < n0) {   // warp-uniform
                acc0[0] += rf * y.x; acc0[1] += rf * y.y; acc0[2] += rf * y.z; acc0[3] += rf * y.w;
            } else {
                acc1[0] += rf * y.x; acc1[1] += rf * y.y; acc1[2] += rf * y.z; acc1[3] += rf * y.w;
            }
        }
    }
    __syncwarp();
}

// Per-atom values loaded one iteration ahead of their use.
struct DescPre {
    int g, cnt, row;
    float4 pi;
    int e0, e1;     // the first 64 neighbour-list entries (lane, 32 + lane)
};

__device__ __forceinline__ DescPre desc_preload(const DescArgs &a, int i, int i_end, int lane)
{
    DescPre p;
    p.g = -2;
    p.cnt = 0;
    p.row = 0;
    p.pi = make_float4(0.f, 0.f, 0.f, 0.f);
    p.e0 = p.e1 = 0;
    if (i < i_end) {
        // read-only loads (ld.global.nc): they may be reordered around the
        // kernel's global stores, which cannot alias them
        p.g = __ldg(a.group + i);
        p.cnt = __ldg(a.count + i);
        p.row = __ldg(a.row + i);
        p.pi = __ldg(a.pos + i);
        const int32_t *rp = a.entries + (size_t)i * a.max_nbr;
        p.e0 = __ldg(rp + lane);
        p.e1 = a.max_nbr > 32 ? __ldg(rp + 32 + lane) : 0;
    }
    return p;
}

// B2 for one radial-channel pair (a, b): all four l at once from two rows of A.
__device__ __forceinline__ float4 b2_pair(const float *sA, int a, int b)
{
    const float4 *pa = reinterpret_cast<const float4 *>(sA + a * kAStride);
    const float4 *pb = reinterpret_cast<const float4 *>(sA + b * kAStride);
    const float4 a0 = pa[0], a1 = pa[1], a2 = pa[2], a3 = pa[3];
    const float4 b0 = pb[0], b1 = pb[1], b2 = pb[2], b3 = pb[3];
    float4 o;
    o.x = a0.x * b0.x;                                                      // l = 0
    o.y = a0.y * b0.y + a0.z * b0.z + a0.w * b0.w;                          // l = 1
    o.z = a1.x * b1.x + a1.y * b1.y + a1.z * b1.z + a1.w * b1.w + a2.x * b2.x;   // l = 2
    o.w = a2.y * b2.y + a2.z * b2.z + a2.w * b2.w + a3.x * b3.x + a3.y * b3.y + a3.z * b3.z +
          a3.w * b3.w;                                                      // l = 3
    return o;
}

template <int N>
__global__ void __launch_bounds__(kWarpsDesc * 32, 4) k_desc(DescArgs a)
{
    constexpr int C = 2 * N;
    constexpr int NPF = C * (C + 1) / 2;          // channel pairs of the full descriptor
    constexpr int NPS = N * (N + 1) / 2;          // channel pairs of a one-species block
    constexpr int MAXP = (NPF + 31) / 32;
    __shared__ __align__(16) DescSmem<N> sm;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const float rc = a.rcut, rc2 = rc * rc;
    // persistent warps taking chunks of the atom sequence dynamically; each
    // atom's scalars and first 64 list entries are loaded one atom ahead
    WarpChunksT<8> wc;   // 8-atom chunks: measured 0.5 % faster than 16 here
    wc.init(a.sched, a.n, lane);
    int p = wc.pos();
    int i = p < a.n ? (a.order ? __ldg(a.order + p) : p) : a.n;
    DescPre cur = desc_preload(a, i, a.n, lane);
    int p2 = a.n, i2 = a.n;
    DescPre nxt;
    for (; p < a.n; p = p2, i = i2, cur = nxt, wc.advance(lane)) {
        p2 = wc.peek();
        i2 = p2 < a.n ? (a.order ? __ldg(a.order + p2) : p2) : a.n;
        nxt = desc_preload(a, i2, a.n, lane);
        const int g = cur.g;
        if (g < 0) {
            if (lane == 0) a.norm[i] = 0.f;
            continue;
        }
        const int cls = group_cls(g);
        const int reg = group_region(g);
        const float4 pi = cur.pi;
        const float4 *shift = a.cells.of(i);
        const int cnt = cur.cnt;
        const int32_t *rowp = a.entries + (size_t)i * a.max_nbr;

        float acc0[4] = {0.f, 0.f, 0.f, 0.f}, acc1[4] = {0.f, 0.f, 0.f, 0.f};
        int nv = 0;   // staged pairs
        int np = 0;   // pairs inside r_cut so far
        float4 *prec = a.pair_rec + (size_t)i * a.max_nbr;
        for (int base = 0; base < cnt; base += 32) {
            const int q = base + lane;
            bool ok = false;
            float3 r = make_float3(0.f, 0.f, 0.f);
            int sj = 0, j = 0;
            if (q < cnt) {
                const int e = base == 0 ? cur.e0 : (base == 32 ? cur.e1 : __ldg(rowp + q));
                j = entry_atom(e);
                const float4 pj = __ldg(a.pos + j);
                sj = entry_species(e);   // the list carries the neighbour's species: no gather
                r = pair_vector(pi, pj, entry_code(e), shift);
                ok = r.x * r.x + r.y * r.y + r.z * r.z < rc2;
            }
            const unsigned m = __ballot_sync(0xffffffffu, ok);
            if (ok) {
                const int at = __popc(m & ((1u << lane) - 1u));
                sm.rec[w][nv + at] = make_float4(r.x, r.y, r.z, __int_as_float(sj));
                // the force kernel reuses the pair vector instead of gathering and filtering again
                prec[np + at] = make_float4(r.x, r.y, r.z, __int_as_float(j | ((sj & 1) << 25)));
            }
            nv += __popc(m);
            np += __popc(m);
            __syncwarp();
            if (nv >= 32) {
                desc_batch<N>(sm, w, lane, 32, rc, acc0, acc1);
                if (lane < nv - 32) sm.rec[w][lane] = sm.rec[w][32 + lane];
                nv -= 32;
                __syncwarp();
            }
        }
        if (nv > 0) desc_batch<N>(sm, w, lane, nv, rc, acc0, acc1);
        if (lane == 0) a.pair_cnt[i] = np;

        // A to shared memory (padded rows) and to global memory (blocks in use only)
        float *sA = sm.st[w].b.A;   // the staging area is free once the pairs are done
        const int my_n = lane >> 2, quad = lane & 3;
        if (my_n < N) {
            *reinterpret_cast<float4 *>(sA + my_n * kAStride + 4 * quad) = make_float4(acc0[0], acc0[1], acc0[2], acc0[3]);
            *reinterpret_cast<float4 *>(sA + (N + my_n) * kAStride + 4 * quad) =
                make_float4(acc1[0], acc1[1], acc1[2], acc1[3]);
            float *Ag = a.A + (size_t)i * (C * 16);
            if (cls != 2)
                *reinterpret_cast<float4 *>(Ag + my_n * 16 + 4 * quad) = make_float4(acc0[0], acc0[1], acc0[2], acc0[3]);
            if (cls != 1)
                *reinterpret_cast<float4 *>(Ag + (N + my_n) * 16 + 4 * quad) =
                    make_float4(acc1[0], acc1[1], acc1[2], acc1[3]);
        }
        __syncwarp();

        // B2 of the class's channel pairs, four l per pair
        const int npairs = cls == 0 ? NPF : NPS;
        const int choff = cls == 0 ? 0 : (cls - 1) * N;
        const int32_t *tab = a.tab[reg];
        float4 *sB = sm.st[w].b.B;
        float ss = 0.f;
#pragma unroll
        for (int k = 0; k < MAXP; ++k) {
            const int t = lane + 32 * k;
            if (t < npairs) {
                const int e = __ldg(tab + 4 * t);
                const float4 bb = b2_pair(sA, choff + (e & 255), choff + ((e >> 8) & 255));
                sB[t] = bb;
                ss += bb.x * bb.x + bb.y * bb.y + bb.z * bb.z + bb.w * bb.w;
            }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        const float nrm = sqrtf(ss);
        const float inv = nrm > 0.f ? 1.f / nrm : 0.f;
        if (lane == 0) a.norm[i] = nrm;

        const int r = cur.row;
        float *d32 = a.D32[reg] + (size_t)r * a.kp32[reg];
        __nv_bfloat16 *dh = a.bf16 ? a.Dhi[reg] + (size_t)r * a.kp64[reg] : nullptr;
        __nv_bfloat16 *dl = a.bf16 ? a.Dlo[reg] + (size_t)r * a.kp64[reg] : nullptr;
        float *dt = a.Dtf[reg] ? a.Dtf[reg] + (size_t)r * a.kp32[reg] : nullptr;
#pragma unroll
        for (int k = 0; k < MAXP; ++k) {
            const int t = lane + 32 * k;
            if (t < npairs) {
                const float4 bb = sB[t];
                const float4 v = make_float4(bb.x * inv, bb.y * inv, bb.z * inv, bb.w * inv);
                *reinterpret_cast<float4 *>(d32 + 4 * t) = v;
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
    a.cells.shift = nl->shift_d;
    a.cells.struct_of = nl->n_structs > 1 ? nl->struct_of : nullptr;
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
    a.order = nullptr;
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
