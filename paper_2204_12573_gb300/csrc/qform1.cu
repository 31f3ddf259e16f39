// Quadratic forms of the one-species compaction groups on the tensor cores,
// 3xBF16 (Eq. 1, Eq. 2 restricted to one species block, Sec. V-B): P = D
// [beta | Sigma] for 128-atom tiles, K = 144 (N = 8) or 112 (N = 7), with the
// fused epilogue E, V, sigma and g = (2/||B||)(beta d - E d).  A full tile's
// g rows are staged in the freed A buffer and stored by TMA, one box per
// 8-column block, so the epilogue warps issue no scattered row stores.
//
// The tile's A operand -- the BF16 hi and lo parts of its 128 descriptor
// rows -- is loaded by TMA once and stays in shared memory for the whole
// tile (double-buffered across tiles, without padding: two 64-column atoms
// with 128-byte swizzle and a 16-column tail with 32-byte swizzle).  The
// epilogue rebuilds d = hi + lo from it, so it reads no descriptor rows from
// global memory (in the general kernel, qform_tc.cu, the epilogue's loads of
// the FP32 rows are its longest stall).  [beta | Sigma] of the tile's group
// streams through a ring of 16-column K steps (32-byte swizzle, hi and lo).
//
// Roles: warp 0 allocates tensor memory and its lane 0 issues the TMA loads
// (the next tile's A while the current one is in use); warp 1's lane 0
// issues the MMAs (two halves of N = K, beta then Sigma, three split products
// per K step, accumulating in tensor-memory columns 0 .. 2K); twelve epilogue
// warps (three per tensor-memory lane quarter) read the accumulator, park
// beta d in columns 2K .. 3K, release the accumulator for the next tile's
// MMAs, combine the partial E and V, write E, V, sigma and the g row, and
// release the A buffer.
//
// Tiles: each CTA's first is blockIdx.x, the rest are claimed from a counter
// by the producer, which hands the tile index to the MMA and epilogue warps
// with the A buffer, so CTAs that start late take fewer tiles.
//
// Every wait is bounded (about 2 s of %globaltimer); on expiry the kernel
// records FLR_ETIMEOUT, stops, waits (bounded) for its own copies and MMAs,
// frees its tensor memory and returns.
#include <algorithm>

#include "internal.cuh"
#include "tc_dev.cuh"

namespace flr {
namespace {

using namespace tc;

constexpr int kQM = 128;                      // atoms per tile
constexpr int kQSubs = 3;                     // epilogue warps per tensor-memory lane quarter
constexpr int kQEpi = 4 * kQSubs;
constexpr int kQThreads = 64 + 32 * kQEpi;
constexpr int kQStages = 3;                   // B ring stages

template <int N>
struct QDims {
    using AT = ATile<N>;
    static constexpr int K = AT::K;
    static constexpr int B_HALF = K * 32;               // K rows of a 16-column step
    static constexpr int B_PART = 2 * B_HALF;           // [beta; Sigma] rows
    static constexpr int STAGE = 2 * B_PART;            // hi and lo
    static constexpr int A_BUF = 2 * AT::PART;          // hi and lo parts of one A tile
    static constexpr int OFF_B = 2 * A_BUF;             // two A buffers, then the ring
    static constexpr int OFF_X = OFF_B + kQStages * STAGE;
    static constexpr int OFF_BAR = OFF_X + 2 * kQSubs * kQM * 16;
    // full, empty, afull[2], aempty[2], tfull, tempty, drain, evx, g staging (read, written)
    static constexpr int N_BARS = 2 * kQStages + 4 + 4 + 2;
    static constexpr int BYTES = OFF_BAR + N_BARS * 8 + 16;
    static constexpr int PARK = 2 * K;
    static constexpr int NCH = (K + 8 * kQSubs - 1) / (8 * kQSubs);   // 8-column chunks per epilogue thread
    static_assert(STAGE % 1024 == 0 && B_HALF % 256 == 0, "layout alignment");
    static_assert(PARK + K <= 512, "accumulator and park must fit the tensor memory");
};

struct Q1Maps {
    CUtensorMap a_full[2];                // BF16 hi / lo descriptor rows, 64 x 128 boxes, 128-byte swizzle
    CUtensorMap a_step[2];                // 16 x 128 boxes, 32-byte swizzle
    CUtensorMap b_step[kGroups][2];       // [beta; Sigma] rows, 16 x K boxes, 32-byte swizzle
    CUtensorMap g_rows;                   // FP32 g rows [row][K], 8 x 128 boxes, no swizzle (stores)
};

struct Q1Args {
    const GroupTab *gtab;
    const int32_t *atom_of_row1;
    float *G1;                // g rows of the one-species region [row][K]
    const float *norm;
    float *energy, *variance, *sigma;
    int var_factored[kGroups];
    int refine;
    float v_small[kGroups];
    int32_t *ref_list;
    int *ref_count;
    int ref_cap;
    int *status;
    int *tile_ctr;            // tiles past the first gridDim.x are claimed from it (zero at launch)
};

__device__ __forceinline__ bool q_warp_wait(uint32_t bar, uint32_t parity, int lane, volatile int *abort_flag,
                                            int *status)
{
    int ok = 1;
    if (lane == 0) ok = mbar_wait(bar, parity, abort_flag) ? 1 : 0;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (!ok && lane == 0) {
        atomicOr(status, kErrTimeout);
        *abort_flag = 1;
    }
    return ok != 0;
}

template <int N>
__global__ void __launch_bounds__(kQThreads, 1) k_qform1(const __grid_constant__ Q1Maps maps, Q1Args a)
{
    using D = QDims<N>;
    using AT = ATile<N>;
    constexpr int K = D::K;
    extern __shared__ uint8_t dyn[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(dyn) + 1023) & ~uintptr_t(1023));
    uint8_t *ring = base + D::OFF_B;
    float4 *evx_buf = reinterpret_cast<float4 *>(base + D::OFF_X);   // [2 tiles][kQSubs][128]
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + D::OFF_BAR);
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(bars + D::N_BARS);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_holder + 1);
    // the tile each A buffer holds, written by the producer before it arms the
    // buffer's barrier (total: no more tiles)
    volatile int *tile_of = reinterpret_cast<volatile int *>(tmem_holder + 2);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + kQStages);
    const uint32_t afull0 = smem_u32(bars + 2 * kQStages), aempty0 = smem_u32(bars + 2 * kQStages + 2);
    const uint32_t tfull = smem_u32(bars + 2 * kQStages + 4), tempty = smem_u32(bars + 2 * kQStages + 5);
    const uint32_t drain = smem_u32(bars + 2 * kQStages + 6), evx = smem_u32(bars + 2 * kQStages + 7);
    const uint32_t gread = smem_u32(bars + 2 * kQStages + 8), gwritten = smem_u32(bars + 2 * kQStages + 9);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tmem_holder)), "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 32) {
        for (int s = 0; s < kQStages; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(afull0 + 8 * b, 1);
            mbar_init(aempty0 + 8 * b, kQEpi);
        }
        mbar_init(tfull, 1);
        mbar_init(tempty, kQEpi);
        mbar_init(drain, 1);
        mbar_init(evx, kQEpi);
        mbar_init(gread, kQEpi);
        mbar_init(gwritten, kQEpi);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_holder;
    const GroupTab &T = *a.gtab;
    int pre[5];
    const int total = one_species_tiles(T, pre);

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer: A tiles and [beta | Sigma] K steps ----------------
            int stage = 0;
            uint32_t phase = 0;
            int last_phase[kQStages], last_a[2] = {-1, -1};
            for (int s = 0; s < kQStages; ++s) last_phase[s] = -1;
            bool ok = true;
            // the first tile of each CTA is blockIdx.x, later ones are claimed
            // from a counter, so CTAs that start late (their SM busy with other
            // work) take fewer tiles instead of delaying the end
            int t = blockIdx.x;
            for (int k = 0; ok; ++k) {
                const int buf = k & 1;
                // the A buffer (and its tile slot) is free once the epilogue of the tile two back has finished
                if (!mbar_wait(aempty0 + 8 * buf, (uint32_t)(((k >> 1) & 1) ^ 1), abort_flag)) { ok = false; break; }
                const uint32_t ab = afull0 + 8 * buf;
                tile_of[buf] = t < total ? t : total;
                if (t >= total) {
                    mbar_arrive(ab);   // no more tiles: release the consumers without data
                    break;
                }
                const OneTile ti = one_species_tile(T, pre, t);
                mbar_expect_tx(ab, D::A_BUF);
#pragma unroll
                for (int part = 0; part < 2; ++part) {
                    const uint32_t dst = smem_u32(base + buf * D::A_BUF + part * AT::PART);
                    for (int at = 0; at < AT::NA; ++at)
                        tma_load_2d(dst + at * (kQM * 128), &maps.a_full[part], 64 * at, ti.row0, ab);
                    for (int ts = 0; ts < AT::NT; ++ts)
                        tma_load_2d(dst + AT::NA * (kQM * 128) + ts * (kQM * 32), &maps.a_step[part],
                                    64 * AT::NA + 16 * ts, ti.row0, ab);
                }
                last_a[buf] = (k >> 1) & 1;
                const int t_next = (int)gridDim.x + atomicAdd(a.tile_ctr, 1);
                for (int ks = 0; ks < AT::KSTEPS; ++ks) {
                    if (!mbar_wait(empty0 + 8 * stage, phase ^ 1, abort_flag)) { ok = false; break; }
                    const uint32_t fb = full0 + 8 * stage;
                    mbar_expect_tx(fb, D::STAGE);
                    const uint32_t sb = smem_u32(ring + stage * D::STAGE);
#pragma unroll
                    for (int part = 0; part < 2; ++part) {
                        const CUtensorMap *m = &maps.b_step[ti.g][part];
                        tma_load_2d(sb + part * D::B_PART, m, 16 * ks, 0, fb);
                        tma_load_2d(sb + part * D::B_PART + D::B_HALF, m, 16 * ks, K, fb);
                    }
                    last_phase[stage] = (int)phase;
                    if (++stage == kQStages) { stage = 0; phase ^= 1; }
                }
                t = t_next;
            }
            if (!ok) {
                atomicOr(a.status, kErrTimeout);
                *abort_flag = 1;
                // let the copies already issued land before shared memory is released
                for (int s = 0; s < kQStages; ++s)
                    if (last_phase[s] >= 0) {
                        const unsigned long long t0 = globaltimer();
                        while (!mbar_try(full0 + 8 * s, (uint32_t)last_phase[s]) && globaltimer() - t0 < kDeadlineNs) {
                        }
                    }
                for (int b = 0; b < 2; ++b)
                    if (last_a[b] >= 0) {
                        const unsigned long long t0 = globaltimer();
                        while (!mbar_try(afull0 + 8 * b, (uint32_t)last_a[b]) && globaltimer() - t0 < kDeadlineNs) {
                        }
                    }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(K >> 3) << 17) |
                                   ((uint32_t)(kQM >> 4) << 24);
            int stage = 0;
            uint32_t phase = 0;
            bool ok = true, issued = false;
            for (int k = 0; ok; ++k) {
                const int buf = k & 1;
                if (!mbar_wait(tempty, (uint32_t)((k & 1) ^ 1), abort_flag)) { ok = false; break; }
                if (!mbar_wait(afull0 + 8 * buf, (uint32_t)((k >> 1) & 1), abort_flag)) { ok = false; break; }
                fence_after();
                if (tile_of[buf] >= total) break;
                const uint32_t ahi0 = smem_u32(base + buf * D::A_BUF), alo0 = ahi0 + AT::PART;
                for (int ks = 0; ks < AT::KSTEPS; ++ks) {
                    if (!mbar_wait(full0 + 8 * stage, phase, abort_flag)) { ok = false; break; }
                    fence_after();
                    const uint64_t ahi = AT::desc(ahi0, ks), alo = AT::desc(alo0, ks);
                    const uint32_t sb = smem_u32(ring + stage * D::STAGE);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const uint64_t bhi = sw32_desc(sb + h * D::B_HALF);
                        const uint64_t blo = sw32_desc(sb + D::B_PART + h * D::B_HALF);
                        const uint32_t td = tmem + (uint32_t)(h * K);
                        mma<true>(td, ahi, bhi, idesc, ks > 0 ? 1u : 0u);
                        mma<true>(td, alo, bhi, idesc, 1u);
                        mma<true>(td, ahi, blo, idesc, 1u);
                    }
                    issued = true;
                    mma_commit(empty0 + 8 * stage);
                    if (++stage == kQStages) { stage = 0; phase ^= 1; }
                }
                if (ok) mma_commit(tfull);
            }
            if (!ok) {
                atomicOr(a.status, kErrTimeout);
                *abort_flag = 1;
            }
            if (issued) {
                mma_commit(drain);
                const unsigned long long t0 = globaltimer();
                while (!mbar_try(drain, 0) && globaltimer() - t0 < kDeadlineNs) {
                }
            }
        }
    } else {
        // ---------------- epilogue: TMEM -> E, V, sigma, g ----------------
        const int qw = warp & 3;
        const int sub = (warp - 2) >> 2;
        const uint32_t tbase = tmem + ((uint32_t)(qw * 32) << 16);
        const int rloc = qw * 32 + lane;
        int nfull = 0;   // full tiles staged so far (the staging barriers' phase)
        bool alive = true;
        for (int k = 0; alive; ++k) {
            const int buf = k & 1;
            // the tile's A rows (TMA-written: acquire their barrier) and which tile it is
            if (!q_warp_wait(afull0 + 8 * buf, (uint32_t)((k >> 1) & 1), lane, abort_flag, a.status)) {
                alive = false;
                break;
            }
            fence_after();
            const int t = tile_of[buf];
            if (t >= total) break;
            const OneTile ti = one_species_tile(T, pre, t);
            const uint8_t *shi = base + buf * D::A_BUF, *slo = shi + AT::PART;
            const int row = ti.row0 + rloc;
            const bool valid = row < ti.rend;
            const int atom = valid ? __ldg(a.atom_of_row1 + row) : 0;
            const float nrm = valid ? __ldg(a.norm + atom) : 0.f;
            const float s2 = nrm > 0.f ? 2.f / nrm : 0.f;
            const bool fact = a.var_factored[ti.g] != 0;
            // its accumulator
            if (!q_warp_wait(tfull, (uint32_t)(k & 1), lane, abort_flag, a.status)) {
                alive = false;
                break;
            }
            fence_after();
            float E = 0.f, V = 0.f, Va = 0.f;
#pragma unroll 1
            for (int c = 8 * sub; c < K; c += 8 * kQSubs) {
                float dv[8], v[8];
                AT::read_d8(shi, slo, rloc, c, dv);
                tmem_ld8(tbase + (uint32_t)c, v);
                tmem_st8(tbase + (uint32_t)(D::PARK + c), v);   // park beta d
#pragma unroll
                for (int q = 0; q < 8; ++q) E += dv[q] * v[q];
                tmem_ld8(tbase + (uint32_t)(K + c), v);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float tq = (fact ? v[q] : dv[q]) * v[q];
                    V += tq;
                    Va += fabsf(tq);
                }
            }
            // the accumulator is free again: the next tile's MMAs overlap the rest
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty);
            // combine the partial sums of the row (double-buffered by tile, bounded wait)
            float4 *xb = evx_buf + (k & 1) * (kQSubs * kQM);
            xb[sub * kQM + rloc] = make_float4(E, V, Va, 0.f);
            __syncwarp();
            if (lane == 0) mbar_arrive(evx);
            if (!q_warp_wait(evx, (uint32_t)(k & 1), lane, abort_flag, a.status)) {
                alive = false;
                break;
            }
            E = 0.f;
            V = 0.f;
            Va = 0.f;
#pragma unroll
            for (int q = 0; q < kQSubs; ++q) {
                const float4 p = xb[q * kQM + rloc];
                E += p.x;
                V += p.y;
                Va += p.z;
            }
            tmem_wait_st();
            // g = (2/||B||)(beta d - E d).  A full tile's g goes out by TMA: once every
            // epilogue warp has read the A buffer, it becomes the tile's staging area
            // [K/8 column blocks][128 rows][8], and one thread stores each column
            // block as a box of the row-major g array.  A partial tile (the last of a
            // group) is stored by its threads, valid rows only.
            const bool full_tile = ti.rend - ti.row0 >= kQM;   // the same for every epilogue warp
            float gv[D::NCH][8];
#pragma unroll
            for (int j = 0; j < D::NCH; ++j) {
                const int c = 8 * sub + 8 * kQSubs * j;
                if (c < K) {
                    float dv[8], pv[8];
                    tmem_ld8(tbase + (uint32_t)(D::PARK + c), pv);
                    AT::read_d8(shi, slo, rloc, c, dv);
#pragma unroll
                    for (int q = 0; q < 8; ++q) gv[j][q] = s2 * (pv[q] - E * dv[q]);
                    if (!full_tile && valid) {
                        float *grow = a.G1 + (size_t)row * K + c;
                        *reinterpret_cast<float4 *>(grow) = make_float4(gv[j][0], gv[j][1], gv[j][2], gv[j][3]);
                        *reinterpret_cast<float4 *>(grow + 4) = make_float4(gv[j][4], gv[j][5], gv[j][6], gv[j][7]);
                    }
                }
            }
            if (full_tile) {
                const uint32_t ph = (uint32_t)(nfull & 1);
                __syncwarp();
                if (lane == 0) mbar_arrive(gread);
                if (!q_warp_wait(gread, ph, lane, abort_flag, a.status)) {
                    alive = false;
                    break;
                }
                float *stg = reinterpret_cast<float *>(base + buf * D::A_BUF);
#pragma unroll
                for (int j = 0; j < D::NCH; ++j) {
                    const int c = 8 * sub + 8 * kQSubs * j;
                    if (c < K) {
                        float4 *dst = reinterpret_cast<float4 *>(stg + ((size_t)(c >> 3) * kQM + rloc) * 8);
                        dst[0] = make_float4(gv[j][0], gv[j][1], gv[j][2], gv[j][3]);
                        dst[1] = make_float4(gv[j][4], gv[j][5], gv[j][6], gv[j][7]);
                    }
                }
                // the generic-proxy writes above are read by the TMA (async proxy)
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(gwritten);
                if (!q_warp_wait(gwritten, ph, lane, abort_flag, a.status)) {
                    alive = false;
                    break;
                }
                if (warp == 2 && lane == 0) {
                    for (int c8 = 0; c8 < K / 8; ++c8)
                        tma_store_2d(&maps.g_rows, smem_u32(stg + (size_t)c8 * kQM * 8), 8 * c8, ti.row0);
                    tma_store_commit();
                    tma_store_wait_read();   // the buffer may be reloaded once the stores have read it
                }
                ++nfull;
            }
            // done with this A buffer
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(aempty0 + 8 * buf);
            if (valid && sub == 0) {
                a.energy[atom] = E;
                if (a.variance) a.variance[atom] = V;
                if (a.sigma) a.sigma[atom] = sqrtf(fmaxf(V, 0.f));
                if (a.refine && !fact && (V * kVarCancel < Va || V < a.v_small[ti.g])) {
                    const int q = atomicAdd(a.ref_count, 1);
                    if (q < a.ref_cap) a.ref_list[q] = atom;
                }
            }
        }
    }
    if (warp == 2 && lane == 0) tma_store_wait_all();   // the g stores have landed
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
    // launched as a programmatic dependent: finish only after the kernel before
    // it on the stream has (nothing here reads its results; the kernels after
    // this one rely on both being complete).  Without that launch it returns at once.
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <int N>
int launch_qform1_n(flr_ctx *ctx, const Q1Args &a, cudaStream_t st, bool pdl)
{
    const size_t smem = 1024 + (size_t)QDims<N>::BYTES;
    cudaError_t e = cudaFuncSetAttribute(k_qform1<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "one-species quadratic-form kernel attributes");
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ctx->num_sms);
    cfg.blockDim = dim3(kQThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    e = cudaLaunchKernelEx(&cfg, k_qform1<N>, *reinterpret_cast<const Q1Maps *>(ctx->q1maps), a);
    return cuda_fail(e, "one-species quadratic-form kernel launch");
}

int ensure_q1_maps(flr_ctx *ctx)
{
    if (ctx->q1maps && ctx->q1maps_n == ctx->ws_n) return FLR_OK;
    Q1Maps m;
    const Dims &D = ctx->dims;
    const int K = D.K[1];
    int s = FLR_OK;
    for (int part = 0; part < 2 && s == FLR_OK; ++part) {
        const void *rows = part == 0 ? (const void *)ctx->Dhi[1] : (const void *)ctx->Dlo[1];
        s = encode_tile_map(&m.a_full[part], rows, true, D.kp64[1], ctx->ws_n, 64, kQM, 128);
        if (s == FLR_OK) s = encode_tile_map(&m.a_step[part], rows, true, D.kp64[1], ctx->ws_n, 16, kQM, 32);
    }
    // the g rows (row-major, K floats a row) for the epilogue's TMA stores
    if (s == FLR_OK) s = encode_tile_map(&m.g_rows, ctx->G[1], false, K, ctx->ws_n, 8, kQM, 0);
    for (int g = 0; g < kGroups && s == FLR_OK; ++g) {
        if (group_full(g)) {
            m.b_step[g][0] = m.b_step[g][1] = CUtensorMap{};
            continue;
        }
        for (int part = 0; part < 2 && s == FLR_OK; ++part) {
            const void *w = part == 0 ? (const void *)ctx->Whi[g] : (const void *)ctx->Wlo[g];
            s = encode_tile_map(&m.b_step[g][part], w, true, D.kp64[1], D.nrows_pad[1], 16, K, 32);
        }
    }
    if (s != FLR_OK) return s;
    if (!ctx->q1maps) ctx->q1maps = new Q1Maps();
    *reinterpret_cast<Q1Maps *>(ctx->q1maps) = m;
    ctx->q1maps_n = ctx->ws_n;
    return FLR_OK;
}

}  // namespace

void free_q1_maps(flr_ctx *ctx)
{
    delete reinterpret_cast<Q1Maps *>(ctx->q1maps);
    ctx->q1maps = nullptr;
}

int launch_qform1(flr_ctx *ctx, const flr_nbrlist *nl, flr_outputs *out, cudaStream_t st, bool pdl)
{
    int s = ensure_q1_maps(ctx);
    if (s != FLR_OK) return s;
    Q1Args a;
    a.gtab = nl->gtab;
    a.atom_of_row1 = nl->atom_of_row + nl->n_cap;
    a.G1 = ctx->G[1];
    a.norm = ctx->norm;
    a.energy = out->energy;
    a.variance = out->variance;
    a.sigma = out->sigma;
    for (int g = 0; g < kGroups; ++g) {
        a.var_factored[g] = ctx->var_factored[g];
        a.v_small[g] = kVarSmallBF16x3 * ctx->sigma_norm[g];
    }
    a.refine = ctx->var_mode == FLR_VAR_AUTO;
    a.ref_list = ctx->ref_list;
    a.ref_count = ctx->ref_count;
    a.ref_cap = ctx->ws_n;
    a.status = ctx->status;
    a.tile_ctr = ctx->sched + 4;
    s = ctx->dims.N == 8 ? launch_qform1_n<8>(ctx, a, st, pdl) : launch_qform1_n<7>(ctx, a, st, pdl);
    if (s != FLR_OK) return s;
    count_launch(ctx);
    return cuda_fail(cudaGetLastError(), "one-species quadratic-form kernel");
}

}  // namespace flr
