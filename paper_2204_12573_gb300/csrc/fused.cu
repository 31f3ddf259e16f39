// One-species atoms in one kernel: descriptor -> quadratic forms on the
// tensor cores -> E, V, sigma and g (Sec. V-B, "Acceleration of
// heterogeneous multi-element system": after the species-block compaction an
// atom whose neighbours are all of one species keeps only that species'
// block of B2 -- 144 components for N = 8 -- and Eq. 1 and Eq. 2 restrict to
// the matching blocks of beta and Sigma).  These atoms are nearly all atoms
// of a slab, so their descriptor rows never leave the chip here: worker
// warps compute each 128-atom tile's normalized descriptors and write them,
// split into BF16 hi and lo parts, straight into the shared-memory A operand
// of the tensor cores (128-byte swizzled, K-major, the layout a TMA load
// would produce); [beta | Sigma] of the tile's compaction group streams
// through a shared-memory ring by TMA in 16-column K blocks (32-byte
// swizzle); one thread issues the MMAs, which accumulate P = D [beta | Sigma]
// in tensor memory (3xBF16: hi.hi + lo.hi + hi.lo, FP32 accumulation); the
// same worker warps then read P back and form E = d . beta d,
// V = d . Sigma d, sigma = sqrt(V) and g = (2/||B||)(beta d - E d), with d
// rebuilt from the hi and lo parts in shared memory.  Only E, V, sigma and
// the g row (for the force kernel) leave the kernel, beside what the force
// kernel needs from the descriptor pass (A rows, pair records, ||B||).
//
// One CTA per SM (the A tile, the B ring and the workers' staging fill the
// shared memory; the accumulator and the parked beta d take 432 of the 512
// tensor-memory columns).  Warp 0 allocates tensor memory and its lane 0
// issues the TMA loads; warp 1's lane 0 issues the MMAs; warps 2..29 are the
// 28 workers (7 per tensor-memory lane quarter).  The A tile holds K = 144
// columns without padding: two 64-column atoms with 128-byte swizzle and a
// 16-column tail with 32-byte swizzle, each MMA K step addressing its own
// block.  Tiles are taken round-robin by CTA; within the CTA's tile sequence
// the workers take rows one at a time from a shared-memory counter, so a
// worker that draws a row of the next tile computes its descriptor while the
// current tile's MMAs run, then does its share of the current tile's
// epilogue, and writes the row into the A tile once every worker has
// finished that epilogue (the epilogue reads the A tile).
//
// Every wait is bounded (about 2 s of %globaltimer); on expiry the kernel
// records FLR_ETIMEOUT, stops, waits (bounded) for its own copies and MMAs,
// frees its tensor memory and returns.
#include <algorithm>

#include "desc_dev.cuh"
#include "tc_dev.cuh"

namespace flr {
namespace {

using namespace tc;

constexpr int kFM = 128;                        // atoms per tile (MMA M)
constexpr int kFWorkers = 28;                   // worker warps, 7 per tensor-memory lane quarter
constexpr int kFSubs = kFWorkers / 4;           // workers per lane quarter
constexpr int kFThreads = 64 + 32 * kFWorkers;
constexpr int kFStages = 3;                     // B ring stages (16-column K blocks, hi and lo)
constexpr int kFBatch = 16;                     // pairs per basis batch of a worker's descriptor

template <int N>
using FWarp = DescWarp<N, kFBatch, true>;

template <int N>
struct FDims {
    static constexpr int K = N * (N + 1) / 2 * 4;       // one-species descriptor length (144 for N = 8)
    static constexpr int NA = K / 64;                   // 64-column atoms with 128-byte swizzle
    static constexpr int NT = (K - 64 * NA) / 16;       // 16-column tail blocks with 32-byte swizzle
    static constexpr int A_PART = NA * kFM * 128 + NT * kFM * 32;   // bytes of the hi (or lo) A tile
    static constexpr int KSTEPS = K / 16;               // MMA K steps of 16 BF16 values
    static constexpr int B_HALF = K * 32;               // K rows of a 16-column K block (32 bytes a row)
    static constexpr int B_PART = 2 * B_HALF;           // [beta; Sigma] rows of a K block
    static constexpr int STAGE = 2 * B_PART;            // hi and lo
    static constexpr int PARK = 2 * K;                  // first tensor-memory column of the parked beta d
    static_assert(K % 16 == 0, "K must be a multiple of 16");
    static_assert(PARK + K <= 512, "accumulator and park must fit the tensor memory");
};

template <int N>
struct FusedSmem {
    // dynamic shared memory, 1024-aligned: A hi | A lo | B ring | workers | exchange | rows | barriers
    static constexpr int OFF_A = 0;
    static constexpr int OFF_B = 2 * FDims<N>::A_PART;
    static constexpr int OFF_W = OFF_B + kFStages * FDims<N>::STAGE;
    static constexpr int OFF_X = OFF_W + kFWorkers * (int)sizeof(FWarp<N>);
    static constexpr int OFF_R = OFF_X + kFSubs * kFM * 16;
    static constexpr int OFF_BAR = OFF_R + 2 * kFM * 4;
    static constexpr int N_BARS = 2 * kFStages + 4 + 4;   // full, empty, afull, accfull, wfree, drain, evx[4]
    static constexpr int BYTES = OFF_BAR + N_BARS * 8 + 16;   // + tensor-memory address, abort flag, row counter
    static_assert(FDims<N>::A_PART % 1024 == 0, "A parts must keep 1024-byte alignment");
};

struct FusedMaps {
    CUtensorMap b[kGroups][2];     // [beta; Sigma] BF16 hi / lo per group, 16 x K boxes, 32-byte swizzle
};

struct FusedArgs {
    DescArgs d;                    // the descriptor pass (A rows, pair records, norms)
    const GroupTab *gtab;
    const int32_t *atom_of_row1;   // atoms of the one-species rows
    float *G1;                     // g rows of the one-species region [row][K]
    float *energy, *variance, *sigma;
    int var_factored[kGroups];
    int refine;
    float v_small[kGroups];
    int32_t *ref_list;
    int *ref_count;
    int ref_cap;
    int *status;
};

// A warp-wide bounded wait on an mbarrier phase (lane 0 waits, the warp
// follows its result); on failure records the timeout and raises the abort flag.
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, int lane, volatile int *abort_flag,
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
__global__ void __launch_bounds__(kFThreads, 1) k_fused(const __grid_constant__ FusedMaps maps, FusedArgs a)
{
    using D = FDims<N>;
    using L = FusedSmem<N>;
    constexpr int K = D::K;
    extern __shared__ uint8_t dyn[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(dyn) + 1023) & ~uintptr_t(1023));
    uint8_t *sAhi = base + L::OFF_A;
    uint8_t *sAlo = base + L::OFF_A + D::A_PART;
    uint8_t *sB = base + L::OFF_B;
    FWarp<N> *sW = reinterpret_cast<FWarp<N> *>(base + L::OFF_W);
    float4 *evx_buf = reinterpret_cast<float4 *>(base + L::OFF_X);
    int *atom_s = reinterpret_cast<int *>(base + L::OFF_R);
    float *norm_s = reinterpret_cast<float *>(base + L::OFF_R + kFM * 4);
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + L::OFF_BAR);
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(bars + L::N_BARS);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_holder + 1);
    int *slot_ctr = reinterpret_cast<int *>(tmem_holder + 2);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + kFStages);
    const uint32_t afull = smem_u32(bars + 2 * kFStages), accfull = smem_u32(bars + 2 * kFStages + 1);
    const uint32_t wfree = smem_u32(bars + 2 * kFStages + 2), drain = smem_u32(bars + 2 * kFStages + 3);
    const uint32_t evx0 = smem_u32(bars + 2 * kFStages + 4);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tmem_holder)), "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 32) {
        for (int s = 0; s < kFStages; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(afull, kFM);          // one arrival per row written
        mbar_init(accfull, 1);
        mbar_init(wfree, kFWorkers);
        mbar_init(drain, 1);
        for (int q = 0; q < 4; ++q) mbar_init(evx0 + 8 * q, kFSubs);
        *abort_flag = 0;
        *slot_ctr = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_holder;
    const GroupTab &T = *a.gtab;
    int pre[5];
    const int total = one_species_tiles(T, pre);
    // this CTA's tiles: blockIdx.x, blockIdx.x + gridDim.x, ...
    const int my_tiles = (int)blockIdx.x < total ? (total - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer: [beta | Sigma] K blocks ----------------
            int stage = 0;
            uint32_t phase = 0;
            int last_phase[kFStages];
            for (int s = 0; s < kFStages; ++s) last_phase[s] = -1;
            bool ok = true;
            for (int tl = 0; tl < my_tiles && ok; ++tl) {
                const OneTile ti = one_species_tile(T, pre, (int)blockIdx.x + tl * (int)gridDim.x);
                for (int ks = 0; ks < D::KSTEPS; ++ks) {
                    if (!mbar_wait(empty0 + 8 * stage, phase ^ 1, abort_flag)) { ok = false; break; }
                    const uint32_t fb = full0 + 8 * stage;
                    mbar_expect_tx(fb, D::STAGE);
                    const uint32_t sb = smem_u32(sB + stage * D::STAGE);
#pragma unroll
                    for (int part = 0; part < 2; ++part) {
                        const CUtensorMap *m = &maps.b[ti.g][part];
                        tma_load_2d(sb + part * D::B_PART, m, 16 * ks, 0, fb);
                        tma_load_2d(sb + part * D::B_PART + D::B_HALF, m, 16 * ks, K, fb);
                    }
                    last_phase[stage] = (int)phase;
                    if (++stage == kFStages) { stage = 0; phase ^= 1; }
                }
            }
            if (!ok) {
                atomicOr(a.status, kErrTimeout);
                *abort_flag = 1;
                for (int s = 0; s < kFStages; ++s)
                    if (last_phase[s] >= 0) {
                        const unsigned long long t0 = globaltimer();
                        while (!mbar_try(full0 + 8 * s, (uint32_t)last_phase[s]) && globaltimer() - t0 < kDeadlineNs) {
                        }
                    }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(K >> 3) << 17) |
                                   ((uint32_t)(kFM >> 4) << 24);
            int stage = 0;
            uint32_t phase = 0;
            bool ok = true, issued = false;
            const uint32_t ahi0 = smem_u32(sAhi), alo0 = smem_u32(sAlo);
            for (int tl = 0; tl < my_tiles && ok; ++tl) {
                // all 128 rows of this tile are written (and every worker is done
                // with the previous tile's accumulator)
                if (!mbar_wait(afull, (uint32_t)(tl & 1), abort_flag)) { ok = false; break; }
                fence_after();
                for (int ks = 0; ks < D::KSTEPS; ++ks) {
                    if (!mbar_wait(full0 + 8 * stage, phase, abort_flag)) { ok = false; break; }
                    fence_after();
                    const uint64_t ahi = ATile<N>::desc(ahi0, ks), alo = ATile<N>::desc(alo0, ks);
                    const uint32_t sb = smem_u32(sB + stage * D::STAGE);
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
                    if (++stage == kFStages) { stage = 0; phase ^= 1; }
                }
                if (ok) mma_commit(accfull);
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
        // ---------------- workers: descriptors, then their share of each epilogue ----------------
        const int wk = warp - 2;                 // worker index
        const int qw = warp & 3;                 // tensor-memory lane quarter this warp may access
        const int sub = wk >> 2;                 // which column groups of that quarter
        const uint32_t tbase = tmem + ((uint32_t)(qw * 32) << 16);
        FWarp<N> &dw = sW[wk];
        const DescArgs &da = a.d;
        bool alive = true;
        int tl_epi = 0;                          // the next tile whose epilogue this warp owes
        const int n_slots = my_tiles * kFM;
        // rows are drawn one at a time; the next row is drawn (and its atom's
        // scalars and first list entries loaded) while the current one is computed
        auto draw = [&]() -> int {
            int v = 0;
            if (lane == 0) v = atomicAdd(slot_ctr, 1);
            return __shfl_sync(0xffffffffu, v, 0);
        };
        auto atom_of_slot = [&](int sl) -> int {
            if (sl >= n_slots) return -1;
            const OneTile x = one_species_tile(T, pre, (int)blockIdx.x + (sl / kFM) * (int)gridDim.x);
            const int row = x.row0 + sl % kFM;
            return row < x.rend ? __ldg(a.atom_of_row1 + row) : -1;
        };
        // the epilogue of CTA tile tl: rows 32 qw .. 32 qw + 31, the column
        // groups sub, sub + kFSubs, ... of 8 columns
        auto epilogue = [&](int tl) -> bool {
            if (!warp_wait(afull, (uint32_t)(tl & 1), lane, abort_flag, a.status) ||
                !warp_wait(accfull, (uint32_t)(tl & 1), lane, abort_flag, a.status))
                return false;
            fence_after();
            const OneTile ti = one_species_tile(T, pre, (int)blockIdx.x + tl * (int)gridDim.x);
            const int rloc = qw * 32 + lane;
            const int atom = atom_s[rloc];
            const bool valid = atom >= 0;
            const float nrm = norm_s[rloc];
            const float s2 = nrm > 0.f ? 2.f / nrm : 0.f;
            const bool fact = a.var_factored[ti.g] != 0;
            float E = 0.f, V = 0.f, Va = 0.f;
#pragma unroll 1
            for (int c = 8 * sub; c < K; c += 8 * kFSubs) {
                float dv[8], v[8];
                ATile<N>::read_d8(sAhi, sAlo, rloc, c, dv);
                tmem_ld8(tbase + (uint32_t)c, v);
                tmem_st8(tbase + (uint32_t)(D::PARK + c), v);   // park beta d
#pragma unroll
                for (int k = 0; k < 8; ++k) E += dv[k] * v[k];
                tmem_ld8(tbase + (uint32_t)(K + c), v);
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const float tq = (fact ? v[k] : dv[k]) * v[k];
                    V += tq;
                    Va += fabsf(tq);
                }
            }
            // combine the kFSubs partial sums of each row (bounded wait, fixed order)
            evx_buf[sub * kFM + rloc] = make_float4(E, V, Va, 0.f);
            __syncwarp();
            if (lane == 0) mbar_arrive(evx0 + 8 * qw);
            if (!warp_wait(evx0 + 8 * qw, (uint32_t)(tl & 1), lane, abort_flag, a.status)) return false;
            E = 0.f;
            V = 0.f;
            Va = 0.f;
#pragma unroll
            for (int q = 0; q < kFSubs; ++q) {
                const float4 p = evx_buf[q * kFM + rloc];
                E += p.x;
                V += p.y;
                Va += p.z;
            }
            tmem_wait_st();
            float *grow = a.G1 + (size_t)(valid ? ti.row0 + rloc : 0) * K;
#pragma unroll 1
            for (int c = 8 * sub; c < K; c += 8 * kFSubs) {
                float dv[8], pv[8];
                tmem_ld8(tbase + (uint32_t)(D::PARK + c), pv);
                ATile<N>::read_d8(sAhi, sAlo, rloc, c, dv);
                if (valid) {
#pragma unroll
                    for (int k = 0; k < 8; k += 4)
                        *reinterpret_cast<float4 *>(grow + c + k) =
                            make_float4(s2 * (pv[k] - E * dv[k]), s2 * (pv[k + 1] - E * dv[k + 1]),
                                        s2 * (pv[k + 2] - E * dv[k + 2]), s2 * (pv[k + 3] - E * dv[k + 3]));
                }
            }
            if (valid && sub == 0) {
                a.energy[atom] = E;
                if (a.variance) a.variance[atom] = V;
                if (a.sigma) a.sigma[atom] = sqrtf(fmaxf(V, 0.f));
                if (a.refine && !fact && (V * kVarCancel < Va || V < a.v_small[ti.g])) {
                    const int q = atomicAdd(a.ref_count, 1);
                    if (q < a.ref_cap) a.ref_list[q] = atom;
                }
            }
            // done with the accumulator, the A tile and the row table of this tile
            fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(wfree);
            return true;
        };

        int s_cur = draw();
        int i_cur = atom_of_slot(s_cur);
        DescPre cur = desc_preload(da, i_cur < 0 ? 0x7fffffff : i_cur, 0x7fffffff, lane);
        while (s_cur < n_slots && alive) {
            const int tl = s_cur / kFM, r = s_cur % kFM;
            const int s_nx = draw();
            const int i_nx = atom_of_slot(s_nx);
            const DescPre nx = desc_preload(da, i_nx < 0 ? 0x7fffffff : i_nx, 0x7fffffff, lane);
            float nrm = 0.f;
            if (i_cur >= 0) nrm = desc_atom<N>(da, dw, lane, cur, i_cur);
            // before this row goes into the A tile: this warp's share of the
            // epilogues of the earlier tiles, then every worker's
            while (tl_epi < tl && alive) {
                alive = epilogue(tl_epi);
                ++tl_epi;
            }
            if (!alive) break;
            if (tl > 0 && !warp_wait(wfree, (uint32_t)((tl - 1) & 1), lane, abort_flag, a.status)) {
                alive = false;
                break;
            }
            if (i_cur >= 0) {
                const float inv = nrm > 0.f ? 1.f / nrm : 0.f;
                const float4 *sBv = dw.st.b.B;
                constexpr int NPS = K / 4;
#pragma unroll
                for (int k = 0; k < (NPS + 31) / 32; ++k) {
                    const int tt = lane + 32 * k;
                    if (tt < NPS) {
                        const float4 bb = sBv[tt];
                        const float4 v = make_float4(bb.x * inv, bb.y * inv, bb.z * inv, bb.w * inv);
                        const __nv_bfloat162 hi01 = __floats2bfloat162_rn(v.x, v.y);
                        const __nv_bfloat162 hi23 = __floats2bfloat162_rn(v.z, v.w);
                        const float2 f01 = __bfloat1622float2(hi01), f23 = __bfloat1622float2(hi23);
                        const __nv_bfloat162 lo01 = __floats2bfloat162_rn(v.x - f01.x, v.y - f01.y);
                        const __nv_bfloat162 lo23 = __floats2bfloat162_rn(v.z - f23.x, v.w - f23.y);
                        uint2 hv, lv;
                        hv.x = *reinterpret_cast<const uint32_t *>(&hi01);
                        hv.y = *reinterpret_cast<const uint32_t *>(&hi23);
                        lv.x = *reinterpret_cast<const uint32_t *>(&lo01);
                        lv.y = *reinterpret_cast<const uint32_t *>(&lo23);
                        const uint32_t o = ATile<N>::off(r, 4 * tt);
                        *reinterpret_cast<uint2 *>(sAhi + o) = hv;
                        *reinterpret_cast<uint2 *>(sAlo + o) = lv;
                    }
                }
            }
            if (lane == 0) {
                atom_s[r] = i_cur;
                norm_s[r] = nrm;
            }
            // the row is written: make it visible to the tensor cores, count it
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(afull);
            s_cur = s_nx;
            i_cur = i_nx;
            cur = nx;
        }
        while (tl_epi < my_tiles && alive) {
            alive = epilogue(tl_epi);
            ++tl_epi;
        }
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

int ensure_fused_maps(flr_ctx *ctx)
{
    if (ctx->fmaps) return FLR_OK;
    FusedMaps m;
    const Dims &D = ctx->dims;
    const int K = D.K[1];
    for (int g = 0; g < kGroups; ++g) {
        if (group_full(g)) {
            m.b[g][0] = m.b[g][1] = CUtensorMap{};
            continue;
        }
        int s = encode_tile_map(&m.b[g][0], ctx->Whi[g], true, D.kp64[1], D.nrows_pad[1], 16, K, 32);
        if (s == FLR_OK) s = encode_tile_map(&m.b[g][1], ctx->Wlo[g], true, D.kp64[1], D.nrows_pad[1], 16, K, 32);
        if (s != FLR_OK) return s;
    }
    ctx->fmaps = new FusedMaps(m);
    return FLR_OK;
}

template <int N>
int launch_fused_n(flr_ctx *ctx, const FusedArgs &a, cudaStream_t st)
{
    const size_t smem = 1024 + (size_t)FusedSmem<N>::BYTES;
    cudaError_t e = cudaFuncSetAttribute(k_fused<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "fused kernel attributes");
    k_fused<N><<<ctx->num_sms, kFThreads, smem, st>>>(*reinterpret_cast<const FusedMaps *>(ctx->fmaps), a);
    return FLR_OK;
}

}  // namespace

bool fused_eligible(const flr_ctx *ctx)
{
    return ctx->use_fused && ctx->p.precision == FLR_PREC_BF16X3 && ctx->p.compaction && ctx->p.n_species == 2 &&
           (ctx->dims.N == 8 || ctx->dims.N == 7) && ctx->p.l_max == 3;
}

void free_fused_maps(flr_ctx *ctx)
{
    delete reinterpret_cast<FusedMaps *>(ctx->fmaps);
    ctx->fmaps = nullptr;
}

int launch_fused(flr_ctx *ctx, const flr_nbrlist *nl, const float4 *pos, const int *species, int n,
                 flr_outputs *out, cudaStream_t st)
{
    if (n <= 0) return FLR_OK;
    int s = ensure_fused_maps(ctx);
    if (s != FLR_OK) return s;
    FusedArgs a;
    DescArgs &d = a.d;
    d.pos = pos;
    d.species = species;
    d.entries = nl->entries;
    d.count = nl->count;
    d.group = nl->group;
    d.row = nl->row;
    d.max_nbr = nl->max_nbr;
    d.n = n;
    d.cells.shift = nl->shift_d;
    d.cells.struct_of = nl->n_structs > 1 ? nl->struct_of : nullptr;
    d.rcut = (float)ctx->p.r_cut;
    d.two_over_rc = (float)(2.0 / ctx->p.r_cut);
    d.tab[0] = ctx->tab_full;
    d.tab[1] = ctx->tab_single;
    for (int r = 0; r < 2; ++r) {
        d.K[r] = ctx->dims.K[r];
        d.kp32[r] = ctx->dims.kp32[r];
        d.kp64[r] = ctx->dims.kp64[r];
        d.D32[r] = nullptr;
        d.Dhi[r] = d.Dlo[r] = nullptr;
        d.Dtf[r] = nullptr;
    }
    d.A = ctx->A;
    d.norm = ctx->norm;
    d.bf16 = 0;
    d.skip_d32_one = 0;
    d.pair_rec = nl->pair_rec;
    d.pair_cnt = nl->pair_cnt;
    d.order = nullptr;
    d.n_dev[0] = d.n_dev[1] = nullptr;
    d.sched = nullptr;
    a.gtab = nl->gtab;
    a.atom_of_row1 = nl->atom_of_row + nl->n_cap;
    a.G1 = ctx->G[1];
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
    s = ctx->dims.N == 8 ? launch_fused_n<8>(ctx, a, st) : launch_fused_n<7>(ctx, a, st);
    if (s != FLR_OK) return s;
    count_launch(ctx);
    return cuda_fail(cudaGetLastError(), "fused one-species kernel");
}

}  // namespace flr
