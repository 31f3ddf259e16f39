// Quadratic-form products on the 5th-generation tensor cores (tcgen05),
// with the energy / variance / gradient epilogue fused.
//
// For a tile of 128 atoms of one compaction group the kernel forms
// P = D_g [beta_g | Sigma_g] (Eq. 1, Eq. 2) 288 columns at a time:
//   * TF32: FP32 operands read as TF32 (kind::tf32), FP32 accumulation;
//   * 3xBF16: both operands split into BF16 hi + lo parts; the K loop runs
//     three times (hi.hi, hi.lo, lo.hi), the lo.lo term is dropped, so the
//     product keeps about 16 significant bits (kind::f16, FP32 accumulate).
// Operand tiles arrive by TMA (128-byte swizzle) into a 3-stage shared
// memory ring guarded by mbarriers; one thread issues the MMAs, which
// accumulate in tensor memory (288 of 512 columns).  Twelve epilogue warps
// (three per TMEM lane quarter, each taking every third 16-column group)
// read the accumulator back with tcgen05.ld, one atom (row) per thread:
//   E = d . (beta d),  V = d . (Sigma d),  sigma = sqrt(V),
//   g = dE/dB = (2/||B||)(beta d - E d)
// and store E, V, sigma per atom and g as the row the force kernel needs,
// so P itself never goes to memory.  A one-species tile (d = 144) is a
// single 288-column chunk whose beta d columns are parked in the free TMEM
// columns 288..431 until E is final; a two-species tile (d = 544) takes
// four chunks of the same CTA, the partial E and V living in the epilogue
// registers and the beta d columns parked in the g row.
//
// Every wait on an mbarrier has a deadline (about 2 s of %globaltimer); on
// expiry the kernel records FLR_ETIMEOUT in the status word, stops issuing
// work, waits (again bounded) for its own copies and MMAs in flight, frees
// its tensor memory and returns.
#include <cuda.h>

#include <algorithm>

#include "internal.cuh"
#include "tc_dev.cuh"

namespace flr {
namespace {

constexpr int BM = 128;
constexpr int NH = 144;            // N of one MMA
constexpr int NC = 2 * NH;         // columns per chunk (one accumulator)
constexpr int kStages = 3;          // three 52 KB stages in flight (measured: 2 and 4 are slower; 4 leaves the epilogue little L1)
constexpr int kTileA = BM * 128;   // bytes (128-byte rows)
constexpr int kTileB = NC * 128;
constexpr int kStageBytes = kTileA + kTileB;
constexpr int kTmemCols = 512;
constexpr int kSubs = 3;            // epilogue warps per TMEM lane quarter (each takes every 3rd 16-column group)
constexpr int kParkCols = 144;      // widest one-species row parked in tensor memory
constexpr int kParkCol0 = NC;       // first TMEM column of the park (after the accumulator)
static_assert(kParkCol0 + kParkCols <= 512, "accumulator and park must fit in 512 TMEM columns");
constexpr int kParkGroups = (kParkCols / 16 + kSubs - 1) / kSubs;   // 16-column groups per epilogue thread
constexpr int kEpiWarps = 4 * kSubs;
constexpr int kThreads = 64 + 32 * kEpiWarps;
using namespace tc;

struct TcArgs {
    int K[2];
    int kp32[2];
    int nkb[2];          // K blocks of 128 bytes per part
    int nch[kGroups];    // 288-column chunks per group
    const float *D32[2]; // FP32 descriptor rows (epilogue dot products)
    float *G[2];         // out: g rows [row][K]
    const int32_t *atom_of_row;
    int n_cap;
    const float *norm;
    float *energy, *variance, *sigma;
    const GroupTab *gtab;
    int var_factored[kGroups];   // 1: the Sigma columns hold L^T d, V = |L^T d|^2
    int refine;                  // queue atoms whose V cancelled for the FP64 variance
    float v_small[kGroups];      // ... or is below this (kVarSmall* x |Sigma_c|_2)
    int32_t *ref_list;
    int *ref_count;
    int ref_cap;
    int *status;
    int only_full;               // take only the tiles of the two-species groups
};

struct TileInfo {
    int g, reg, row0, rend, nch;
};
__device__ __forceinline__ TileInfo decode_tile(const GroupTab &T, const int *nchunks, int t)
{
    TileInfo ti;
    int g = 0;
    while (g < kGroups - 1 && t >= T.tiles_tc[g + 1]) ++g;
    ti.g = g;
    ti.reg = group_region(g);
    ti.row0 = T.off[g] + (t - T.tiles_tc[g]) * BM;
    ti.rend = T.off[g] + T.count[g];
    ti.nch = nchunks[g];
    return ti;
}

// The tiles a launch takes: all of them, or (only_full) the two-species
// groups' tiles alone, numbered 0 .. count-1 so that consecutive CTAs take
// consecutive ones and no CTA gets a second tile before every CTA has one.
__device__ __forceinline__ int tc_tile_count(const TcArgs &a, const GroupTab &T)
{
    if (!a.only_full) return T.tiles_tc[kGroups];
    int m = 0;
#pragma unroll
    for (int g = 0; g < kGroups; ++g)
        if (group_full(g)) m += T.tiles_tc[g + 1] - T.tiles_tc[g];
    return m;
}
__device__ __forceinline__ int tc_tile(const TcArgs &a, const GroupTab &T, int u)
{
    if (!a.only_full) return u;
#pragma unroll
    for (int g = 0; g < kGroups; ++g) {
        if (!group_full(g)) continue;
        const int m = T.tiles_tc[g + 1] - T.tiles_tc[g];
        if (u < m) return T.tiles_tc[g] + u;
        u -= m;
    }
    return T.tiles_tc[kGroups];
}

// d[c .. c+15] of a descriptor row (four float4 loads through the read-only
// path, so they may be issued ahead of the g-row stores; c is a multiple of 4)
__device__ __forceinline__ void load16(const float *p, float v[16])
{
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float4 q = __ldg(reinterpret_cast<const float4 *>(p + 4 * k));
        v[4 * k] = q.x;
        v[4 * k + 1] = q.y;
        v[4 * k + 2] = q.z;
        v[4 * k + 3] = q.w;
    }
}

// Epilogue: wait for a full accumulator (lane 0 waits, the warp follows its
// result, so the warp stays converged); false on timeout or abort.
__device__ __forceinline__ bool acc_wait(uint32_t tfull, int it, int lane, volatile int *abort_flag, int *status)
{
    int okw = 1;
    if (lane == 0) okw = mbar_wait(tfull, (uint32_t)(it & 1), abort_flag) ? 1 : 0;
    okw = __shfl_sync(0xffffffffu, okw, 0);
    if (!okw && lane == 0) {
        atomicOr(status, kErrTimeout);
        *abort_flag = 1;
    }
    if (okw) fence_after();
    return okw != 0;
}

// While the MMAs of the next tile run, pull this thread's descriptor row of
// tile tn into L2, so that tile's reads of it do not wait on DRAM.
__device__ __forceinline__ void prefetch_next_rows(const TcArgs &a, const GroupTab &T, int tn, int total, int rloc,
                                                   int sub)
{
    if (tn >= total) return;
    const TileInfo tj = decode_tile(T, a.nch, tc_tile(a, T, tn));
    const int rown = tj.row0 + rloc;
    if (rown >= tj.rend) return;
    const char *dn = reinterpret_cast<const char *>(a.D32[tj.reg] + (size_t)rown * a.kp32[tj.reg]);
    const int bytes = 4 * a.K[tj.reg];
    for (int o = 128 * sub; o < bytes; o += 128 * kSubs) asm volatile("prefetch.global.L2 [%0];" ::"l"(dn + o));
}

// Combine the partial E, V, sum|.| of the kSubs column sets of a row through
// shared memory (double-buffered by tile, bounded mbarrier wait, fixed order).
__device__ __forceinline__ bool exchange(float4 *evx_buf, uint32_t evx, int tl, int sub, int rloc, int lane,
                                         volatile int *abort_flag, int *status, float &E, float &V, float &Va)
{
    float4 *xb = evx_buf + (tl & 1) * (kSubs * BM);
    xb[sub * BM + rloc] = make_float4(E, V, Va, 0.f);
    __syncwarp();
    int okx = 1;
    if (lane == 0) {
        mbar_arrive(evx);
        okx = mbar_wait(evx, (uint32_t)(tl & 1), abort_flag) ? 1 : 0;
    }
    okx = __shfl_sync(0xffffffffu, okx, 0);
    __syncwarp();
    if (!okx) {
        if (lane == 0) {
            atomicOr(status, kErrTimeout);
            *abort_flag = 1;
        }
        return false;
    }
    E = 0.f;
    V = 0.f;
    Va = 0.f;
#pragma unroll
    for (int q = 0; q < kSubs; ++q) {
        const float4 p = xb[q * BM + rloc];
        E += p.x;
        V += p.y;
        Va += p.z;
    }
    return true;
}

template <bool BF16>
__global__ void __launch_bounds__(kThreads, 1) k_qform_tc(const __grid_constant__ TcMaps maps, TcArgs a)
{
    // a kernel launched after this one as a programmatic dependent (the
    // one-species tiles) may start once every CTA of this grid is resident:
    // it takes the SMs this grid's few two-species tiles leave free
    asm volatile("griddepcontrol.launch_dependents;");
    extern __shared__ uint8_t dyn[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(dyn) + 1023) & ~uintptr_t(1023));
    uint8_t *sA = base;
    uint8_t *sB = base + kStages * kTileA;
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + kStages * kStageBytes);
    // bars: full[kStages], empty[kStages], tfull, tempty, drain, evx
    uint32_t *tmem_holder = reinterpret_cast<uint32_t *>(bars + 2 * kStages + 4);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_holder + 1);
    // partial (E, V, sum |d_k (Sigma d)_k|) of each row from the kSubs column
    // sets, double-buffered by tile
    float4 *evx_buf = reinterpret_cast<float4 *>(base + kStages * kStageBytes + 128);
    // beta d of one-species tiles, parked until E is known (padded rows: conflict-free float4 access)

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + kStages);
    const uint32_t tfull = smem_u32(bars + 2 * kStages), tempty = smem_u32(bars + 2 * kStages + 1);
    const uint32_t drain = smem_u32(bars + 2 * kStages + 2);
    const uint32_t evx = smem_u32(bars + 2 * kStages + 3);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"(smem_u32(tmem_holder)), "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (threadIdx.x == 32) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(full0 + 8 * s, 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        mbar_init(tfull, 1);
        mbar_init(tempty, kEpiWarps);
        mbar_init(drain, 1);
        mbar_init(evx, kEpiWarps);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tmem_holder;
    const GroupTab &T = *a.gtab;
    const int total = tc_tile_count(a, T);

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer ----------------
            int stage = 0;
            uint32_t phase = 0;
            int last_phase[kStages];
            for (int s = 0; s < kStages; ++s) last_phase[s] = -1;
            bool ok = true;
            for (int u = blockIdx.x; u < total && ok; u += gridDim.x) {
                const TileInfo ti = decode_tile(T, a.nch, tc_tile(a, T, u));
                const int nkb = a.nkb[ti.reg];
                const int nkt = BF16 ? 3 * nkb : nkb;
                for (int ch = 0; ch < ti.nch && ok; ++ch) {
                    for (int kb = 0; kb < nkt; ++kb) {
                        const int part = BF16 ? kb / nkb : 0;
                        const int kk = BF16 ? kb % nkb : kb;
                        if (!mbar_wait(empty0 + 8 * stage, phase ^ 1, abort_flag)) { ok = false; break; }
                        const uint32_t fb = full0 + 8 * stage;
                        mbar_expect_tx(fb, kStageBytes);
                        const int x = kk * (BF16 ? 64 : 32);
                        const CUtensorMap *am = &maps.a[ti.reg][(BF16 && part == 2) ? 1 : 0];
                        const CUtensorMap *bm = &maps.b[ti.g][(BF16 && part == 1) ? 1 : 0];
                        const uint32_t da = smem_u32(sA + stage * kTileA);
                        const uint32_t db = smem_u32(sB + stage * kTileB);
                        tma_load_2d(da, am, x, ti.row0, fb);
                        tma_load_2d(db, bm, x, ch * NC, fb);
                        tma_load_2d(db + NH * 128, bm, x, ch * NC + NH, fb);
                        last_phase[stage] = (int)phase;
                        if (++stage == kStages) { stage = 0; phase ^= 1; }
                    }
                }
            }
            if (!ok) {
                atomicOr(a.status, kErrTimeout);
                *abort_flag = 1;
                // let the copies already issued land before shared memory is released
                for (int s = 0; s < kStages; ++s)
                    if (last_phase[s] >= 0) {
                        const unsigned long long t0 = globaltimer();
                        while (!mbar_try(full0 + 8 * s, (uint32_t)last_phase[s]) &&
                               globaltimer() - t0 < kDeadlineNs) {
                        }
                    }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer ----------------
            const uint32_t fmt = BF16 ? 1u : 2u;   // BF16 or TF32 operands
            const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(NH >> 3) << 17) |
                                   ((uint32_t)(BM >> 4) << 24);
            int stage = 0;
            uint32_t phase = 0;
            int it = 0;   // accumulator uses (chunks)
            bool ok = true;
            bool issued = false;
            for (int u = blockIdx.x; u < total && ok; u += gridDim.x) {
                const TileInfo ti = decode_tile(T, a.nch, tc_tile(a, T, u));
                const int nkb = a.nkb[ti.reg];
                const int nkt = BF16 ? 3 * nkb : nkb;
                const int K = a.K[ti.reg];
                for (int ch = 0; ch < ti.nch && ok; ++ch, ++it) {
                    if (!mbar_wait(tempty, (uint32_t)((it & 1) ^ 1), abort_flag)) { ok = false; break; }
                    fence_after();
                    for (int kb = 0; kb < nkt; ++kb) {
                        if (!mbar_wait(full0 + 8 * stage, phase, abort_flag)) { ok = false; break; }
                        fence_after();
                        const uint32_t da = smem_u32(sA + stage * kTileA);
                        const uint32_t db = smem_u32(sB + stage * kTileB);
                        const uint64_t ad = sw128_desc(da);
                        const uint64_t bd0 = sw128_desc(db), bd1 = sw128_desc(db + NH * 128);
                        // K steps past K (the zero padding of the last block) are skipped
                        const int kk = BF16 ? kb % nkb : kb;
                        const int kleft = K - kk * (BF16 ? 64 : 32);
#pragma unroll
                        for (int ks = 0; ks < 4; ++ks) {
                            if (ks * (BF16 ? 16 : 8) >= kleft) break;
                            const uint32_t accum = (kb | ks) != 0;
                            mma<BF16>(tmem, ad + 2 * ks, bd0 + 2 * ks, idesc, accum);
                            mma<BF16>(tmem + NH, ad + 2 * ks, bd1 + 2 * ks, idesc, accum);
                        }
                        issued = true;
                        mma_commit(empty0 + 8 * stage);
                        if (++stage == kStages) { stage = 0; phase ^= 1; }
                    }
                    if (ok) mma_commit(tfull);
                }
            }
            if (!ok) {
                atomicOr(a.status, kErrTimeout);
                *abort_flag = 1;
            }
            if (issued) {
                // drain: wait until every MMA this thread issued has completed
                mma_commit(drain);
                const unsigned long long t0 = globaltimer();
                while (!mbar_try(drain, 0) && globaltimer() - t0 < kDeadlineNs) {
                }
            }
        }
    } else {
        // ---------------- epilogue: TMEM -> E, V, sigma, g ----------------
        // Warp (quarter qw, set sub) reads TMEM lanes 32 qw .. 32 qw + 31 (one
        // row per thread) and every kSubs-th 16-column group starting at sub.
        // The kSubs partial E and V of a row are combined through shared
        // memory (double-buffered by tile, guarded by a bounded mbarrier wait).
        // One-species tiles park beta d in tensor memory beside the accumulator
        // (columns kParkCol0..), so the accumulator is released as soon as it
        // is read and g = s2 (beta d - E d) is formed without a round trip
        // through global memory; two-species tiles (four column chunks) park
        // beta d in the g row and fix it up afterwards.
        const int qw = warp & 3;                // TMEM lane quarter of this warp
        const int sub = (warp - 2) >> 2;        // which column groups
        const uint32_t tbase = tmem + ((uint32_t)(qw * 32) << 16);
        const int rloc = qw * 32 + lane;        // row within the tile
        int it = 0;
        int tl = 0;                             // tiles done by this CTA
        bool alive = true;
        for (int u = blockIdx.x; u < total && alive; u += gridDim.x) {
            const TileInfo ti = decode_tile(T, a.nch, tc_tile(a, T, u));
            const int K = a.K[ti.reg];
            const int row = ti.row0 + rloc;
            const bool valid = row < ti.rend;
            const int atom = valid ? a.atom_of_row[(size_t)ti.reg * a.n_cap + row] : 0;
            const float nrm = valid ? a.norm[atom] : 0.f;
            const float *d = a.D32[ti.reg] + (size_t)(valid ? row : 0) * a.kp32[ti.reg];
            float *grow = a.G[ti.reg] + (size_t)(valid ? row : 0) * K;
            const float s2 = nrm > 0.f ? 2.f / nrm : 0.f;
            const bool fact = a.var_factored[ti.g] != 0;
            const bool in_smem = ti.nch == 1 && (K % 16) == 0 && 2 * K <= NC && K <= kParkCols;
            float E = 0.f, V = 0.f, Va = 0.f;
            if (in_smem) {
                // one-species tile: one chunk holding [beta d | Sigma d]; this
                // thread takes at most kParkGroups groups of 16 columns
                if (!acc_wait(tfull, it, lane, abort_flag, a.status)) {
                    alive = false;
                    break;
                }
                ++it;
#pragma unroll
                for (int j = 0; j < kParkGroups; ++j) {
                    const int c = 16 * (sub + kSubs * j);
                    if (c >= K) break;
                    float dv[16];
                    if (valid) {
                        load16(d + c, dv);
                    } else {
#pragma unroll
                        for (int k = 0; k < 16; ++k) dv[k] = 0.f;
                    }
                    float v[16];
                    tmem_ld16(tbase + (uint32_t)c, v);
                    tmem_st16(tbase + (uint32_t)(kParkCol0 + c), v);   // park beta d beside the accumulator
#pragma unroll
                    for (int k = 0; k < 16; ++k) E += dv[k] * v[k];
                    tmem_ld16(tbase + (uint32_t)(K + c), v);
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        const float tq = (fact ? v[k] : dv[k]) * v[k];
                        V += tq;
                        Va += fabsf(tq);
                    }
                }
                // the accumulator is free again: the next MMAs overlap the rest below
                fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(tempty);
                prefetch_next_rows(a, T, u + gridDim.x, total, rloc, sub);
                if (!exchange(evx_buf, evx, tl, sub, rloc, lane, abort_flag, a.status, E, V, Va)) {
                    alive = false;
                    break;
                }
                tmem_wait_st();
                // g = (2/||B||)(beta d - E d) from the parked beta d (d read again);
                // the tensor-memory reads are warp-collective, so every lane takes part
#pragma unroll
                for (int j = 0; j < kParkGroups; ++j) {
                    const int c = 16 * (sub + kSubs * j);
                    if (c >= K) break;
                    float pv[16];
                    tmem_ld16(tbase + (uint32_t)(kParkCol0 + c), pv);
                    if (valid) {
#pragma unroll
                        for (int k = 0; k < 16; k += 4) {
                            const float4 q = __ldg(reinterpret_cast<const float4 *>(d + c + k));
                            *reinterpret_cast<float4 *>(grow + c + k) =
                                make_float4(s2 * (pv[k] - E * q.x), s2 * (pv[k + 1] - E * q.y),
                                            s2 * (pv[k + 2] - E * q.z), s2 * (pv[k + 3] - E * q.w));
                        }
                    }
                }
            } else {
                // two-species tile: column chunks of NC, beta d parked in the g row
                for (int ch = 0; ch < ti.nch; ++ch, ++it) {
                    if (!acc_wait(tfull, it, lane, abort_flag, a.status)) {
                        alive = false;
                        break;
                    }
                    const int c0 = ch * NC;
#pragma unroll 1
                    for (int c = 16 * sub; c < NC; c += 16 * kSubs) {
                        const int cg = c0 + c;
                        float v[16], dv[16];
                        const bool beta_cols = cg + 16 <= K, sigma_cols = cg >= K && cg + 16 <= 2 * K;
                        if (valid && beta_cols) load16(d + cg, dv);
                        else if (valid && sigma_cols && !fact) load16(d + cg - K, dv);
                        tmem_ld16(tbase + (uint32_t)c, v);
                        if (valid && cg < 2 * K) {
                            if (beta_cols) {
#pragma unroll
                                for (int k = 0; k < 16; ++k) E += dv[k] * v[k];
#pragma unroll
                                for (int k = 0; k < 16; k += 4)
                                    *reinterpret_cast<float4 *>(grow + cg + k) = make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
                            } else if (sigma_cols) {
#pragma unroll
                                for (int k = 0; k < 16; ++k) {
                                    const float tq = (fact ? v[k] : dv[k]) * v[k];
                                    V += tq;
                                    Va += fabsf(tq);
                                }
                            } else {                                  // a group straddling K or 2K
#pragma unroll
                                for (int k = 0; k < 16; ++k) {
                                    const int cc = cg + k;
                                    if (cc < K) {
                                        E += __ldg(d + cc) * v[k];
                                        grow[cc] = v[k];
                                    } else if (cc < 2 * K) {
                                        const float tq = (fact ? v[k] : __ldg(d + cc - K)) * v[k];
                                        V += tq;
                                        Va += fabsf(tq);
                                    }
                                }
                            }
                        }
                    }
                    // the accumulator is free again: the next MMAs overlap the rest below
                    fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(tempty);
                }
                if (!alive) break;
                prefetch_next_rows(a, T, u + gridDim.x, total, rloc, sub);
                if (!exchange(evx_buf, evx, tl, sub, rloc, lane, abort_flag, a.status, E, V, Va)) {
                    alive = false;
                    break;
                }
                if (valid) {
                    // g = (2/||B||)(beta d - E d) over the 16-column groups this set parked
                    float4 *g4 = reinterpret_cast<float4 *>(grow);
                    const float4 *d4 = reinterpret_cast<const float4 *>(d);
                    const int nk = K / 4;
#pragma unroll 1
                    for (int k0 = 4 * sub; k0 < nk; k0 += 4 * kSubs) {
                        float4 p[4], q[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            if (k0 + u < nk) {
                                p[u] = g4[k0 + u];
                                q[u] = __ldg(d4 + k0 + u);
                            }
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            if (k0 + u < nk)
                                g4[k0 + u] = make_float4(s2 * (p[u].x - E * q[u].x), s2 * (p[u].y - E * q[u].y),
                                                         s2 * (p[u].z - E * q[u].z), s2 * (p[u].w - E * q[u].w));
                    }
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
            ++tl;   // tiles this CTA processed (the exchange buffer's parity)
        }
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn get_encoder()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

int encode(CUtensorMap *m, const void *ptr, bool bf16, int cols, int rows, int box_rows)
{
    return encode_tile_map(m, ptr, bf16, cols, rows, 128 / (bf16 ? 2 : 4), box_rows, 128);
}

}  // namespace

// A 2-D row-major tensor map (FP32 or BF16) with a box of box_cols x box_rows
// and the given swizzle width (32, 64 or 128 bytes; box_cols x element size
// must equal it), or none (0).
int encode_tile_map(CUtensorMap *m, const void *ptr, bool bf16, int cols, int rows, int box_cols, int box_rows,
                    int swizzle_bytes)
{
    EncodeTiledFn fn = get_encoder();
    if (!fn) {
        set_error("cuTensorMapEncodeTiled is not available from the driver");
        return FLR_ECUDA;
    }
    const int esz = bf16 ? 2 : 4;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * esz};
    cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    const CUtensorMapSwizzle sw = swizzle_bytes == 0    ? CU_TENSOR_MAP_SWIZZLE_NONE
                                  : swizzle_bytes == 32 ? CU_TENSOR_MAP_SWIZZLE_32B
                                  : swizzle_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                                        : CU_TENSOR_MAP_SWIZZLE_128B;
    CUresult r = fn(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                    const_cast<void *>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed with code " + std::to_string((int)r));
        return FLR_ECUDA;
    }
    return FLR_OK;
}

namespace {

int ensure_maps(flr_ctx *ctx)
{
    const int prec = ctx->p.precision;
    if (ctx->maps && ctx->maps_n == ctx->ws_n && ctx->maps_prec == prec) return FLR_OK;
    if (!ctx->maps) ctx->maps = new TcMaps();
    const bool bf16 = prec == FLR_PREC_BF16X3;
    const Dims &D = ctx->dims;
    for (int r = 0; r < 2; ++r) {
        if (bf16) {
            int st = encode(&ctx->maps->a[r][0], ctx->Dhi[r], true, D.kp64[r], ctx->ws_n, BM);
            if (st == FLR_OK) st = encode(&ctx->maps->a[r][1], ctx->Dlo[r], true, D.kp64[r], ctx->ws_n, BM);
            if (st != FLR_OK) return st;
        } else {
            // TF32: the rows rounded to nearest TF32 (the tensor core would truncate FP32 rows)
            int st = encode(&ctx->maps->a[r][0], ctx->Dtf[r], false, D.kp32[r], ctx->ws_n, BM);
            if (st != FLR_OK) return st;
            ctx->maps->a[r][1] = ctx->maps->a[r][0];
        }
    }
    for (int g = 0; g < kGroups; ++g) {
        const int r = group_region(g);
        if (bf16) {
            int st = encode(&ctx->maps->b[g][0], ctx->Whi[g], true, D.kp64[r], D.nrows_pad[r], NH);
            if (st == FLR_OK) st = encode(&ctx->maps->b[g][1], ctx->Wlo[g], true, D.kp64[r], D.nrows_pad[r], NH);
            if (st != FLR_OK) return st;
        } else {
            int st = encode(&ctx->maps->b[g][0], ctx->Wtf[g], false, D.kp32[r], D.nrows_pad[r], NH);
            if (st != FLR_OK) return st;
            ctx->maps->b[g][1] = ctx->maps->b[g][0];
        }
    }
    ctx->maps_n = ctx->ws_n;
    ctx->maps_prec = prec;
    return FLR_OK;
}

}  // namespace

int launch_qform_tc(flr_ctx *ctx, const flr_nbrlist *nl, flr_outputs *out, cudaStream_t st, bool only_full)
{
    int s = ensure_maps(ctx);
    if (s != FLR_OK) return s;
    const bool bf16 = ctx->p.precision == FLR_PREC_BF16X3;
    TcArgs a;
    for (int r = 0; r < 2; ++r) {
        a.K[r] = ctx->dims.K[r];
        a.kp32[r] = ctx->dims.kp32[r];
        a.nkb[r] = bf16 ? ctx->dims.kp64[r] / 64 : ctx->dims.kp32[r] / 32;
        a.D32[r] = ctx->D32[r];
        a.G[r] = ctx->G[r];
    }
    for (int g = 0; g < kGroups; ++g) a.nch[g] = ctx->dims.nrows_pad[group_region(g)] / NC;
    a.atom_of_row = nl->atom_of_row;
    a.n_cap = nl->n_cap;
    a.norm = ctx->norm;
    a.energy = out->energy;
    a.variance = out->variance;
    a.sigma = out->sigma;
    a.gtab = nl->gtab;
    for (int g = 0; g < kGroups; ++g) a.var_factored[g] = ctx->var_factored[g];
    a.refine = ctx->var_mode == FLR_VAR_AUTO;
    for (int g = 0; g < kGroups; ++g)   // TF32 is the low-precision option: only the cancellation test
        a.v_small[g] = bf16 ? kVarSmallBF16x3 * ctx->sigma_norm[g] : 0.f;
    a.ref_list = ctx->ref_list;
    a.ref_count = ctx->ref_count;
    a.ref_cap = ctx->ws_n;
    a.status = ctx->status;
    a.only_full = only_full ? 1 : 0;
    // ring + barriers (128 B) + the E / V exchange (2 tiles x kSubs sets x BM float4);
    // more than half of the SM's shared memory, so one CTA (holding all 512 TMEM
    // columns) runs per SM
    const size_t smem = 1024 + (size_t)kStages * kStageBytes + 128 + 2 * kSubs * BM * sizeof(float4);
    cudaError_t e;
    if (bf16) {
        e = cudaFuncSetAttribute(k_qform_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) k_qform_tc<true><<<ctx->num_sms, kThreads, smem, st>>>(*ctx->maps, a);
    } else {
        e = cudaFuncSetAttribute(k_qform_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) k_qform_tc<false><<<ctx->num_sms, kThreads, smem, st>>>(*ctx->maps, a);
    }
    if (e != cudaSuccess) return cuda_fail(e, "tensor-core GEMM attributes");
    count_launch(ctx);
    return cuda_fail(cudaGetLastError(), "tensor-core quadratic-form GEMM");
}

}  // namespace flr
