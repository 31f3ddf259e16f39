// Device code of the per-atom normalized ACE-B2 descriptor (Sec. V-B "Local
// structure descriptors" and "Acceleration of heterogeneous multi-element
// system"), shared by the descriptor kernel (desc.cu), which writes each
// atom's row of the quadratic-form operand to global memory, and the fused
// one-species kernel (fused.cu), which writes it into the shared-memory
// operand tile of the tensor cores.
//
// One warp per atom.  Lanes take the neighbour-list entries 32 at a time
// (coalesced row loads) and compact the pairs inside r_cut into a per-warp
// queue, so the basis is evaluated only for those pairs with the lanes full;
// then every lane owns 8 coefficients of A (radial index n = lane / 4, four
// harmonics, both neighbour species) and accumulates them over the queued
// pairs, so no cross-lane reduction of A is needed.  B2 = sum_m A_a A_b is
// contracted for the atom's compaction class only (both species blocks, or
// the one block its neighbours occupy), one radial-channel pair (all four l)
// per lane from float4 rows of A.
#pragma once

#include "basis.cuh"
#include "internal.cuh"

namespace flr {
namespace {

constexpr int kDescAStride = 20;   // padded channel stride of A in shared memory (conflict-free float4 rows)
constexpr int kYStride = 20;       // padded row of staged harmonics (conflict-free float4 stores)
constexpr int kRfStride = 12;      // padded row of a pair's staged radial values (two conflict-free float4 stores)

struct DescArgs {
    const float4 *pos;
    const int32_t *species;
    const int32_t *entries, *count, *group, *row;
    int max_nbr, n;
    Cells cells;               // per-structure image shifts
    float rcut;
    float two_over_rc;         // 2 / r_cut (the radial basis' x = 2 r / r_cut - 1 as one FMA)
    const int32_t *tab[2];     // compact index -> (a, b, l)
    int K[2], kp32[2], kp64[2];
    float *A;                  // [n][2N*16]
    float *norm;               // [n]
    float *D32[2];
    __nv_bfloat16 *Dhi[2], *Dlo[2];
    int bf16;                  // also write BF16 hi/lo rows
    int skip_d32_one;          // do not write the FP32 rows of the one-species region (their
                               // quadratic forms read only the BF16 rows)
    float *Dtf[2];             // also write rows rounded to nearest TF32 (TF32 precision), or nullptr
    float4 *pair_rec;          // [n][max_nbr] out: pairs inside r_cut (r_ij, j | s_j << 25)
    int32_t *pair_cnt;         // [n] out: their number
    const int32_t *order;      // order in which atoms are taken (nullptr: by index)
    const int *n_dev[2];       // when set, the atoms to take are order[0 .. *n_dev[0] + *n_dev[1]) (capped at n)
    int *sched;                // work counter, zero at launch
};

// Per warp, the staged basis of a batch of up to BATCH pairs and, once the
// pairs are done, the rows of A and the unnormalized B2 (kept here between
// the norm reduction and the scaled stores instead of in registers) share one
// region.  ONE: only one-species atoms are taken (B2 of one block).
template <int N, int BATCH = 32, bool ONE = false>
union __align__(16) DescStage {
    struct {
        float Y[BATCH][kYStride];        // harmonics of the staged pairs
        float Rf[BATCH][kRfStride];      // their radial values, one padded row per pair
    } p;
    struct {
        float A[2 * N * kDescAStride];
        float4 B[ONE ? N * (N + 1) / 2 : (2 * N) * (2 * N + 1) / 2];   // unnormalized B2 of the class's channel pairs
    } b;
};

// One warp's shared memory: the compacted pairs inside r_cut (r_ij and the
// neighbour's species; a batch is evaluated once BATCH are queued, so fewer
// than BATCH + 32 wait at a time) and the staging region.
template <int N, int BATCH = 32, bool ONE = false>
struct __align__(16) DescWarp {
    static constexpr int kBatch = BATCH;
    static constexpr bool kOne = ONE;
    float4 rec[BATCH + 32];
    DescStage<N, BATCH, ONE> st;
};

// Basis of up to BATCH staged pairs (lane p evaluates pair p), then the lanes
// that own A coefficients accumulate over them.  The basis is stored with the
// pairs of a species-0 neighbour first (each species keeps list order, so
// every accumulator sums in the same order as an unsorted pass), so the
// accumulation picks the accumulator by a warp-uniform index test instead of
// loading each pair's species.
template <int N, class W>
__device__ __forceinline__ void desc_batch(W &dw, int lane, int m, float rc, float tr, float acc0[4], float acc1[4])
{
    float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
    if (lane < m) r = dw.rec[lane];
    const bool s1 = lane < m && __float_as_int(r.w) != 0;
    const unsigned b1 = __ballot_sync(0xffffffffu, s1);
    const int n0 = m - __popc(b1);
    if (lane < m) {
        const int below1 = __popc(b1 & ((1u << lane) - 1u));
        const int slot = s1 ? n0 + below1 : lane - below1;
        const float d2 = r.x * r.x + r.y * r.y + r.z * r.z;
        const float rr = sqrtf(d2), inv = 1.f / rr;
        float Rf[N], dummy[N];
        radial<N, false>(rr, rc, tr, Rf, dummy);
        float Y[16];
        real_ylm(r.x * inv, r.y * inv, r.z * inv, Y);
        static_assert(N >= 5 && N <= 8, "two float4 rows of radial values");
        float4 *rrow = reinterpret_cast<float4 *>(&dw.st.p.Rf[slot][0]);
        rrow[0] = make_float4(Rf[0], Rf[1], Rf[2], Rf[3]);
        rrow[1] = make_float4(Rf[4], N > 5 ? Rf[N > 5 ? 5 : 0] : 0.f, N > 6 ? Rf[N > 6 ? 6 : 0] : 0.f,
                              N > 7 ? Rf[N > 7 ? 7 : 0] : 0.f);
#pragma unroll
        for (int k = 0; k < 16; k += 4)
            *reinterpret_cast<float4 *>(&dw.st.p.Y[slot][k]) = make_float4(Y[k], Y[k + 1], Y[k + 2], Y[k + 3]);
    }
    __syncwarp();
    const int my_n = lane >> 2, quad = lane & 3;
    if (my_n < N) {
        // species-0 pairs, then species-1 pairs (the staged order), each in list order
#pragma unroll 4
        for (int p = 0; p < n0; ++p) {
            const float rf = dw.st.p.Rf[p][my_n];
            const float4 y = *reinterpret_cast<const float4 *>(&dw.st.p.Y[p][4 * quad]);
            acc0[0] += rf * y.x; acc0[1] += rf * y.y; acc0[2] += rf * y.z; acc0[3] += rf * y.w;
        }
#pragma unroll 4
        for (int p = n0; p < m; ++p) {
            const float rf = dw.st.p.Rf[p][my_n];
            const float4 y = *reinterpret_cast<const float4 *>(&dw.st.p.Y[p][4 * quad]);
            acc1[0] += rf * y.x; acc1[1] += rf * y.y; acc1[2] += rf * y.z; acc1[3] += rf * y.w;
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
    const float4 *pa = reinterpret_cast<const float4 *>(sA + a * kDescAStride);
    const float4 *pb = reinterpret_cast<const float4 *>(sA + b * kDescAStride);
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

// The descriptor of atom i with group g = cur.g >= 0: scans the neighbour
// list, records the pairs inside r_cut (pair_rec, pair_cnt) for the force
// kernel, accumulates A (written to global memory, blocks of the class only),
// contracts B2 of the class's channel pairs into dw.st.b.B (unnormalized;
// with KEEP0, channel pair `lane` goes to *b0 instead, so the first 32 stay
// in registers), writes ||B|| to norm[i] and returns it.  The caller scales
// B by 1 / ||B|| and writes the normalized row where its quadratic-form
// kernel reads it.
template <int N, class W, bool KEEP0 = false>
__device__ __forceinline__ float desc_atom(const DescArgs &a, W &dw, int lane, const DescPre &cur, int i,
                                          float4 *b0 = nullptr)
{
    constexpr int C = 2 * N;
    constexpr int BATCH = W::kBatch;
    constexpr int NPF = C * (C + 1) / 2;          // channel pairs of the full descriptor
    constexpr int NPS = N * (N + 1) / 2;          // channel pairs of a one-species block
    constexpr int MAXP = ((W::kOne ? NPS : NPF) + 31) / 32;
    const float rc = a.rcut, rc2 = rc * rc;
    const int g = cur.g;
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
            dw.rec[nv + at] = make_float4(r.x, r.y, r.z, __int_as_float(sj));
            // the force kernel reuses the pair vector instead of gathering and filtering again
            prec[np + at] = make_float4(r.x, r.y, r.z, __int_as_float(j | ((sj & 1) << 25)));
        }
        nv += __popc(m);
        np += __popc(m);
        __syncwarp();
        while (nv >= BATCH) {
            desc_batch<N>(dw, lane, BATCH, rc, a.two_over_rc, acc0, acc1);
            const float4 rest = lane < nv - BATCH ? dw.rec[BATCH + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
            __syncwarp();
            if (lane < nv - BATCH) dw.rec[lane] = rest;
            nv -= BATCH;
            __syncwarp();
        }
    }
    if (nv > 0) desc_batch<N>(dw, lane, nv, rc, a.two_over_rc, acc0, acc1);
    if (lane == 0) a.pair_cnt[i] = np;

    // A to shared memory (padded rows) and to global memory (blocks in use only)
    float *sA = dw.st.b.A;   // the staging area is free once the pairs are done
    const int my_n = lane >> 2, quad = lane & 3;
    if (my_n < N) {
        // the B2 pass reads only the rows of the class's blocks
        if (cls != 2)
            *reinterpret_cast<float4 *>(sA + my_n * kDescAStride + 4 * quad) = make_float4(acc0[0], acc0[1], acc0[2], acc0[3]);
        if (cls != 1)
            *reinterpret_cast<float4 *>(sA + (N + my_n) * kDescAStride + 4 * quad) =
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
    const int npairs = (W::kOne || cls != 0) ? NPS : NPF;
    const int choff = cls == 0 ? 0 : (cls - 1) * N;
    const int32_t *tab = a.tab[reg];
    float4 *sB = dw.st.b.B;
    float ss = 0.f;
#pragma unroll
    for (int k = 0; k < MAXP; ++k) {
        const int t = lane + 32 * k;
        if (t < npairs) {
            const int e = __ldg(tab + 4 * t);
            const float4 bb = b2_pair(sA, choff + (e & 255), choff + ((e >> 8) & 255));
            if (KEEP0 && k == 0)
                *b0 = bb;   // the caller keeps channel pair `lane` in registers
            else
                sB[t] = bb;
            ss += bb.x * bb.x + bb.y * bb.y + bb.z * bb.z + bb.w * bb.w;
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    const float nrm = sqrtf(ss);
    if (lane == 0) a.norm[i] = nrm;
    __syncwarp();
    return nrm;
}

// The atoms a descriptor launch takes: a.n, or the count(s) a.n_dev point to.
__device__ __forceinline__ int desc_count(const DescArgs &a)
{
    if (!a.n_dev[0]) return a.n;
    const int m = *a.n_dev[0] + (a.n_dev[1] ? *a.n_dev[1] : 0);
    return m < a.n ? m : a.n;
}

}  // namespace
}  // namespace flr
