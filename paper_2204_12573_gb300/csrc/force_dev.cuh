// Device code of the force evaluation (Sec. V-B, "Acceleration of force
// predictions"): the per-warp state and the per-atom and per-pair steps of
// the force kernel (force.cu).
//
// Given g = dE/dB of an atom, the gradient is pushed back through the B2
// contraction once per atom,
//   w_{a,lm} = dE/dA_{a,lm} = sum_b G_{ab,l} A_{b,lm},  G_aa = 2 g_aa,
// and each neighbour pair then needs only
//   f_ij = dE_i/dr_ij = sum_{n,lm} w_{(s_j,n),lm} grad phi_{n,lm}(r_ij),
// which costs O(N L^2) per pair instead of O(d).  F_i += f_ij, F_j -= f_ij.
//
// A warp walks atoms one at a time.  For each it copies g and the A rows of
// the atom's class into shared memory (cp.async, one atom ahead), unpacks g
// into a dense symmetric channel matrix G~, forms w = G~ A into one of four
// w slots, then appends the atom's pairs inside r_cut -- recorded by the
// descriptor kernel as (r_ij, j, s_j) -- to a per-warp FIFO queue; whenever
// 32 pairs are queued they are evaluated with one pair per lane, whatever
// atoms they belong to, so the per-pair path always runs with full lanes.
// Forces are accumulated as 64-bit fixed point (2^-32 eV/A) through global
// atomics; integer sums do not depend on order or on how an atom's pairs were
// split over batches, so forces are bitwise reproducible.
#pragma once

#include "basis.cuh"
#include "internal.cuh"

namespace flr {
namespace {

constexpr int kAStride = 20;                  // float4-aligned, conflict-free A rows
constexpr int kSlots = 4;                     // atoms whose w may be referenced by queued pairs
constexpr float kFixScale = 4294967296.0f;    // 2^32
constexpr double kFixInv = 1.0 / 4294967296.0;

struct ForceArgs {
    const float4 *pos;
    const int32_t *species;
    const int32_t *entries, *count, *group, *row;
    int max_nbr, n;
    float rcut;
    float two_over_rc;         // 2 / r_cut (x = 2 r / r_cut - 1 as one FMA per pair)
    int K[2];
    const float *G[2];         // g = dE/dB rows from the quadratic-form epilogue
    const float *A, *norm;
    float *energy, *variance, *sigma;
    unsigned long long *Facc;
    double *vir_part;          // [gridDim.x][9]
    float *vir_atom;           // [n][9] per-atom virial, or nullptr (batches of structures need it)
    const float *weight;       // [n] per-atom weights u_i on E_i (backward pass), or nullptr
    const float4 *pair_rec;    // [n][max_nbr] pairs inside r_cut from the descriptor kernel
    const int32_t *pair_cnt;   // [n]
    const int32_t *tab[2];     // compact index -> channel pair (a | b << 8), per region
    int *sched;                // work counter, zero at launch
    int *status;
    const int32_t *order;      // atoms taken as order[0 .. m) (nullptr: 0 .. n-1 by index), with
    const int *n_dev[4];       // m = the sum of the counts these point to (capped at n)
    int vir_base;              // first row of this launch's block partials in vir_part
};

// Dense G~ layout for a class of CG channels: lane half h owns channels
// [h * gd_half(CG), ...), rows b are gd_row(CG) floats apart (a multiple of
// 8, so every float4 load is aligned), planes l are gd_plane(CG) apart.
__host__ __device__ constexpr int gd_half(int CG) { return ((CG + 1) / 2 + 3) / 4 * 4; }
__host__ __device__ constexpr int gd_row(int CG) { return 2 * gd_half(CG); }
__host__ __device__ constexpr int gd_plane(int CG) { return CG * gd_row(CG) + 8; }

// Shared-memory state of one warp (one contiguous block per warp), for atoms
// of any compaction class.
template <int N>
struct __align__(16) ForceWarp {
    static constexpr bool kOne = false;               // holds both species blocks
    static constexpr int CGM = 2 * N;                 // widest class
    static constexpr int WSLOT = 2 * 16 * 8 + 4;      // [species][lm][n (8, padded)] + pad
    float4 q[64];                      // queued pairs: r_ij, packed (j | s_j << 25 | slot << 26)
    float Gd[4 * gd_plane(CGM)];       // G~[l][b][a] of the atom's class
    float A[2 * N * kAStride];         // A rows of the atom's class
    float gr[CGM * (CGM + 1) / 2 * 4]; // raw g row of the next atom (cp.async)
    float W[kSlots * WSLOT];
    long long V[kSlots][9];            // virial of each slot's atom (when requested), fixed point
    int atom[kSlots];
    int qseq[64];                      // atom sequence number of each queued pair
};

// The same state for atoms of the one-species classes only: one block of N
// channels in G~, A and w (all of such an atom's pairs have a neighbour of
// that species), so a warp needs less than half the shared memory.
template <int N>
struct __align__(16) ForceWarp1 {
    static constexpr bool kOne = true;
    static constexpr int CGM = N;
    static constexpr int WSLOT = 16 * 8 + 4;          // [lm][n (8, padded)] + pad
    float4 q[64];
    float Gd[4 * gd_plane(N)];
    float A[N * kAStride];
    float gr[N * (N + 1) / 2 * 4];
    float W[kSlots * WSLOT];
    long long V[kSlots][9];
    int atom[kSlots];
    int qseq[64];
};

// Where each compact channel pair (a, b) of g lands in the dense G~ of its
// class: offsets of (b, a) and (a, b), equal on the diagonal; the
// two-species layout, then the one-species one.
template <int N>
__host__ __device__ constexpr int goff_count() { return (2 * N) * (2 * N + 1) / 2 + N * (N + 1) / 2; }

template <int N>
__device__ __forceinline__ void init_goff(const ForceArgs &a, int2 *goff, int tid, int nthreads)
{
    constexpr int C = 2 * N, NPF = C * (C + 1) / 2, NPS = N * (N + 1) / 2;
    for (int t = tid; t < NPF + NPS; t += nthreads) {
        const bool full = t < NPF;
        const int e = __ldg(full ? a.tab[0] + 4 * t : a.tab[1] + 4 * (t - NPF));
        const int ca = e & 255, cb = (e >> 8) & 255;
        const int RS = full ? gd_row(C) : gd_row(N);
        goff[t] = make_int2(cb * RS + ca, ca * RS + cb);
    }
}

// |v| must stay below 2^15 eV/A (else the status word reports a non-finite
// or overflowing force), which keeps the warp sums below in 32-bit range.
__device__ __forceinline__ long long to_fix(float v, int *status)
{
    const float s = v * kFixScale;
    if (!(fabsf(s) < 140737488355328.0f)) {   // 2^47; also catches NaN
        atomicOr(status, kErrNonFinite);
        return 0;
    }
    return __float2ll_rn(s);
}

// Evaluate m <= 32 queued pairs, one per lane.
template <int N, class FW>
__device__ __forceinline__ void force_batch(FW &fw, int lane, int m, float rc, float tr,
                                            unsigned long long *Facc, int *status, float vir[9], bool want_vatom)
{
    int my_slot = -1;
    float pr[3] = {0.f, 0.f, 0.f}, pf[3] = {0.f, 0.f, 0.f};   // this lane's r_ij and f_ij (per-atom virial)
    if (lane < m) {
        const float4 rec = fw.q[lane];
        const int packed = __float_as_int(rec.w);
        const int j = packed & 0x1FFFFFF;
        const int sj = (packed >> 25) & 1;
        const int slot = (packed >> 26) & 3;
        const float d2 = rec.x * rec.x + rec.y * rec.y + rec.z * rec.z;
        const float rr = sqrtf(d2), inv = 1.f / rr;
        const float ux = rec.x * inv, uy = rec.y * inv, uz = rec.z * inv;
        // R_n = T_n(x) f_c with x = 2r/r_cut - 1, f_c = (r_cut - r)^2 (the
        // descriptor's radial basis).  The sums over n run on T_n and T_n'
        // alone, and f_c, f_c' and dx/dr = 2/r_cut scale the per-pair totals:
        //   c_lm = f_c s_lm,  c'_lm = (2/r_cut) f_c s'_lm + f_c' s_lm,
        //   s_lm = sum_n w_{n,lm} T_n(x),  s'_lm = sum_n w_{n,lm} T_n'(x),
        // so T_0 = 1 and T_1' = 1 cost no multiply and T_0' = 0 no term.
        const float x = rr * tr - 1.f;
        const float tc = rc - rr;
        const float fc = tc * tc, dfc = -2.f * tc, k1 = tr * fc;
        float T[N], dT[N];
        cheb_tail<N>(x, T, dT);
        const float *wp = fw.W + slot * FW::WSLOT + (FW::kOne ? 0 : sj * 128);
        const float xx = ux * ux, yy = uy * uy, zz = uz * uz;
        // f = u (sum_lm c'_lm Y_lm - (1/r) sum_lm l c_lm Y_lm) + (1/r) sum_lm c_lm grad P_lm(u)
        float sp_y = 0.f, s_y0 = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
        float ls[4] = {0.f, 0.f, 0.f, 0.f};   // sum of s Y per l
#pragma unroll
        for (int lm = 0; lm < 16; ++lm) {
            const float4 w0 = *reinterpret_cast<const float4 *>(wp + lm * 8);
            const float4 w1 = *reinterpret_cast<const float4 *>(wp + lm * 8 + 4);
            const float wv[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
            float s = wv[0] + wv[1] * x, sp = wv[1];
#pragma unroll
            for (int n = 2; n < N; ++n) {
                s += wv[n] * T[n];
                sp += wv[n] * dT[n];
            }
            float Y, dx, dy, dz;
            ylm_one(lm, ux, uy, uz, xx, yy, zz, Y, dx, dy, dz);
            sp_y += sp * Y;
            if (l_of(lm) > 0) ls[l_of(lm)] += s * Y;
            else s_y0 += s * Y;
            // only the components of grad P_lm that are not identically zero
            if (grad_nz(lm, 0)) gx += s * dx;
            if (grad_nz(lm, 1)) gy += s * dy;
            if (grad_nz(lm, 2)) gz += s * dz;
        }
        const float radial_part = k1 * sp_y + dfc * (s_y0 + ls[1] + ls[2] + ls[3]);
        const float lsum = fc * (ls[1] + 2.f * ls[2] + 3.f * ls[3]);
        const float coef = radial_part - lsum * inv;
        const float gsc = fc * inv;
        const float fx = coef * ux + gx * gsc;
        const float fy = coef * uy + gy * gsc;
        const float fz = coef * uz + gz * gsc;
        const long long ix = to_fix(fx, status), iy = to_fix(fy, status), iz = to_fix(fz, status);
        unsigned long long *dj = Facc + 3 * (size_t)j;
        atomicAdd(dj + 0, (unsigned long long)(-ix));
        atomicAdd(dj + 1, (unsigned long long)(-iy));
        atomicAdd(dj + 2, (unsigned long long)(-iz));
        unsigned long long *di = Facc + 3 * (size_t)fw.atom[slot];
        atomicAdd(di + 0, (unsigned long long)ix);
        atomicAdd(di + 1, (unsigned long long)iy);
        atomicAdd(di + 2, (unsigned long long)iz);
        // W_ab -= (r_ij)_a (f_ij)_b, one FMA per entry
        pr[0] = rec.x; pr[1] = rec.y; pr[2] = rec.z;
        pf[0] = fx; pf[1] = fy; pf[2] = fz;
#pragma unroll
        for (int k = 0; k < 9; ++k) vir[k] = fmaf(-pr[k / 3], pf[k % 3], vir[k]);
        my_slot = slot;
    }
    // The per-atom virial (when requested): the queue is filled atom by atom,
    // so each slot's pairs occupy consecutive lanes.  Every lane finds the
    // mask of its segment and the segment is summed with warp reductions on
    // 32-bit halves of the fixed-point values (|v| < 2^47, so the high parts
    // of 32 lanes cannot overflow); integer sums do not depend on how an
    // atom's pairs were split over batches.
    if (want_vatom) {
        const int prev_slot = __shfl_up_sync(0xffffffffu, my_slot, 1);
        const unsigned heads = __ballot_sync(0xffffffffu, lane < m && (lane == 0 || my_slot != prev_slot));
        const unsigned valid = m >= 32 ? 0xffffffffu : ((1u << m) - 1u);
        unsigned seg;
        if (lane < m) {
            const unsigned below = heads & (0xffffffffu >> (31 - lane));          // heads at or below this lane
            const unsigned start = 1u << (31 - __clz(below));
            const unsigned above = heads & ~(0xffffffffu >> (31 - lane));         // heads above this lane
            const unsigned stop = above ? (above & (0u - above)) : 0u;            // lowest of them, or none
            seg = (stop ? (stop - start) : (valid & ~(start - 1u)));
        } else {
            seg = ~valid;   // idle lanes form one group of their own
        }
        const bool leader = (seg & (0u - seg)) == (1u << lane);                    // lowest lane of the segment
#pragma unroll
        for (int c = 0; c < 9; ++c) {
            const long long x = lane < m ? to_fix(-pr[c / 3] * pf[c % 3], status) : 0;
            const unsigned lo = __reduce_add_sync(seg, (unsigned)(x & 0x3FFFFF));
            const int hi = __reduce_add_sync(seg, (int)(x >> 22));
            if (leader && lane < m) fw.V[my_slot][c] += (long long)hi * 4194304ll + (long long)lo;
        }
    }
    __syncwarp();
}

// Evaluate every queued pair (all) or every full batch, and compact the queue.
template <int N, class FW>
__device__ __forceinline__ void drain(FW &fw, int lane, int &nq, bool all, float rc, float tr,
                                      unsigned long long *Facc, int *status, float vir[9], bool want_vatom)
{
    while (nq >= 32 || (all && nq > 0)) {
        const int m = nq < 32 ? nq : 32;
        force_batch<N, FW>(fw, lane, m, rc, tr, Facc, status, vir, want_vatom);
        const int rest = nq - m;
        float4 r4 = make_float4(0.f, 0.f, 0.f, 0.f);
        int sq = 0;
        if (lane < rest) {
            r4 = fw.q[m + lane];
            sq = fw.qseq[m + lane];
        }
        __syncwarp();
        if (lane < rest) {
            fw.q[lane] = r4;
            fw.qseq[lane] = sq;
        }
        __syncwarp();
        nq = rest;
    }
}

// Release a slot: write its atom's virial (when requested) and clear it.
template <class FW>
__device__ __forceinline__ void flush_slot(FW &fw, int lane, int slot, float *vir_atom)
{
    const int i = fw.atom[slot];
    if (lane < 9) {
        if (vir_atom && i >= 0) vir_atom[9 * (size_t)i + lane] = (float)((double)fw.V[slot][lane] * kFixInv);
        fw.V[slot][lane] = 0;
    }
    __syncwarp();
    if (lane == 0) fw.atom[slot] = -1;
    __syncwarp();
}

// Warp start: no slot in use, no virial.
template <class FW>
__device__ __forceinline__ void init_warp(FW &fw, int lane)
{
    if (lane < kSlots) fw.atom[lane] = -1;
    for (int k = lane; k < 9 * kSlots; k += 32) fw.V[k / 9][k % 9] = 0;
}

// w_{a,lm} = sum_b G~_{ab,l} A_{b,lm} over the CG channels of a class.  Lane
// (lm, half) owns harmonic lm of half of the channels a; G~ is dense in
// shared memory as [l][b][a] (row b contiguous in a), so each b costs one
// A value and H/4 float4 loads of G~ for H FMAs per lane.
template <int CG, int N, bool ONE = false>
__device__ __forceinline__ void w_dense(const float *sGd, const float *sA, float *ws, int choff, int half, int lm)
{
    constexpr int H = gd_half(CG);
    constexpr int RS = gd_row(CG);
    constexpr int LS = gd_plane(CG);
    const int l = l_of(lm);
    const int a0 = half * H;
    const float *gp = sGd + l * LS + a0;
    float acc[H];
#pragma unroll
    for (int k = 0; k < H; ++k) acc[k] = 0.f;
#pragma unroll
    for (int b = 0; b < CG; ++b) {
        const float av = sA[(ONE ? b : choff + b) * kAStride + lm];
#pragma unroll
        for (int k = 0; k < H; k += 4) {
            const float4 gv = *reinterpret_cast<const float4 *>(gp + b * RS + k);
            acc[k] += gv.x * av;
            acc[k + 1] += gv.y * av;
            acc[k + 2] += gv.z * av;
            acc[k + 3] += gv.w * av;
        }
    }
#pragma unroll
    for (int k = 0; k < H; ++k) {
        if (a0 + k < CG) {                         // the last half may be padded
            if (ONE) {
                ws[lm * 8 + a0 + k] = acc[k];     // the one block
            } else {
                const int ch = choff + a0 + k;    // channel = species * N + n
                ws[(ch / N) * 128 + lm * 8 + (ch % N)] = acc[k];
            }
        }
    }
}

// Per-atom values loaded one iteration ahead, so their latency overlaps the
// previous atom's work.
struct AtomPre {
    int g, row, np;
    float nrm;
    float4 r0;      // pair record `lane` of the atom
};

__device__ __forceinline__ AtomPre preload(const ForceArgs &a, int i, int i_end, int lane)
{
    AtomPre p;
    p.g = -2;
    p.row = 0;
    p.np = 0;
    p.nrm = 0.f;
    p.r0 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i < i_end) {
        // read-only loads (ld.global.nc): free to move across the force
        // atomics; all four are issued at once
        p.g = __ldg(a.group + i);
        p.row = __ldg(a.row + i);
        p.nrm = __ldg(a.norm + i);
        p.np = __ldg(a.pair_cnt + i);
    }
    return p;
}

// The atom's first 32 pair records, on the lanes below its pair count only
// (the row holds max_nbr slots, of which about 17 are in use).  Issued once
// the count has arrived -- after the previous atom's work -- so the load
// waits for nothing and reads no unused slot.
__device__ __forceinline__ void preload_pairs(const ForceArgs &a, AtomPre &p, int i, int i_end, int lane)
{
    if (i < i_end && lane < p.np) p.r0 = __ldg(a.pair_rec + (size_t)i * a.max_nbr + lane);
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }
// 16 bytes global -> shared, through L2 only (.cg)
__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}

// Start copying atom i's g row (raw, compact order) and the A rows of its
// class's channels into the warp's shared buffers (cp.async; lane t % 32
// copies chunk t).  The buffers must no longer be in use.
template <int N, bool ONE = false>
__device__ __forceinline__ void rows_async(const ForceArgs &a, const AtomPre &p, int i, int i_end, float *gr, float *sA,
                                           int lane)
{
    constexpr int C = 2 * N;
    if (i >= i_end || p.g < 0 || !(p.nrm > 0.f)) return;
    const int cls = group_cls(p.g), reg = group_region(p.g);
    const int K = a.K[reg];
    const int Cg = cls == 0 ? C : N;
    const int choff = cls == 0 ? 0 : (cls - 1) * N;
    const float *g = a.G[reg] + (size_t)p.row * K;
    for (int t = lane; 4 * t < K; t += 32) cp_async16(gr + 4 * t, g + 4 * t);
    const float *Ag = a.A + (size_t)i * (C * 16);
    for (int k = lane; k < Cg * 4; k += 32) {
        const int ch = choff + (k >> 2);
        cp_async16(sA + (ONE ? (k >> 2) : ch) * kAStride + 4 * (k & 3), Ag + ch * 16 + 4 * (k & 3));
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// The work of one atom that has an environment (g >= 0, ||B|| > 0): claim a
// w slot (evaluating queued pairs that still refer to it), build G~ from the
// atom's g row, form w = G~ A, start copying the next atom's rows (nxt, i2;
// nothing when i2 >= i_end), then queue the atom's pairs and evaluate every
// full batch.
template <int N, class FW>
__device__ __forceinline__ void force_atom(const ForceArgs &a, FW &fw, const int2 *goff_all, int lane,
                                           const AtomPre &cur, int i, const AtomPre &nxt, int i2, int i_end,
                                           int &nq, int &seq, float vir[9], bool want_vatom)
{
    constexpr int C = 2 * N;
    const float rc = a.rcut;
    const int g = cur.g;
    const int cls = group_cls(g), reg = group_region(g);
    const int K = a.K[reg];
    const int choff = cls == 0 ? 0 : (cls - 1) * N;

    // w slot for this atom: if a queued pair still refers to the slot, evaluate the queue first
    const int slot = seq & (kSlots - 1);
    if (nq > 0 && fw.qseq[0] <= seq - kSlots)
        drain<N, FW>(fw, lane, nq, true, rc, a.two_over_rc, a.Facc, a.status, vir, want_vatom);
    if (want_vatom) flush_slot(fw, lane, slot, a.vir_atom);   // otherwise the slot holds nothing to write
    if (lane == 0) fw.atom[slot] = i;

    // this atom's g row and A rows were copied into shared memory while the
    // previous atom was processed
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncwarp();
    // g = dE/dB of this atom (compact order of its class, written by the
    // quadratic-form epilogue; scaled by u_i in the backward pass) ->
    // dense symmetric G~[l][b][a] with the diagonal doubled
    {
        const float4 *g4 = reinterpret_cast<const float4 *>(fw.gr);
        const int2 *goff = goff_all + (reg == 0 ? 0 : C * (C + 1) / 2);
        const float u = a.weight ? __ldg(a.weight + i) : 1.f;
        const int LS = cls == 0 ? gd_plane(C) : gd_plane(N);
        for (int t = lane; 4 * t < K; t += 32) {
            const int2 of = goff[t];
            const int o1 = of.x, o2 = of.y;
            float4 v = g4[t];
            const float sc = o1 == o2 ? 2.f * u : u;   // the diagonal of G~ is doubled
            v.x *= sc;
            v.y *= sc;
            v.z *= sc;
            v.w *= sc;
            fw.Gd[o1] = v.x;
            fw.Gd[o2] = v.x;
            fw.Gd[LS + o1] = v.y;
            fw.Gd[LS + o2] = v.y;
            fw.Gd[2 * LS + o1] = v.z;
            fw.Gd[2 * LS + o2] = v.z;
            fw.Gd[3 * LS + o1] = v.w;
            fw.Gd[3 * LS + o2] = v.w;
        }
    }
    float *ws = fw.W + slot * FW::WSLOT;
    // w_dense writes every channel of the atom's class; pairs only read
    // the species blocks of that class, so the slot needs no clearing
    __syncwarp();
    {
        const int lm = lane & 15, half = lane >> 4;
        if (FW::kOne)
            w_dense<N, N, true>(fw.Gd, fw.A, ws, choff, half, lm);
        else if (cls == 0)
            w_dense<C, N>(fw.Gd, fw.A, ws, 0, half, lm);
        else
            w_dense<N, N>(fw.Gd, fw.A, ws, choff, half, lm);
    }
    __syncwarp();
    // the g and A buffers are free: start copying the next atom's rows
    rows_async<N, FW::kOne>(a, nxt, i2, i_end, fw.gr, fw.A, lane);

    // queue the atom's pairs inside r_cut (recorded by the descriptor kernel)
    const int np = cur.np;
    const float4 *pr = a.pair_rec + (size_t)i * a.max_nbr;
    for (int base = 0; base < np; base += 32) {
        const int take = min(32, np - base);
        if (lane < take) {
            float4 r = base == 0 ? cur.r0 : __ldg(pr + base + lane);
            r.w = __int_as_float(__float_as_int(r.w) | (slot << 26));
            fw.q[nq + lane] = r;
            fw.qseq[nq + lane] = seq;
        }
        nq += take;
        __syncwarp();
        drain<N, FW>(fw, lane, nq, false, rc, a.two_over_rc, a.Facc, a.status, vir, want_vatom);
    }
    ++seq;
}

}  // namespace
}  // namespace flr
