// Energy, variance, uncertainty and forces from the quadratic-form products.
//
// Given P = [beta d, Sigma d] for an atom's descriptor row (Eq. 1, Eq. 2):
//   E = d . (beta d),  V = d . (Sigma d),  sigma = sqrt(V)
//   g = dE/dB = (2/||B||) (beta d - E d)                (beta symmetric)
// and then the reordered summation of Sec. V-B ("Acceleration of force
// predictions"): instead of forming dd/dr (d x 3 per neighbour), the
// gradient is pushed back through the B2 contraction once per atom,
//   w_{a,lm} = dE/dA_{a,lm} = sum_b G_{ab,l} A_{b,lm},  G_aa = 2 g_aa,
// and each neighbour pair then needs only
//   f_ij = dE_i/dr_ij = sum_{n,lm} w_{(s_j,n),lm} grad phi_{n,lm}(r_ij),
// which costs O(N L^2) per pair instead of O(d).  F_i += f_ij, F_j -= f_ij.
//
// Work layout: persistent warps walk the atoms.  For each atom a warp reads
// g (E, V and sigma were already written by the quadratic-form epilogue),
// unpacks it into a dense symmetric channel matrix G~ in shared memory,
// forms w = G~ A (w goes to one of four shared-memory slots), then appends
// the atom's pairs inside r_cut -- recorded by the descriptor kernel as
// (r_ij, j, s_j), so nothing is gathered or filtered again -- to a per-warp
// FIFO queue; whenever 32 pairs are queued they are evaluated with one pair
// per lane, whatever atoms they belong to, so the expensive per-pair path
// always runs with full lanes.  Forces are accumulated as 64-bit fixed point
// (2^-32 eV/A) through global atomics, +f_ij on F_i and -f_ij on F_j; integer
// sums do not depend on order or on how an atom's pairs were split over
// batches, so forces are bitwise reproducible and independent of what else is
// evaluated alongside.
#include "basis.cuh"
#include "internal.cuh"

namespace flr {
namespace {

constexpr int kWarpsForce = 4;                // warps per CTA (shared memory: 36 KB)
constexpr int kAStride = 20;                  // float4-aligned, conflict-free A rows
constexpr int kSlots = 4;                     // atoms whose w may be referenced by queued pairs
constexpr int kWSlot = 2 * 16 * 8 + 4;        // floats per w slot: [species][lm][n (8, padded)] + pad
constexpr float kFixScale = 4294967296.0f;    // 2^32
constexpr double kFixInv = 1.0 / 4294967296.0;

struct ForceArgs {
    const float4 *pos;
    const int32_t *species;
    const int32_t *entries, *count, *group, *row;
    int max_nbr, n;
    float rcut;
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
};

// Dense G~ layout for a class of CG channels: lane half h owns channels
// [h * gd_half(CG), ...), rows b are gd_row(CG) floats apart (a multiple of
// 8, so every float4 load is aligned), planes l are gd_plane(CG) apart.
__host__ __device__ constexpr int gd_half(int CG) { return ((CG + 1) / 2 + 3) / 4 * 4; }
__host__ __device__ constexpr int gd_row(int CG) { return 2 * gd_half(CG); }
__host__ __device__ constexpr int gd_plane(int CG) { return CG * gd_row(CG) + 8; }

template <int N>
struct ForceSmem {
    float Gd[kWarpsForce][4 * gd_plane(2 * N)];          // G~[l][b][a] of the widest class
    float A[kWarpsForce][2 * N * kAStride];
    float gr[kWarpsForce][(2 * N) * (2 * N + 1) / 2 * 4];   // raw g row of the next atom (cp.async)
    float W[kWarpsForce][kSlots * kWSlot];
    float4 q[kWarpsForce][64];                  // queued pairs: r_ij, packed (j | s_j << 25 | slot << 26)
    long long V[kWarpsForce][kSlots][9];         // virial of each slot's atom (when requested), fixed point
    int atom[kWarpsForce][kSlots];
    int qseq[kWarpsForce][64];                  // atom sequence number of each queued pair
    float vir[kWarpsForce][9];
    int2 goff[(2 * N) * (2 * N + 1) / 2 + N * (N + 1) / 2];   // G~ offsets (b a, a b) of each compact pair:
                                                             // two-species layout, then one-species
};

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
template <int N>
__device__ __forceinline__ void force_batch(ForceSmem<N> &sm, int w, int lane, int m, float rc,
                                            unsigned long long *Facc, int *status, float vir[9], bool want_vatom)
{
    int my_slot = -1;
    float dv[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (lane < m) {
        const float4 rec = sm.q[w][lane];
        const int packed = __float_as_int(rec.w);
        const int j = packed & 0x1FFFFFF;
        const int sj = (packed >> 25) & 1;
        const int slot = (packed >> 26) & 3;
        const float d2 = rec.x * rec.x + rec.y * rec.y + rec.z * rec.z;
        const float rr = sqrtf(d2), inv = 1.f / rr;
        const float ux = rec.x * inv, uy = rec.y * inv, uz = rec.z * inv;
        float Rf[N], dRf[N];
        radial<N, true>(rr, rc, Rf, dRf);
        const float *wp = sm.W[w] + slot * kWSlot + sj * 128;
        const float xx = ux * ux, yy = uy * uy, zz = uz * uz;
        // f = u (sum_lm c'_lm Y_lm - (1/r) sum_lm l c_lm Y_lm) + (1/r) sum_lm c_lm grad P_lm(u),
        // c_lm = sum_n w_{n,lm} R_n f_c,  c'_lm = sum_n w_{n,lm} (R_n f_c)'
        float radial_part = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
        float ls[4] = {0.f, 0.f, 0.f, 0.f};   // sum of c Y per l
#pragma unroll
        for (int lm = 0; lm < 16; ++lm) {
            const float4 w0 = *reinterpret_cast<const float4 *>(wp + lm * 8);
            const float4 w1 = *reinterpret_cast<const float4 *>(wp + lm * 8 + 4);
            const float wv[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
            float c = 0.f, cp = 0.f;
#pragma unroll
            for (int n = 0; n < N; ++n) {
                c += wv[n] * Rf[n];
                cp += wv[n] * dRf[n];
            }
            float Y, dx, dy, dz;
            ylm_one(lm, ux, uy, uz, xx, yy, zz, Y, dx, dy, dz);
            radial_part += cp * Y;
            if (l_of(lm) > 0) ls[l_of(lm)] += c * Y;
            // only the components of grad P_lm that are not identically zero
            if (grad_nz(lm, 0)) gx += c * dx;
            if (grad_nz(lm, 1)) gy += c * dy;
            if (grad_nz(lm, 2)) gz += c * dz;
        }
        const float lsum = ls[1] + 2.f * ls[2] + 3.f * ls[3];
        const float coef = radial_part - lsum * inv;
        const float fx = coef * ux + gx * inv;
        const float fy = coef * uy + gy * inv;
        const float fz = coef * uz + gz * inv;
        const long long ix = to_fix(fx, status), iy = to_fix(fy, status), iz = to_fix(fz, status);
        unsigned long long *dj = Facc + 3 * (size_t)j;
        atomicAdd(dj + 0, (unsigned long long)(-ix));
        atomicAdd(dj + 1, (unsigned long long)(-iy));
        atomicAdd(dj + 2, (unsigned long long)(-iz));
        unsigned long long *di = Facc + 3 * (size_t)sm.atom[w][slot];
        atomicAdd(di + 0, (unsigned long long)ix);
        atomicAdd(di + 1, (unsigned long long)iy);
        atomicAdd(di + 2, (unsigned long long)iz);
        dv[0] = -rec.x * fx; dv[1] = -rec.x * fy; dv[2] = -rec.x * fz;
        dv[3] = -rec.y * fx; dv[4] = -rec.y * fy; dv[5] = -rec.y * fz;
        dv[6] = -rec.z * fx; dv[7] = -rec.z * fy; dv[8] = -rec.z * fz;
#pragma unroll
        for (int k = 0; k < 9; ++k) vir[k] += dv[k];
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
            const long long x = lane < m ? to_fix(dv[c], status) : 0;
            const unsigned lo = __reduce_add_sync(seg, (unsigned)(x & 0x3FFFFF));
            const int hi = __reduce_add_sync(seg, (int)(x >> 22));
            if (leader && lane < m) sm.V[w][my_slot][c] += (long long)hi * 4194304ll + (long long)lo;
        }
    }
    __syncwarp();
}

// Evaluate every queued pair and compact the queue.
template <int N>
__device__ __forceinline__ void drain(ForceSmem<N> &sm, int w, int lane, int &nq, bool all, float rc,
                                      unsigned long long *Facc, int *status, float vir[9], bool want_vatom)
{
    while (nq >= 32 || (all && nq > 0)) {
        const int m = nq < 32 ? nq : 32;
        force_batch<N>(sm, w, lane, m, rc, Facc, status, vir, want_vatom);
        const int rest = nq - m;
        float4 r4 = make_float4(0.f, 0.f, 0.f, 0.f);
        int sq = 0;
        if (lane < rest) {
            r4 = sm.q[w][m + lane];
            sq = sm.qseq[w][m + lane];
        }
        __syncwarp();
        if (lane < rest) {
            sm.q[w][lane] = r4;
            sm.qseq[w][lane] = sq;
        }
        __syncwarp();
        nq = rest;
    }
}

// Release a slot: write its atom's virial (when requested) and clear it.
template <int N>
__device__ __forceinline__ void flush_slot(ForceSmem<N> &sm, int w, int lane, int slot, float *vir_atom)
{
    const int i = sm.atom[w][slot];
    if (lane < 9) {
        if (vir_atom && i >= 0) vir_atom[9 * (size_t)i + lane] = (float)((double)sm.V[w][slot][lane] * kFixInv);
        sm.V[w][slot][lane] = 0;
    }
    __syncwarp();
    if (lane == 0) sm.atom[w][slot] = -1;
    __syncwarp();
}

// w_{a,lm} = sum_b G~_{ab,l} A_{b,lm} over the CG channels of a class.  Lane
// (lm, half) owns harmonic lm of half of the channels a; G~ is dense in
// shared memory as [l][b][a] (row b contiguous in a), so each b costs one
// A value and H/4 float4 loads of G~ for H FMAs per lane.
template <int CG, int N>
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
        const float av = sA[(choff + b) * kAStride + lm];
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
            const int ch = choff + a0 + k;        // channel = species * N + n
            ws[(ch / N) * 128 + lm * 8 + (ch % N)] = acc[k];
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
        // read-only loads (ld.global.nc): free to move across the force atomics.
        // All five are issued at once, none waits for another: the pair count
        // and record row exist for every atom (lane < 32 <= max_nbr) and are
        // used only when the atom has pairs, and only below the count.
        p.g = __ldg(a.group + i);
        p.row = __ldg(a.row + i);
        p.nrm = __ldg(a.norm + i);
        p.np = __ldg(a.pair_cnt + i);
        p.r0 = __ldg(a.pair_rec + (size_t)i * a.max_nbr + lane);
    }
    return p;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }
__device__ __forceinline__ void cp_async16(void *dst, const void *src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}

// Start copying atom i's g row (raw, compact order) and the A rows of its
// class's channels into the warp's shared buffers (cp.async; lane t % 32
// copies chunk t).  The buffers must no longer be in use.
template <int N>
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
        cp_async16(sA + ch * kAStride + 4 * (k & 3), Ag + ch * 16 + 4 * (k & 3));
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

template <int N>
__global__ void __launch_bounds__(kWarpsForce * 32, 4) k_force(ForceArgs a)
{
    constexpr int C = 2 * N;
    __shared__ __align__(16) ForceSmem<N> sm;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const float rc = a.rcut;
    float vir[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) vir[k] = 0.f;
    if (lane < kSlots) sm.atom[w][lane] = -1;
    for (int k = lane; k < 9 * kSlots; k += 32) sm.V[w][k / 9][k % 9] = 0;
    const bool want_vatom = a.vir_atom != nullptr;
    {
        // where each compact channel pair (a, b) of g lands in the dense G~ of
        // its class: offsets of (b, a) and (a, b); equal on the diagonal
        constexpr int NPF = C * (C + 1) / 2, NPS = N * (N + 1) / 2;
        for (int t = threadIdx.x; t < NPF + NPS; t += blockDim.x) {
            const bool full = t < NPF;
            const int e = __ldg(full ? a.tab[0] + 4 * t : a.tab[1] + 4 * (t - NPF));
            const int ca = e & 255, cb = (e >> 8) & 255;
            const int RS = full ? gd_row(C) : gd_row(N);
            sm.goff[t] = make_int2(cb * RS + ca, ca * RS + cb);
        }
    }
    __syncthreads();
    int nq = 0;        // queued pairs
    int seq = 0;       // atoms given a w slot so far by this warp
    // warps take chunks of consecutive atoms dynamically; the next atom's
    // scalars are loaded, and its g and A rows copied, one atom ahead
    WarpChunks wc;
    wc.init(a.sched, a.n, lane);
    int i = wc.pos();
    AtomPre cur = preload(a, i, a.n, lane);
    rows_async<N>(a, cur, i, a.n, sm.gr[w], sm.A[w], lane);
    int i2 = a.n;
    AtomPre nxt;
    for (; i < a.n; i = i2, cur = nxt, wc.advance(lane)) {
        i2 = wc.peek();
        nxt = preload(a, i2, a.n, lane);
        const int g = cur.g;
        if (g < 0 || !(cur.nrm > 0.f)) {
            // no environment inside r_cut: no forces from this centre
            if (lane == 0 && g < 0) {
                a.energy[i] = 0.f;
                if (a.variance) a.variance[i] = 0.f;
                if (a.sigma) a.sigma[i] = 0.f;
            }
            if (want_vatom && lane < 9) a.vir_atom[9 * (size_t)i + lane] = 0.f;
            rows_async<N>(a, nxt, i2, a.n, sm.gr[w], sm.A[w], lane);
            continue;
        }
        const int cls = group_cls(g), reg = group_region(g);
        const int K = a.K[reg];
        const int choff = cls == 0 ? 0 : (cls - 1) * N;

        // w slot for this atom: if a queued pair still refers to the slot, evaluate the queue first
        const int slot = seq & (kSlots - 1);
        if (nq > 0 && sm.qseq[w][0] <= seq - kSlots) drain<N>(sm, w, lane, nq, true, rc, a.Facc, a.status, vir, want_vatom);
        if (want_vatom) flush_slot<N>(sm, w, lane, slot, a.vir_atom);   // otherwise the slot holds nothing to write
        if (lane == 0) sm.atom[w][slot] = i;

        // this atom's g row and A rows were copied into shared memory while the
        // previous atom was processed
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncwarp();
        // g = dE/dB of this atom (compact order of its class, written by the
        // quadratic-form epilogue; scaled by u_i in the backward pass) ->
        // dense symmetric G~[l][b][a] with the diagonal doubled
        {
            const float4 *g4 = reinterpret_cast<const float4 *>(sm.gr[w]);
            const int2 *goff = sm.goff + (reg == 0 ? 0 : C * (C + 1) / 2);
            const float u = a.weight ? __ldg(a.weight + i) : 1.f;
            const int LS = cls == 0 ? gd_plane(C) : gd_plane(N);
            float *sGd = sm.Gd[w];
            for (int t = lane; 4 * t < K; t += 32) {
                const int2 of = goff[t];
                const int o1 = of.x, o2 = of.y;
                float4 v = g4[t];
                const float sc = o1 == o2 ? 2.f * u : u;   // the diagonal of G~ is doubled
                v.x *= sc;
                v.y *= sc;
                v.z *= sc;
                v.w *= sc;
                sGd[o1] = v.x;
                sGd[o2] = v.x;
                sGd[LS + o1] = v.y;
                sGd[LS + o2] = v.y;
                sGd[2 * LS + o1] = v.z;
                sGd[2 * LS + o2] = v.z;
                sGd[3 * LS + o1] = v.w;
                sGd[3 * LS + o2] = v.w;
            }
        }
        float *sA = sm.A[w];   // A rows of the class's channels (already copied)
        float *ws = sm.W[w] + slot * kWSlot;
        // w_dense writes every channel of the atom's class; pairs only read
        // the species blocks of that class, so the slot needs no clearing
        __syncwarp();
        {
            const int lm = lane & 15, half = lane >> 4;
            if (cls == 0)
                w_dense<C, N>(sm.Gd[w], sA, ws, 0, half, lm);
            else
                w_dense<N, N>(sm.Gd[w], sA, ws, choff, half, lm);
        }
        __syncwarp();
        // the g and A buffers are free: start copying the next atom's rows
        rows_async<N>(a, nxt, i2, a.n, sm.gr[w], sm.A[w], lane);

        // queue the atom's pairs inside r_cut (recorded by the descriptor kernel)
        const int np = cur.np;
        const float4 *pr = a.pair_rec + (size_t)i * a.max_nbr;
        for (int base = 0; base < np; base += 32) {
            const int take = min(32, np - base);
            if (lane < take) {
                float4 r = base == 0 ? cur.r0 : __ldg(pr + base + lane);
                r.w = __int_as_float(__float_as_int(r.w) | (slot << 26));
                sm.q[w][nq + lane] = r;
                sm.qseq[w][nq + lane] = seq;
            }
            nq += take;
            __syncwarp();
            drain<N>(sm, w, lane, nq, false, rc, a.Facc, a.status, vir, want_vatom);
        }
        ++seq;
    }  // atoms
    drain<N>(sm, w, lane, nq, true, rc, a.Facc, a.status, vir, want_vatom);
    if (want_vatom)
        for (int s = 0; s < kSlots; ++s) flush_slot<N>(sm, w, lane, s, a.vir_atom);

    // virial: warp reduce, then a fixed-order FP64 sum over the block's warps
#pragma unroll
    for (int k = 0; k < 9; ++k)
        for (int o = 16; o; o >>= 1) vir[k] += __shfl_xor_sync(0xffffffffu, vir[k], o);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 9; ++k) sm.vir[w][k] = vir[k];
    __syncthreads();
    if (threadIdx.x < 9) {
        double s = 0.0;
        for (int q = 0; q < kWarpsForce; ++q) s += (double)sm.vir[q][threadIdx.x];
        a.vir_part[(size_t)blockIdx.x * 9 + threadIdx.x] = s;
    }
}

// ---- finalize: fixed point -> float forces, optional velocity half-kick,
// ---- FP64 block partials of E, max sigma, isolated atoms, kinetic energy
struct FinArgs {
    const unsigned long long *Facc;
    const float *energy, *sigma, *norm;
    float *forces;
    int n;
    double *part;          // [gridDim.x][4]
    KickArgs kick;
    float sign;            // 1: forces; -1: gradient of the (weighted) energy
};

__global__ void __launch_bounds__(256) k_finalize(FinArgs a)
{
    __shared__ double sE[8], sK[8];
    __shared__ float sS[8];
    __shared__ int sI[8];
    double e = 0.0, ke = 0.0;
    float smax = 0.f;
    int iso = 0;
    for (int i = blockIdx.x * 256 + threadIdx.x; i < a.n; i += gridDim.x * 256) {
        float f[3];
        // RN(x) * 2^-32 is exact scaling of the correctly rounded integer, so
        // this equals RN(x * 2^-32) without FP64 arithmetic
#pragma unroll
        for (int c = 0; c < 3; ++c)
            f[c] = a.sign * (__ll2float_rn((long long)a.Facc[3 * (size_t)i + c]) * 0x1p-32f);
        a.forces[3 * (size_t)i + 0] = f[0];
        a.forces[3 * (size_t)i + 1] = f[1];
        a.forces[3 * (size_t)i + 2] = f[2];
        e += (double)a.energy[i];
        if (a.sigma) smax = fmaxf(smax, a.sigma[i]);
        iso += a.norm[i] > 0.f ? 0 : 1;
        if (a.kick.enabled) {
            const int s = min(max(a.kick.species[i], 0), kSpecies - 1);
            float4 v = a.kick.vel[i];
            const float h = a.kick.half_dt_over_m[s];
            v.x += h * f[0];
            v.y += h * f[1];
            v.z += h * f[2];
            a.kick.vel[i] = v;
            ke += (double)(a.kick.half_m[s] * (v.x * v.x + v.y * v.y + v.z * v.z));
        }
    }
    for (int o = 16; o; o >>= 1) {
        e += __shfl_xor_sync(0xffffffffu, e, o);
        ke += __shfl_xor_sync(0xffffffffu, ke, o);
        smax = fmaxf(smax, __shfl_xor_sync(0xffffffffu, smax, o));
        iso += __shfl_xor_sync(0xffffffffu, iso, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        sE[w] = e;
        sK[w] = ke;
        sS[w] = smax;
        sI[w] = iso;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double E = 0.0, KE = 0.0;
        float S = 0.f;
        int I = 0;
        for (int q = 0; q < 8; ++q) {
            E += sE[q];
            KE += sK[q];
            S = fmaxf(S, sS[q]);
            I += sI[q];
        }
        double *p = a.part + (size_t)blockIdx.x * 4;
        p[0] = E;
        p[1] = KE;
        p[2] = (double)S;
        p[3] = (double)I;
    }
}

struct TotArgs {
    const double *vir_part;
    int n_vir;
    const double *part;
    int n_part;
    double *totals;
    const int32_t *nl_flags;
    const int *ref_count;    // atoms whose variance was re-evaluated in FP64 (or nullptr)
    int kick;
};

__global__ void __launch_bounds__(1024) k_totals(TotArgs a)
{
    __shared__ double red[32][12];
    double acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = 0.0;
    for (int b = threadIdx.x; b < a.n_vir; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < 9; ++k) acc[k] += a.vir_part[(size_t)b * 9 + k];
    for (int b = threadIdx.x; b < a.n_part; b += blockDim.x) {
        acc[9] += a.part[(size_t)b * 4 + 0];
        acc[10] += a.part[(size_t)b * 4 + 1];
        acc[11] = fmax(acc[11], a.part[(size_t)b * 4 + 2]);
    }
    double iso = 0.0;
    for (int b = threadIdx.x; b < a.n_part; b += blockDim.x) iso += a.part[(size_t)b * 4 + 3];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 16; o; o >>= 1) {
#pragma unroll
        for (int k = 0; k < 11; ++k) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
        acc[11] = fmax(acc[11], __shfl_xor_sync(0xffffffffu, acc[11], o));
        iso += __shfl_xor_sync(0xffffffffu, iso, o);
    }
    __shared__ double riso[32];
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < 12; ++k) red[w][k] = acc[k];
        riso[w] = iso;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t[12] = {0};
        double I = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
            for (int k = 0; k < 11; ++k) t[k] += red[q][k];
            t[11] = fmax(t[11], red[q][11]);
            I += riso[q];
        }
        a.totals[FLR_TOT_ENERGY] = t[9];
        for (int k = 0; k < 9; ++k) a.totals[FLR_TOT_VIRIAL + k] = t[k];
        a.totals[FLR_TOT_MAX_SIGMA] = t[11];
        a.totals[FLR_TOT_N_ISOLATED] = I;
        if (a.kick) a.totals[FLR_TOT_KINETIC] = t[10];
        a.totals[FLR_TOT_N_VAR_FP64] = a.ref_count ? (double)*a.ref_count : 0.0;
    }
}

// Per-structure totals of a batch: one block per structure sums its atoms in
// a fixed order (E in FP64, the per-atom virials, max sigma, isolated atoms).
struct SegArgs {
    const int32_t *offsets;
    int n_structs;
    const float *energy, *sigma, *norm, *vir_atom;
    double *totals;   // [n_structs][FLR_NTOTALS]
};

__global__ void __launch_bounds__(256) k_seg_totals(SegArgs a)
{
    __shared__ double red[8][12];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int s = blockIdx.x; s < a.n_structs; s += gridDim.x) {
        double acc[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[k] = 0.0;
        for (int i = a.offsets[s] + threadIdx.x; i < a.offsets[s + 1]; i += blockDim.x) {
            acc[0] += (double)a.energy[i];
#pragma unroll
            for (int k = 0; k < 9; ++k) acc[1 + k] += (double)a.vir_atom[9 * (size_t)i + k];
            if (a.sigma) acc[10] = fmax(acc[10], (double)a.sigma[i]);
            acc[11] += a.norm[i] > 0.f ? 0.0 : 1.0;
        }
        for (int o = 16; o; o >>= 1) {
#pragma unroll
            for (int k = 0; k < 10; ++k) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], o);
            acc[10] = fmax(acc[10], __shfl_xor_sync(0xffffffffu, acc[10], o));
            acc[11] += __shfl_xor_sync(0xffffffffu, acc[11], o);
        }
        if (lane == 0)
#pragma unroll
            for (int k = 0; k < 12; ++k) red[w][k] = acc[k];
        __syncthreads();
        if (threadIdx.x == 0) {
            double t[12] = {0};
            for (int q = 0; q < 8; ++q) {
                for (int k = 0; k < 10; ++k) t[k] += red[q][k];
                t[10] = fmax(t[10], red[q][10]);
                t[11] += red[q][11];
            }
            double *o = a.totals + (size_t)s * FLR_NTOTALS;
            for (int k = 0; k < FLR_NTOTALS; ++k) o[k] = 0.0;
            o[FLR_TOT_ENERGY] = t[0];
            for (int k = 0; k < 9; ++k) o[FLR_TOT_VIRIAL + k] = t[1 + k];
            o[FLR_TOT_MAX_SIGMA] = t[10];
            o[FLR_TOT_N_ISOLATED] = t[11];
        }
        __syncthreads();
    }
}

}  // namespace

int launch_seg_totals(flr_ctx *ctx, const flr_nbrlist *nl, const flr_outputs *out, const float *vir_atom,
                      double *totals, cudaStream_t st)
{
    SegArgs s;
    s.offsets = nl->offsets_d;
    s.n_structs = nl->n_structs;
    s.energy = out->energy;
    s.sigma = out->sigma;
    s.norm = ctx->norm;
    s.vir_atom = vir_atom;
    s.totals = totals;
    k_seg_totals<<<std::max(1, std::min(nl->n_structs, ctx->num_sms * 8)), 256, 0, st>>>(s);
    count_launch(ctx);
    return cuda_fail(cudaGetLastError(), "per-structure totals");
}

int launch_force(flr_ctx *ctx, const flr_nbrlist *nl, const float4 *pos, const int *species, int n,
                 flr_outputs *out, float *vir_atom, const float *weight, cudaStream_t st)
{
    ForceArgs a;
    a.pos = pos;
    a.species = species;
    a.entries = nl->entries;
    a.count = nl->count;
    a.group = nl->group;
    a.row = nl->row;
    a.max_nbr = nl->max_nbr;
    a.n = n;
    a.rcut = (float)ctx->p.r_cut;
    for (int r = 0; r < 2; ++r) {
        a.K[r] = ctx->dims.K[r];
        a.G[r] = ctx->G[r];
    }
    a.A = ctx->A;
    a.norm = ctx->norm;
    a.energy = out->energy;
    a.variance = out->variance;
    a.sigma = out->sigma;
    a.Facc = reinterpret_cast<unsigned long long *>(ctx->Facc);
    a.vir_part = ctx->partials;
    a.vir_atom = vir_atom;
    a.weight = weight;
    a.pair_rec = nl->pair_rec;
    a.pair_cnt = nl->pair_cnt;
    a.tab[0] = ctx->tab_full;
    a.tab[1] = ctx->tab_single;
    a.status = ctx->status;
    a.sched = ctx->sched + 1;
    {
        const cudaError_t e = cudaMemsetAsync(a.sched, 0, sizeof(int), st);
        if (e != cudaSuccess) return cuda_fail(e, "force work counter");
    }
    const long long work = (n + kWarpsForce - 1) / kWarpsForce;
    int grid;
    if (ctx->dims.N == 8) {
        grid = std::min(kMaxPartials, persistent_grid(k_force<8>, kWarpsForce * 32, ctx->num_sms, work));
        k_force<8><<<grid, kWarpsForce * 32, 0, st>>>(a);
    } else {
        grid = std::min(kMaxPartials, persistent_grid(k_force<7>, kWarpsForce * 32, ctx->num_sms, work));
        k_force<7><<<grid, kWarpsForce * 32, 0, st>>>(a);
    }
    ctx->n_part = grid;
    count_launch(ctx);
    return cuda_fail(cudaGetLastError(), "force kernel");
}

int launch_finalize(flr_ctx *ctx, const flr_nbrlist *nl, int n, flr_outputs *out, const KickArgs &kick, float sign,
                    cudaStream_t st)
{
    (void)nl;
    const int n_vir = ctx->n_part;
    const int nfin = std::min(kMaxPartials, persistent_grid(k_finalize, 256, ctx->num_sms, (n + 255) / 256));
    FinArgs f;
    f.Facc = reinterpret_cast<const unsigned long long *>(ctx->Facc);
    f.energy = out->energy;
    f.sigma = out->sigma;
    f.norm = ctx->norm;
    f.forces = out->forces;
    f.n = n;
    f.part = ctx->partials + (size_t)kMaxPartials * 9;
    f.kick = kick;
    f.sign = sign;
    k_finalize<<<nfin, 256, 0, st>>>(f);
    TotArgs t;
    t.vir_part = ctx->partials;
    t.n_vir = n_vir;
    t.part = f.part;
    t.n_part = nfin;
    t.totals = out->totals;
    t.nl_flags = nl ? nl->flags : nullptr;
    t.ref_count = ctx->var_mode == FLR_VAR_AUTO ? ctx->ref_count : nullptr;
    t.kick = kick.enabled;
    if (out->totals) k_totals<<<1, 1024, 0, st>>>(t);
    count_launch(ctx, out->totals ? 2 : 1);
    return cuda_fail(cudaGetLastError(), "finalize");
}

}  // namespace flr
