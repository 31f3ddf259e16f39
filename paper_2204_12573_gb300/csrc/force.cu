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
// evaluated alongside.  The per-warp state and the per-atom and per-pair
// steps are in force_dev.cuh; each warp's state is one contiguous block of
// shared memory.
#include <cstddef>

#include "force_dev.cuh"

namespace flr {
namespace {

constexpr int kWarpsForce = 4;                // warps per CTA
constexpr int kForceBlocks = 4;               // CTAs per SM, any class (shared memory and registers allow 4)
constexpr int kForce1Blocks = 5;              // CTAs per SM, one-species classes only (96 registers)

template <class FW, int N>
struct ForceSmem {
    FW wp[kWarpsForce];
    float vir[kWarpsForce][9];
    int2 goff[goff_count<N>()];
};

// The atoms a force launch takes: a.n by index, or order[0 .. m) with m on the device.
__device__ __forceinline__ int force_count(const ForceArgs &a)
{
    if (!a.n_dev[0]) return a.n;
    int m = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (a.n_dev[k]) m += *a.n_dev[k];
    return m < a.n ? m : a.n;
}

// FW = ForceWarp<N> takes atoms of any class; FW = ForceWarp1<N> only atoms
// of the one-species classes (their smaller per-warp state lets more warps
// share an SM).
template <int N, class FW, int MINB>
__global__ void __launch_bounds__(kWarpsForce * 32, MINB) k_force(ForceArgs a)
{
    __shared__ __align__(16) ForceSmem<FW, N> sm;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    FW &fw = sm.wp[w];
    float vir[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) vir[k] = 0.f;
    init_warp(fw, lane);
    const bool want_vatom = a.vir_atom != nullptr;
    init_goff<N>(a, sm.goff, threadIdx.x, blockDim.x);
    __syncthreads();
    int nq = 0;        // queued pairs
    int seq = 0;       // atoms given a w slot so far by this warp
    // warps take chunks of consecutive positions of the atom sequence
    // dynamically; the next atom's scalars are loaded, and its g and A rows
    // copied, one atom ahead
    const int n_take = force_count(a);
    const int i_end = a.order ? 0x7fffffff : a.n;
    // chunks of up to kWarpChunk atoms, shorter when there are fewer than
    // four chunks' worth per warp of the grid
    const int per_warp = n_take / (4 * (int)gridDim.x * kWarpsForce);
    WarpChunksR wc;
    wc.init(a.sched, n_take, per_warp < 1 ? 1 : (per_warp < kWarpChunk ? per_warp : kWarpChunk), lane);
    int p = wc.pos();
    int i = p < n_take ? (a.order ? __ldg(a.order + p) : p) : i_end;
    AtomPre cur = preload(a, i, i_end, lane);
    preload_pairs(a, cur, i, i_end, lane);
    rows_async<N, FW::kOne>(a, cur, i, i_end, fw.gr, fw.A, lane);
    int p2 = n_take, i2 = i_end;
    AtomPre nxt;
    for (; p < n_take; p = p2, i = i2, cur = nxt, wc.advance(lane)) {
        p2 = wc.peek();
        i2 = p2 < n_take ? (a.order ? __ldg(a.order + p2) : p2) : i_end;
        nxt = preload(a, i2, i_end, lane);
        const int g = cur.g;
        if (g < 0 || !(cur.nrm > 0.f)) {
            // no environment inside r_cut: no forces from this centre
            if (lane == 0 && g < 0) {
                a.energy[i] = 0.f;
                if (a.variance) a.variance[i] = 0.f;
                if (a.sigma) a.sigma[i] = 0.f;
            }
            if (want_vatom && lane < 9) a.vir_atom[9 * (size_t)i + lane] = 0.f;
            rows_async<N, FW::kOne>(a, nxt, i2, i_end, fw.gr, fw.A, lane);
            preload_pairs(a, nxt, i2, i_end, lane);
            continue;
        }
        force_atom<N, FW>(a, fw, sm.goff, lane, cur, i, nxt, i2, i_end, nq, seq, vir, want_vatom);
        preload_pairs(a, nxt, i2, i_end, lane);
    }  // atoms
    drain<N, FW>(fw, lane, nq, true, a.rcut, a.two_over_rc, a.Facc, a.status, vir, want_vatom);
    if (want_vatom)
        for (int s = 0; s < kSlots; ++s) flush_slot(fw, lane, s, a.vir_atom);

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
        a.vir_part[(size_t)(a.vir_base + blockIdx.x) * 9 + threadIdx.x] = s;
    }
}

// Atoms with an empty neighbour list (group < 0) belong to no compaction
// group, so neither the quadratic forms nor the class-ordered force launches
// visit them: their outputs are zero.
__global__ void __launch_bounds__(256) k_zero_isolated(const int32_t *group, int n, float *energy, float *variance,
                                                       float *sigma, float *vir_atom)
{
    const int i = blockIdx.x * 256 + threadIdx.x;
    if (i >= n || group[i] >= 0) return;
    energy[i] = 0.f;
    if (variance) variance[i] = 0.f;
    if (sigma) sigma[i] = 0.f;
    if (vir_atom)
        for (int k = 0; k < 9; ++k) vir_atom[9 * (size_t)i + k] = 0.f;
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

// One block per total, 13 blocks on 13 SMs (9 virial entries, E, kinetic
// energy, max sigma, isolated atoms): the FP64 pipe of one SM is narrow on
// this part, and one block holding every total waited on the latency of its
// serial loads (22 us per evaluation).  Each block sums its column of the
// partials in a fixed order (rows strided over its threads, a fixed
// shuffle tree, the warps in order).
constexpr int kTotThreads = 256;
constexpr int kTotBlocks = 13;
__global__ void __launch_bounds__(kTotThreads) k_totals(TotArgs a)
{
    __shared__ double red[kTotThreads / 32];
    const int q = blockIdx.x;
    const bool is_max = q == 11;   // sigma >= 0: 0 is the identity of the max as of the sum
    const double *src = q < 9 ? a.vir_part + q : a.part + (q - 9);
    const int stride = q < 9 ? 9 : 4;
    const int n = q < 9 ? a.n_vir : a.n_part;
    double acc = 0.0;
    for (int b = threadIdx.x; b < n; b += kTotThreads) {
        const double v = src[(size_t)b * stride];
        acc = is_max ? fmax(acc, v) : acc + v;
    }
    for (int o = 16; o; o >>= 1) {
        const double y = __shfl_xor_sync(0xffffffffu, acc, o);
        acc = is_max ? fmax(acc, y) : acc + y;
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x != 0) return;
    double t = red[0];
    for (int w = 1; w < kTotThreads / 32; ++w) t = is_max ? fmax(t, red[w]) : t + red[w];
    if (q < 9) {
        a.totals[FLR_TOT_VIRIAL + q] = t;
    } else if (q == 9) {
        a.totals[FLR_TOT_ENERGY] = t;
    } else if (q == 10) {
        if (a.kick) a.totals[FLR_TOT_KINETIC] = t;
    } else if (q == 11) {
        a.totals[FLR_TOT_MAX_SIGMA] = t;
    } else {
        a.totals[FLR_TOT_N_ISOLATED] = t;
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

template <int N>
int launch_force_n(flr_ctx *ctx, const flr_nbrlist *nl, ForceArgs a, int n, cudaStream_t st)
{
    // two launches over the compaction rows: the two-species rows with the
    // general per-warp state, the one-species rows (nearly all atoms) with the
    // smaller one; each launch's block partials of the virial follow the other's
    const int *cnt = reinterpret_cast<const int *>(reinterpret_cast<const char *>(nl->gtab) + offsetof(GroupTab, count));
    cudaError_t e = cudaMemsetAsync(ctx->sched + 1, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->sched + 3, 0, sizeof(int), st);
    if (e != cudaSuccess) return cuda_fail(e, "force work counters");
    const long long work = (n + kWarpsForce - 1) / kWarpsForce;
    ForceArgs a0 = a, a1 = a;
    a0.order = nl->atom_of_row;
    a0.n_dev[0] = cnt + 0;
    a0.n_dev[1] = cnt + 3;
    a0.n_dev[2] = a0.n_dev[3] = nullptr;
    a0.sched = ctx->sched + 1;
    a0.vir_base = 0;
    const int grid0 = persistent_grid(k_force<N, ForceWarp<N>, kForceBlocks>, kWarpsForce * 32, ctx->num_sms, work);
    a1.order = nl->atom_of_row + nl->n_cap;
    a1.n_dev[0] = cnt + 1;
    a1.n_dev[1] = cnt + 2;
    a1.n_dev[2] = cnt + 4;
    a1.n_dev[3] = cnt + 5;
    a1.sched = ctx->sched + 3;
    a1.vir_base = grid0;
    const int grid1 = persistent_grid(k_force<N, ForceWarp1<N>, kForce1Blocks>, kWarpsForce * 32, ctx->num_sms, work);
    if (grid0 + grid1 > kMaxPartials) {
        set_error("force launch: too many blocks for the virial partials");
        return FLR_EINVAL;
    }
    k_force<N, ForceWarp<N>, kForceBlocks><<<grid0, kWarpsForce * 32, 0, st>>>(a0);
    k_force<N, ForceWarp1<N>, kForce1Blocks><<<grid1, kWarpsForce * 32, 0, st>>>(a1);
    k_zero_isolated<<<(n + 255) / 256, 256, 0, st>>>(nl->group, n, a.energy, a.variance, a.sigma, a.vir_atom);
    ctx->n_part = grid0 + grid1;
    count_launch(ctx, 3);
    return cuda_fail(cudaGetLastError(), "force kernels");
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
    a.two_over_rc = (float)(2.0 / ctx->p.r_cut);
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
    a.order = nullptr;
    for (int k = 0; k < 4; ++k) a.n_dev[k] = nullptr;
    a.vir_base = 0;
    if (n <= 0) {
        ctx->n_part = 0;
        return FLR_OK;
    }
    return ctx->dims.N == 8 ? launch_force_n<8>(ctx, nl, a, n, st) : launch_force_n<7>(ctx, nl, a, n, st);
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
    if (out->totals) k_totals<<<kTotBlocks, kTotThreads, 0, st>>>(t);
    count_launch(ctx, out->totals ? 2 : 1);
    return cuda_fail(cudaGetLastError(), "finalize");
}

}  // namespace flr
