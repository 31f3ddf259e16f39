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
// which costs O(N L^2) per pair instead of O(d).  F_i += f_ij, F_j -= f_ij;
// the scatter to j goes through 64-bit fixed-point atomics (2^-32 eV/A
// resolution), whose integer sums do not depend on arrival order, so the
// forces are bitwise reproducible.
#include "basis.cuh"
#include "internal.cuh"

namespace flr {
namespace {

constexpr int kAStride = 17;
constexpr float kFixScale = 4294967296.0f;   // 2^32

struct ForceArgs {
    const float4 *pos;
    const int32_t *species;
    const int32_t *entries, *count, *group, *row;
    int max_nbr, n;
    CellArg cell;
    float rcut;
    const float *D32[2];
    int kp32[2], K[2];
    const float *P[2];
    const float *A, *norm;
    float *energy, *variance, *sigma;
    unsigned long long *Facc;
    double *vir_part;          // [gridDim.x][9]
    int *status;
};

template <int N>
struct ForceSmem {
    float G[kWarpsDesc][(2 * N) * (2 * N + 1) / 2 * 4];
    float A[kWarpsDesc][2 * N * kAStride];
    float W[kWarpsDesc][2 * N * kAStride];
    float vir[kWarpsDesc][9];
};

__device__ __forceinline__ int tri(int a, int b, int C) { return a * C - a * (a - 1) / 2 + (b - a); }

__device__ __forceinline__ void fix_add(unsigned long long *dst, float v, int *status)
{
    const float s = v * kFixScale;
    if (!(fabsf(s) < 9.0e18f)) {   // also catches NaN
        atomicOr(status, kErrNonFinite);
        return;
    }
    atomicAdd(dst, (unsigned long long)__float2ll_rn(s));
}

template <int N>
__global__ void __launch_bounds__(kWarpsDesc * 32) k_force(ForceArgs a)
{
    constexpr int KF = (2 * N) * (2 * N + 1) / 2 * 4;
    constexpr int NK = (KF + 31) / 32;
    __shared__ __align__(16) ForceSmem<N> sm;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float vir[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) vir[k] = 0.f;
    // persistent warps: a fixed grid walks the atoms (and keeps the virial partials few)
    for (int i = blockIdx.x * kWarpsDesc + w; i < a.n; i += gridDim.x * kWarpsDesc) {
    const int g = a.group[i];

    if (g >= 0) {
        const int cls = group_cls(g), reg = group_region(g);
        const int K = a.K[reg];
        const int r = a.row[i];
        const float *d = a.D32[reg] + (size_t)r * a.kp32[reg];
        const float *pr = a.P[reg] + (size_t)r * (2 * K);
        float dv[NK], pb[NK];
        float E = 0.f, V = 0.f;
#pragma unroll
        for (int k = 0; k < NK; ++k) {
            const int o = lane + 32 * k;
            dv[k] = 0.f;
            pb[k] = 0.f;
            if (o < K) {
                dv[k] = d[o];
                pb[k] = pr[o];
                E += dv[k] * pb[k];
                V += dv[k] * pr[K + o];
            }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            E += __shfl_xor_sync(0xffffffffu, E, o);
            V += __shfl_xor_sync(0xffffffffu, V, o);
        }
        if (lane == 0) {
            a.energy[i] = E;
            if (a.variance) a.variance[i] = V;
            if (a.sigma) a.sigma[i] = sqrtf(fmaxf(V, 0.f));
        }
        const float nrm = a.norm[i];
        if (nrm > 0.f) {
            // g = (2/||B||)(beta d - E d) in the class's compact order
            const float s2 = 2.f / nrm;
            float *sG = sm.G[w];
#pragma unroll
            for (int k = 0; k < NK; ++k) {
                const int o = lane + 32 * k;
                if (o < K) sG[o] = s2 * (pb[k] - E * dv[k]);
            }
            // A of the blocks in use (zeros elsewhere)
            float *sA = sm.A[w];
            const float *Ag = a.A + (size_t)i * (2 * N * 16);
            for (int k = lane; k < 2 * N * 16; k += 32) {
                const int c = k >> 4, lm = k & 15;
                const bool used = cls == 0 || (c / N) == (cls - 1);
                sA[c * kAStride + lm] = used ? Ag[k] : 0.f;
            }
            __syncwarp();
            // w = G~ A over the class's channels
            const int Cg = cls == 0 ? 2 * N : N;
            const int choff = cls == 0 ? 0 : (cls - 1) * N;
            float *sW = sm.W[w];
            const int my_n = lane >> 2, quad = lane & 3;
            for (int k = lane; k < 2 * N * kAStride; k += 32) sW[k] = 0.f;
            __syncwarp();
            if (my_n < N) {
                for (int blk = 0; blk < (cls == 0 ? 2 : 1); ++blk) {
                    const int aloc = blk * N + my_n;   // channel inside the class
                    float acc[4] = {0.f, 0.f, 0.f, 0.f};
                    for (int bloc = 0; bloc < Cg; ++bloc) {
                        const int lo = min(aloc, bloc), hi = max(aloc, bloc);
                        const float *gp = sG + tri(lo, hi, Cg) * 4;
                        const float dbl = aloc == bloc ? 2.f : 1.f;
                        const float *ap = sA + (choff + bloc) * kAStride + 4 * quad;
#pragma unroll
                        for (int k = 0; k < 4; ++k) acc[k] += dbl * gp[l_of(4 * quad + k)] * ap[k];
                    }
#pragma unroll
                    for (int k = 0; k < 4; ++k) sW[(choff + aloc) * kAStride + 4 * quad + k] = acc[k];
                }
            }
            __syncwarp();

            // per-pair forces
            const float4 pi = a.pos[i];
            const int cnt = a.count[i];
            const int32_t *rowp = a.entries + (size_t)i * a.max_nbr;
            const float rc = a.rcut, rc2 = rc * rc;
            float fi[3] = {0.f, 0.f, 0.f};
            for (int base = 0; base < cnt; base += 32) {
                const int q = base + lane;
                if (q < cnt) {
                    int j, sx, sy, sz;
                    decode_entry(rowp[q], j, sx, sy, sz);
                    const float4 pj = a.pos[j];
                    const float3 rv = pair_vector(pi, pj, sx, sy, sz, a.cell);
                    const float d2 = rv.x * rv.x + rv.y * rv.y + rv.z * rv.z;
                    if (d2 < rc2) {
                        const int sj = a.species[j];
                        const float rr = sqrtf(d2), inv = 1.f / rr;
                        const float ux = rv.x * inv, uy = rv.y * inv, uz = rv.z * inv;
                        float Rf[N], dRf[N];
                        radial<N, true>(rr, rc, Rf, dRf);
                        float Y[16];
                        real_ylm(ux, uy, uz, Y);
                        const float *wp = sW + (sj == 0 ? 0 : N) * kAStride;
                        float c[16], cp[16];
#pragma unroll
                        for (int lm = 0; lm < 16; ++lm) {
                            float s = 0.f, t = 0.f;
#pragma unroll
                            for (int n = 0; n < N; ++n) {
                                const float wv = wp[n * kAStride + lm];
                                s += wv * Rf[n];
                                t += wv * dRf[n];
                            }
                            c[lm] = s;
                            cp[lm] = t;
                        }
                        float gx, gy, gz, lsum;
                        ylm_grad_contract(ux, uy, uz, c, Y, gx, gy, gz, lsum);
                        float radial_part = 0.f;
#pragma unroll
                        for (int lm = 0; lm < 16; ++lm) radial_part += cp[lm] * Y[lm];
                        const float coef = radial_part - lsum * inv;
                        const float fx = coef * ux + gx * inv;
                        const float fy = coef * uy + gy * inv;
                        const float fz = coef * uz + gz * inv;
                        fi[0] += fx;
                        fi[1] += fy;
                        fi[2] += fz;
                        unsigned long long *dst = a.Facc + 3 * (size_t)j;
                        fix_add(dst + 0, -fx, a.status);
                        fix_add(dst + 1, -fy, a.status);
                        fix_add(dst + 2, -fz, a.status);
                        vir[0] -= rv.x * fx; vir[1] -= rv.x * fy; vir[2] -= rv.x * fz;
                        vir[3] -= rv.y * fx; vir[4] -= rv.y * fy; vir[5] -= rv.y * fz;
                        vir[6] -= rv.z * fx; vir[7] -= rv.z * fy; vir[8] -= rv.z * fz;
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < 3; ++c)
                for (int o = 16; o; o >>= 1) fi[c] += __shfl_xor_sync(0xffffffffu, fi[c], o);
            if (lane == 0) {
                unsigned long long *dst = a.Facc + 3 * (size_t)i;
                fix_add(dst + 0, fi[0], a.status);
                fix_add(dst + 1, fi[1], a.status);
                fix_add(dst + 2, fi[2], a.status);
            }
        }
    } else {
        if (lane == 0) {
            a.energy[i] = 0.f;
            if (a.variance) a.variance[i] = 0.f;
            if (a.sigma) a.sigma[i] = 0.f;
        }
    }
    __syncwarp();
    }  // atoms
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
        for (int q = 0; q < kWarpsDesc; ++q) s += (double)sm.vir[q][threadIdx.x];
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
#pragma unroll
        for (int c = 0; c < 3; ++c)
            f[c] = (float)((double)(long long)a.Facc[3 * (size_t)i + c] * (1.0 / 4294967296.0));
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
            ke += (double)a.kick.half_m[s] * (double)(v.x * v.x + v.y * v.y + v.z * v.z);
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
    }
}

}  // namespace

int launch_force(flr_ctx *ctx, const flr_nbrlist *nl, const float4 *pos, const int *species, int n,
                 flr_outputs *out, cudaStream_t st)
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
    for (int c = 0; c < 9; ++c) a.cell.c[c] = nl->plan.cell[c];
    a.rcut = (float)ctx->p.r_cut;
    for (int r = 0; r < 2; ++r) {
        a.D32[r] = ctx->D32[r];
        a.kp32[r] = ctx->dims.kp32[r];
        a.K[r] = ctx->dims.K[r];
        a.P[r] = ctx->P[r];
    }
    a.A = ctx->A;
    a.norm = ctx->norm;
    a.energy = out->energy;
    a.variance = out->variance;
    a.sigma = out->sigma;
    a.Facc = reinterpret_cast<unsigned long long *>(ctx->Facc);
    a.vir_part = ctx->partials;
    a.status = ctx->status;
    const long long work = (n + kWarpsDesc - 1) / kWarpsDesc;
    int grid;
    if (ctx->dims.N == 8) {
        grid = std::min(kMaxPartials, persistent_grid(k_force<8>, kWarpsDesc * 32, ctx->num_sms, work));
        k_force<8><<<grid, kWarpsDesc * 32, 0, st>>>(a);
    } else {
        grid = std::min(kMaxPartials, persistent_grid(k_force<7>, kWarpsDesc * 32, ctx->num_sms, work));
        k_force<7><<<grid, kWarpsDesc * 32, 0, st>>>(a);
    }
    ctx->n_part = grid;
    count_launch(ctx);
    return cuda_fail(cudaGetLastError(), "force kernel");
}

int launch_finalize(flr_ctx *ctx, const flr_nbrlist *nl, int n, flr_outputs *out, const KickArgs &kick,
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
    k_finalize<<<nfin, 256, 0, st>>>(f);
    TotArgs t;
    t.vir_part = ctx->partials;
    t.n_vir = n_vir;
    t.part = f.part;
    t.n_part = nfin;
    t.totals = out->totals;
    t.nl_flags = nl ? nl->flags : nullptr;
    t.kick = kick.enabled;
    if (out->totals) k_totals<<<1, 1024, 0, st>>>(t);
    count_launch(ctx, out->totals ? 2 : 1);
    return cuda_fail(cudaGetLastError(), "finalize");
}

}  // namespace flr
