// Velocity-Verlet integration in metal units (Sec. VI-A: MD with the
// force field at every step).  The first half kick and the drift are fused
// here; the second half kick is fused into the force finalize kernel.  The
// drift kernel also checks every atom's displacement since the last
// neighbour build and raises the list's rebuild flag when one moved more
// than half the skin, so the rebuild decision never leaves the device.
//
// Also here: the Nose-Hoover thermostat half steps (one thread advances the
// thermostat from the kinetic energy on the device; the velocity scaling is
// fused into the drift or done by a scaling pass), the kinetic-energy
// reduction that starts a thermostatted call, the count of atoms whose
// sigma exceeds the stop threshold, and the same-species coordination count.
#include <algorithm>

#include "internal.cuh"

namespace flr {
namespace {

struct DriftArgs {
    float4 *pos;
    float4 *vel;
    const float *forces;
    const int32_t *species;
    const float4 *pos_ref;
    int32_t *flags;
    int n;
    float dt;
    float disp2_max;
    float half_dt_over_m[kSpecies];
    const double *scale;   // thermostat velocity scale applied before the kick, or nullptr
};

__global__ void __launch_bounds__(256) k_md_drift(DriftArgs a)
{
    const int i = blockIdx.x * 256 + threadIdx.x;
    bool moved = false;
    if (i < a.n) {
        const int s = min(max(a.species[i], 0), kSpecies - 1);
        const float h = a.half_dt_over_m[s];
        float4 v = a.vel[i];
        if (a.scale) {
            const float sc = (float)*a.scale;
            v.x *= sc;
            v.y *= sc;
            v.z *= sc;
        }
        v.x += h * a.forces[3 * (size_t)i + 0];
        v.y += h * a.forces[3 * (size_t)i + 1];
        v.z += h * a.forces[3 * (size_t)i + 2];
        float4 p = a.pos[i];
        p.x += a.dt * v.x;
        p.y += a.dt * v.y;
        p.z += a.dt * v.z;
        a.vel[i] = v;
        a.pos[i] = p;
        const float4 r = a.pos_ref[i];
        const float dx = p.x - r.x, dy = p.y - r.y, dz = p.z - r.z;
        moved = dx * dx + dy * dy + dz * dz > a.disp2_max;
    }
    if (__any_sync(0xffffffffu, moved) && (threadIdx.x & 31) == 0) a.flags[0] = 1;
}

// Host-state MD: the state crosses the host link as x, y, z rows (12 bytes
// per atom and array instead of 16); these two kernels move it between those
// staging rows and the float4 working copies.  w of the positions is set to
// 0 (unused by every kernel), w of the velocities likewise.
__global__ void __launch_bounds__(256) k_state_unpack(const float *p3, const float *v3, float4 *pos, float4 *vel,
                                                      int n)
{
    const int i = blockIdx.x * 256 + threadIdx.x;
    if (i >= n) return;
    const size_t k = 3 * (size_t)i;
    pos[i] = make_float4(p3[k], p3[k + 1], p3[k + 2], 0.f);
    vel[i] = make_float4(v3[k], v3[k + 1], v3[k + 2], 0.f);
}

__global__ void __launch_bounds__(256) k_state_pack(const float4 *src, float *dst3, int n)
{
    const int i = blockIdx.x * 256 + threadIdx.x;
    if (i >= n) return;
    const size_t k = 3 * (size_t)i;
    const float4 v = src[i];
    dst3[k] = v.x;
    dst3[k + 1] = v.y;
    dst3[k + 2] = v.z;
}

// Kinetic energy sum_i m_i v_i^2 / 2 (eV) in a fixed order: fixed grid,
// per-block FP64 partials, then one block sums them.
constexpr int kKeBlocks = 256;
__global__ void __launch_bounds__(256) k_kinetic_part(const float4 *vel, const int32_t *species, int n,
                                                      float m0, float m1, double *part)
{
    __shared__ double red[8];
    double ke = 0.0;
    for (int i = blockIdx.x * 256 + threadIdx.x; i < n; i += kKeBlocks * 256) {
        const float4 v = vel[i];
        const float m = species[i] == 0 ? m0 : m1;
        ke += (double)(m * (v.x * v.x + v.y * v.y + v.z * v.z));
    }
    for (int o = 16; o; o >>= 1) ke += __shfl_xor_sync(0xffffffffu, ke, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ke;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += red[w];
        part[blockIdx.x] = t;
    }
}
__global__ void k_kinetic_sum(const double *part, double *ke)
{
    double t = 0.0;
    for (int b = 0; b < kKeBlocks; ++b) t += part[b];
    *ke = t;
}

// One Nose-Hoover half step (one thermostat):
//   xi += G dt/4;  s = exp(-xi dt/2) (velocities and KE scaled by s, s^2);
//   eta += xi dt/2;  xi += G dt/4,   with G = (2 KE - g kB T) / Q.
// sc: [0] xi, [1] eta, [2] KE (eV, the velocities' current value), [3] s.
// ke_in: kinetic energy to start from (nullptr: sc[2]).
__global__ void k_thermo_half(double *sc, const double *ke_in, double gkT, double Q, double dt, double *totals)
{
    double xi = sc[0], eta = sc[1];
    double ke = ke_in ? *ke_in : sc[2];
    xi += 0.25 * dt * (2.0 * ke - gkT) / Q;
    const double s = exp(-0.5 * dt * xi);
    ke *= s * s;
    eta += 0.5 * dt * xi;
    xi += 0.25 * dt * (2.0 * ke - gkT) / Q;
    sc[0] = xi;
    sc[1] = eta;
    sc[2] = ke;
    sc[3] = s;
    if (totals) {
        totals[FLR_TOT_KINETIC] = ke;
        totals[FLR_TOT_THERMOSTAT] = 0.5 * Q * xi * xi + gkT * eta;
    }
}

__global__ void __launch_bounds__(256) k_scale_vel(float4 *vel, int n, const double *scale)
{
    const int i = blockIdx.x * 256 + threadIdx.x;
    if (i >= n) return;
    const float sc = (float)*scale;
    float4 v = vel[i];
    v.x *= sc;
    v.y *= sc;
    v.z *= sc;
    vel[i] = v;
}

// Atoms whose sigma exceeds thr (integer count: order-independent).
__global__ void __launch_bounds__(256) k_count_above(const float *sigma, int n, float thr, int *count)
{
    int c = 0;
    for (int i = blockIdx.x * 256 + threadIdx.x; i < n; i += gridDim.x * 256) c += sigma[i] > thr ? 1 : 0;
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

// Atoms of species cs with a neighbour of species cs closer than sqrt(rc2),
// from the pair records of the last descriptor pass (pairs inside r_cut).
__global__ void __launch_bounds__(256) k_cn_count(const int32_t *group, const int32_t *pair_cnt,
                                                  const float4 *pair_rec, int max_nbr, const int32_t *species,
                                                  int n, int cs, float rc2, int *count)
{
    int c = 0;
    for (int i = blockIdx.x * 256 + threadIdx.x; i < n; i += gridDim.x * 256) {
        if (species[i] != cs || group[i] < 0) continue;
        const int np = pair_cnt[i];
        const float4 *r = pair_rec + (size_t)i * max_nbr;
        bool hit = false;
        for (int k = 0; k < np && !hit; ++k) {
            const float4 q = r[k];
            const int sj = (__float_as_int(q.w) >> 25) & 1;
            hit = sj == cs && q.x * q.x + q.y * q.y + q.z * q.z < rc2;
        }
        c += hit ? 1 : 0;
    }
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(count, c);
}

__global__ void k_store_count(const int *count, double *totals, int index) { totals[index] = (double)*count; }

__global__ void k_set_flag(int32_t *flags) { flags[0] = 1; }
__global__ void k_clear_counter(int32_t *flags) { flags[1] = 0; }
__global__ void k_copy_rebuilds(const int32_t *flags, double *totals) { totals[FLR_TOT_N_REBUILDS] = flags[1]; }

}  // namespace

int launch_md_drift(flr_ctx *ctx, flr_nbrlist *nl, float4 *pos, float4 *vel, const float *forces,
                    const int *species, int n, const KickArgs &kick, float dt, float disp2_max,
                    cudaStream_t st)
{
    DriftArgs a;
    a.pos = pos;
    a.vel = vel;
    a.forces = forces;
    a.species = species;
    a.pos_ref = nl->pos_ref;
    a.flags = nl->flags;
    a.n = n;
    a.dt = dt;
    a.disp2_max = disp2_max;
    for (int s = 0; s < kSpecies; ++s) a.half_dt_over_m[s] = kick.half_dt_over_m[s];
    a.scale = kick.scale;
    k_md_drift<<<(n + 255) / 256, 256, 0, st>>>(a);
    count_launch(ctx);
    return cuda_fail(cudaGetLastError(), "md drift");
}

int launch_state_unpack(flr_ctx *ctx, const float *pos3, const float *vel3, float4 *pos, float4 *vel, int n,
                        cudaStream_t st)
{
    if (n <= 0) return FLR_OK;
    k_state_unpack<<<(n + 255) / 256, 256, 0, st>>>(pos3, vel3, pos, vel, n);
    count_launch(ctx);
    return cuda_fail(cudaGetLastError(), "unpack host state");
}

int launch_state_pack(flr_ctx *ctx, const float4 *src, float *dst3, int n, cudaStream_t st)
{
    if (n <= 0) return FLR_OK;
    k_state_pack<<<(n + 255) / 256, 256, 0, st>>>(src, dst3, n);
    count_launch(ctx);
    return cuda_fail(cudaGetLastError(), "pack host state");
}

int launch_kinetic(flr_ctx *ctx, const float4 *vel, const int32_t *species, int n, const double *masses,
                   double *part, double *ke, cudaStream_t st)
{
    // m v^2 / 2 in eV for v in A/ps and m in amu: 1 amu A^2/ps^2 = 1.0364269e-4 eV
    k_kinetic_part<<<kKeBlocks, 256, 0, st>>>(vel, species, n, (float)(0.5 * masses[0] * 1.0364269e-4),
                                              (float)(0.5 * masses[1] * 1.0364269e-4), part);
    k_kinetic_sum<<<1, 1, 0, st>>>(part, ke);
    count_launch(ctx, 2);
    return cuda_fail(cudaGetLastError(), "kinetic energy");
}

int launch_thermo_half(flr_ctx *ctx, double *sc, const double *ke_in, double gkT, double Q, double dt, double *totals,
                       cudaStream_t st)
{
    k_thermo_half<<<1, 1, 0, st>>>(sc, ke_in, gkT, Q, dt, totals);
    count_launch(ctx);
    return cuda_fail(cudaGetLastError(), "thermostat");
}

int launch_scale_vel(flr_ctx *ctx, float4 *vel, int n, const double *scale, cudaStream_t st)
{
    k_scale_vel<<<(n + 255) / 256, 256, 0, st>>>(vel, n, scale);
    count_launch(ctx);
    return cuda_fail(cudaGetLastError(), "thermostat velocity scaling");
}

int launch_count_above(flr_ctx *ctx, const float *sigma, int n, float thr, int *count, double *totals,
                       cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int), st);
    if (e != cudaSuccess) return cuda_fail(e, "uncertainty count");
    k_count_above<<<std::max(1, std::min((n + 255) / 256, ctx->num_sms * 4)), 256, 0, st>>>(sigma, n, thr, count);
    if (totals) k_store_count<<<1, 1, 0, st>>>(count, totals, FLR_TOT_N_UNCERTAIN);
    count_launch(ctx, totals ? 2 : 1);
    return cuda_fail(cudaGetLastError(), "uncertainty count");
}

int launch_cn_count(flr_ctx *ctx, const flr_nbrlist *nl, const int32_t *species, int n, int cs, float rc,
                    int *count, double *totals, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int), st);
    if (e != cudaSuccess) return cuda_fail(e, "coordination count");
    k_cn_count<<<std::max(1, std::min((n + 255) / 256, ctx->num_sms * 4)), 256, 0, st>>>(
        nl->group, nl->pair_cnt, nl->pair_rec, nl->max_nbr, species, n, cs, rc * rc, count);
    if (totals) k_store_count<<<1, 1, 0, st>>>(count, totals, FLR_TOT_N_CN);
    count_launch(ctx, totals ? 2 : 1);
    return cuda_fail(cudaGetLastError(), "coordination count");
}

int launch_set_rebuild(flr_ctx *ctx, flr_nbrlist *nl, cudaStream_t st)
{
    k_set_flag<<<1, 1, 0, st>>>(nl->flags);
    count_launch(ctx);
    return cuda_fail(cudaGetLastError(), "set rebuild flag");
}

int launch_clear_rebuild_counter(flr_ctx *ctx, flr_nbrlist *nl, cudaStream_t st)
{
    k_clear_counter<<<1, 1, 0, st>>>(nl->flags);
    count_launch(ctx);
    return cuda_fail(cudaGetLastError(), "clear rebuild counter");
}

int launch_copy_rebuilds(flr_ctx *ctx, flr_nbrlist *nl, double *totals, cudaStream_t st)
{
    k_copy_rebuilds<<<1, 1, 0, st>>>(nl->flags, totals);
    count_launch(ctx);
    return cuda_fail(cudaGetLastError(), "copy rebuild counter");
}

}  // namespace flr
