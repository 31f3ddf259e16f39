// Velocity-Verlet integration in metal units (Sec. VI-A: MD with the
// force field at every step).  The first half kick and the drift are fused
// here; the second half kick is fused into the force finalize kernel.  The
// drift kernel also checks every atom's displacement since the last
// neighbour build and raises the list's rebuild flag when one moved more
// than half the skin, so the rebuild decision never leaves the device.
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
};

__global__ void __launch_bounds__(256) k_md_drift(DriftArgs a)
{
    const int i = blockIdx.x * 256 + threadIdx.x;
    bool moved = false;
    if (i < a.n) {
        const int s = min(max(a.species[i], 0), kSpecies - 1);
        const float h = a.half_dt_over_m[s];
        float4 v = a.vel[i];
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
    k_md_drift<<<(n + 255) / 256, 256, 0, st>>>(a);
    count_launch(ctx);
    return cuda_fail(cudaGetLastError(), "md drift");
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
