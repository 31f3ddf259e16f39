// C ABI of libflare_gb: context, model upload, workspace, entry points.
// See include/flare_gb.h for the contract of every exported function.
#include <algorithm>
#include <cstddef>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "internal.cuh"

namespace flr {

static thread_local std::string g_err;

void set_error(const std::string &msg) { g_err = msg; }

int cuda_fail(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return FLR_OK;
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? FLR_ENOMEM : FLR_ECUDA;
}

static cudaEvent_t prof_event(ProfState *p)
{
    if (p->n_pool > 0) return p->pool[--p->n_pool];
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void prof_begin(flr_ctx *ctx, int cls, cudaStream_t st)
{
    ProfState *p = ctx->prof;
    if (!p || !p->on) return;
    if (p->n_recs == p->cap) {
        int cap = p->cap ? 2 * p->cap : 1024;
        ProfState::Rec *r = new ProfState::Rec[cap];
        for (int k = 0; k < p->n_recs; ++k) r[k] = p->recs[k];
        delete[] p->recs;
        p->recs = r;
        p->cap = cap;
    }
    ProfState::Rec &r = p->recs[p->n_recs];
    r.a = prof_event(p);
    r.b = nullptr;
    r.cls = cls;
    cudaEventRecord(r.a, st);
}

void prof_end(flr_ctx *ctx, int cls, cudaStream_t st)
{
    ProfState *p = ctx->prof;
    if (!p || !p->on) return;
    ProfState::Rec &r = p->recs[p->n_recs];
    if (r.cls != cls) return;
    r.b = prof_event(p);
    cudaEventRecord(r.b, st);
    ++p->n_recs;
}

static void prof_drain(ProfState *p)
{
    for (int k = 0; k < p->n_recs; ++k) {
        ProfState::Rec &r = p->recs[k];
        float ms = 0.f;
        cudaEventSynchronize(r.b);
        cudaEventElapsedTime(&ms, r.a, r.b);
        p->ms[r.cls] += ms;
        p->count[r.cls] += 1;
        for (cudaEvent_t e : {r.a, r.b}) {
            if (p->n_pool == p->pool_cap) {
                int cap = p->pool_cap ? 2 * p->pool_cap : 2048;
                cudaEvent_t *q = new cudaEvent_t[cap];
                for (int i = 0; i < p->n_pool; ++i) q[i] = p->pool[i];
                delete[] p->pool;
                p->pool = q;
                p->pool_cap = cap;
            }
            p->pool[p->n_pool++] = e;
        }
    }
    p->n_recs = 0;
}

int launch_set_rebuild(flr_ctx *ctx, flr_nbrlist *nl, cudaStream_t st);
int launch_clear_rebuild_counter(flr_ctx *ctx, flr_nbrlist *nl, cudaStream_t st);
int launch_copy_rebuilds(flr_ctx *ctx, flr_nbrlist *nl, double *totals, cudaStream_t st);

namespace {

int round_up(int x, int m) { return (x + m - 1) / m * m; }

uint16_t f2bf(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7fffffffu) > 0x7f800000u) return 0x7fc0;
    u += 0x7fffu + ((u >> 16) & 1u);   // round to nearest even
    return (uint16_t)(u >> 16);
}
float bf2f(uint16_t h)
{
    uint32_t u = (uint32_t)h << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

int tri(int a, int b, int C) { return a * C - a * (a - 1) / 2 + (b - a); }

template <typename T>
int dev_alloc(T **p, size_t count, const char *what)
{
    *p = nullptr;
    if (count == 0) count = 1;
    return cuda_fail(cudaMalloc(reinterpret_cast<void **>(p), sizeof(T) * count), what);
}

void free_workspace(flr_ctx *ctx)
{
    cudaFree(ctx->A);
    cudaFree(ctx->norm);
    for (int r = 0; r < 2; ++r) {
        cudaFree(ctx->D32[r]);
        cudaFree(ctx->Dhi[r]);
        cudaFree(ctx->Dlo[r]);
        cudaFree(ctx->Dtf[r]);
        cudaFree(ctx->P[r]);
        ctx->Dtf[r] = nullptr;
        ctx->D32[r] = nullptr;
        ctx->Dhi[r] = ctx->Dlo[r] = nullptr;
        ctx->P[r] = nullptr;
        cudaFree(ctx->G[r]);
        ctx->G[r] = nullptr;
    }
    cudaFree(ctx->Facc);
    cudaFree(ctx->partials);
    cudaFree(ctx->vir_atom);
    ctx->vir_atom = nullptr;
    cudaFree(ctx->scratch_out);
    ctx->scratch_out = nullptr;
    cudaFree(ctx->ref_list);
    ctx->ref_list = nullptr;
    ctx->A = ctx->norm = nullptr;
    ctx->Facc = nullptr;
    ctx->partials = nullptr;
    ctx->ws_n = 0;
}

// Workspace for n atoms: A, norms, descriptor rows per region (FP32 and
// BF16 hi/lo), quadratic-form products, fixed-point force accumulators and
// reduction partials.  Grown (never shrunk) on demand; allocation happens
// before any kernel of the call is enqueued.
int ensure_workspace(flr_ctx *ctx, int n)
{
    if (n <= ctx->ws_n) return FLR_OK;
    cudaDeviceSynchronize();
    free_workspace(ctx);
    const Dims &D = ctx->dims;
    const size_t N = (size_t)std::max(n, 1);
    int s = FLR_OK;
    if (s == FLR_OK) s = dev_alloc(&ctx->A, N * D.nA, "workspace A");
    if (s == FLR_OK) s = dev_alloc(&ctx->norm, N, "workspace norm");
    for (int r = 0; r < 2 && s == FLR_OK; ++r) {
        s = dev_alloc(&ctx->D32[r], N * D.kp32[r], "workspace D32");
        if (s == FLR_OK) s = dev_alloc(&ctx->Dhi[r], N * D.kp64[r], "workspace Dhi");
        if (s == FLR_OK) s = dev_alloc(&ctx->Dlo[r], N * D.kp64[r], "workspace Dlo");
        if (s == FLR_OK) s = dev_alloc(&ctx->P[r], N * 2 * D.K[r], "workspace P");
        if (s == FLR_OK) s = dev_alloc(&ctx->G[r], N * D.K[r], "workspace G");
    }
    if (s == FLR_OK) s = dev_alloc(&ctx->Facc, N * 3, "workspace forces");
    if (s == FLR_OK) s = dev_alloc(&ctx->vir_atom, N * 9, "workspace virial");
    if (s == FLR_OK) s = dev_alloc(&ctx->scratch_out, N * 3, "workspace outputs");
    if (s == FLR_OK) s = dev_alloc(&ctx->ref_list, N, "workspace variance queue");
    if (s == FLR_OK) s = dev_alloc(&ctx->partials, (size_t)kMaxPartials * 13 + 16, "workspace partials");
    // descriptor rows are written up to K only: their padding columns stay zero from here on
    for (int r = 0; r < 2 && s == FLR_OK; ++r) {
        s = cuda_fail(cudaMemset(ctx->D32[r], 0, sizeof(float) * N * D.kp32[r]), "workspace D32");
        if (s == FLR_OK) s = cuda_fail(cudaMemset(ctx->Dhi[r], 0, sizeof(__nv_bfloat16) * N * D.kp64[r]), "workspace Dhi");
        if (s == FLR_OK) s = cuda_fail(cudaMemset(ctx->Dlo[r], 0, sizeof(__nv_bfloat16) * N * D.kp64[r]), "workspace Dlo");
    }
    if (s == FLR_OK) s = cuda_fail(cudaDeviceSynchronize(), "workspace");
    if (s != FLR_OK) {
        free_workspace(ctx);
        return s;
    }
    ctx->ws_n = (int)N;
    return FLR_OK;
}

int check_system(const flr_ctx *ctx, const flr_nbrlist *nl, const flr_system *sys)
{
    if (!sys || !nl) {
        set_error("null system or neighbour list");
        return FLR_EINVAL;
    }
    if (nl->ctx != ctx) {
        set_error("neighbour list belongs to another context");
        return FLR_EINVAL;
    }
    if (sys->n_atoms < 0 || sys->n_atoms > nl->n_cap) {
        set_error("n_atoms out of range for this neighbour list");
        return FLR_EINVAL;
    }
    if (sys->n_atoms > 0 && (!sys->pos || !sys->species)) {
        set_error("null pos or species");
        return FLR_EINVAL;
    }
    if (reinterpret_cast<uintptr_t>(sys->pos) % 16) {
        set_error("pos must be 16-byte aligned float[n][4]");
        return FLR_EINVAL;
    }
    return FLR_OK;
}

int check_model(const flr_ctx *ctx)
{
    for (int s = 0; s < ctx->p.n_species; ++s)
        if (!ctx->model_set[s]) {
            set_error("flr_set_model has not been called for species " + std::to_string(s));
            return FLR_ENOMODEL;
        }
    return FLR_OK;
}

int status_to_code(int st)
{
    if (st & kErrTimeout) {
        set_error("a device-side wait timed out (results invalid)");
        return FLR_ETIMEOUT;
    }
    if (st & kErrOverflow) {
        set_error("neighbour list overflow: an atom has more than max_nbr neighbours");
        return FLR_ENBR_OVERFLOW;
    }
    if (st & kErrShift) {
        set_error("image shift out of range (positions far outside the cell, or cell too narrow)");
        return FLR_EDEVICE;
    }
    if (st & kErrNonFinite) {
        set_error("non-finite or overflowing force");
        return FLR_EDEVICE;
    }
    if (st & kErrSpecies) {
        set_error("species index out of range");
        return FLR_EINVAL;
    }
    return FLR_OK;
}

// The quadratic forms of every compaction group at the context's precision
// (the forward and the backward pass use the same kernels, so the forces of
// the weighted energy with unit weights are bitwise the forward forces).
int launch_qform(flr_ctx *ctx, const flr_nbrlist *nl, flr_outputs *out, cudaStream_t st)
{
    if (ctx->p.precision == FLR_PREC_FP32) return launch_qform_simt(ctx, nl, out, st);
    if (ctx->p.precision == FLR_PREC_BF16X3 && ctx->p.compaction) {
        // two-species tiles on the general kernel, one-species tiles on the
        // kernel with the resident A tile.  With the overlap option the second
        // starts as a programmatic dependent of the first, on the SMs its few
        // tiles leave free (its tile counter is cleared before both, so no
        // stream operation sits between the two launches)
        const cudaError_t e = cudaMemsetAsync(ctx->sched + 4, 0, sizeof(int), st);
        if (e != cudaSuccess) return cuda_fail(e, "quadratic-form tile counter");
        int s = launch_qform_tc(ctx, nl, out, st, true);
        if (s == FLR_OK) s = launch_qform1(ctx, nl, out, st, ctx->overlap != 0);
        return s;
    }
    return launch_qform_tc(ctx, nl, out, st);
}

// Outputs are written from the quadratic forms on: with a host read-back of
// the previous results still in flight (flr_md_step_host), wait for it here,
// after the descriptor kernel has already run beside it.
int gate_outputs(flr_ctx *ctx, cudaStream_t st)
{
    if (!ctx->out_gate) return FLR_OK;
    return cuda_fail(cudaStreamWaitEvent(st, ctx->out_gate, 0), "wait for the host read-back");
}

int evaluate(flr_ctx *ctx, const flr_nbrlist *nl, const float4 *pos, const int *species, int n,
             flr_outputs *out, const KickArgs &kick, cudaStream_t st, double *seg_totals = nullptr)
{
    if (n == 0) return FLR_OK;
    cudaError_t e = cudaMemsetAsync(ctx->Facc, 0, sizeof(long long) * 3 * (size_t)n, st);
    if (e != cudaSuccess) return cuda_fail(e, "clear force accumulators");
    int s = FLR_OK;
    if (fused_eligible(ctx)) {
        // two-species atoms: descriptor rows and tensor-core tiles as below;
        // one-species atoms: the fused kernel.  Atoms without neighbours keep
        // ||B|| = 0 from this clear.
        e = cudaMemsetAsync(ctx->norm, 0, sizeof(float) * (size_t)n, st);
        if (e == cudaSuccess && ctx->var_mode == FLR_VAR_AUTO) e = cudaMemsetAsync(ctx->ref_count, 0, sizeof(int), st);
        if (e != cudaSuccess) return cuda_fail(e, "clear norms");
        const int *cnt = reinterpret_cast<const int *>(reinterpret_cast<const char *>(nl->gtab) + offsetof(GroupTab, count));
        prof_begin(ctx, FLR_KERNEL_DESCRIPTOR, st);
        s = launch_desc(ctx, nl, pos, species, n, st, nl->atom_of_row, cnt + 0, cnt + 3);
        prof_end(ctx, FLR_KERNEL_DESCRIPTOR, st);
        if (s == FLR_OK) s = gate_outputs(ctx, st);
        prof_begin(ctx, FLR_KERNEL_QFORM, st);
        if (s == FLR_OK) s = launch_qform_tc(ctx, nl, out, st, true);
        prof_end(ctx, FLR_KERNEL_QFORM, st);
        prof_begin(ctx, FLR_KERNEL_FUSED, st);
        if (s == FLR_OK) s = launch_fused(ctx, nl, pos, species, n, out, st);
        prof_end(ctx, FLR_KERNEL_FUSED, st);
        if (s == FLR_OK && ctx->var_mode == FLR_VAR_AUTO) {
            // the FP64 variance reads FP32 descriptor rows: write them for the queued atoms
            prof_begin(ctx, FLR_KERNEL_QFORM, st);
            s = launch_desc(ctx, nl, pos, species, ctx->ws_n, st, ctx->ref_list, ctx->ref_count);
            if (s == FLR_OK) s = launch_variance_fp64(ctx, nl, out, st);
            prof_end(ctx, FLR_KERNEL_QFORM, st);
        }
        if (s != FLR_OK) return s;
    } else {
        // with 3xBF16 and compaction the one-species quadratic forms read only
        // the BF16 rows, so their FP32 rows are not written here
        const bool skip32 = ctx->p.precision == FLR_PREC_BF16X3 && ctx->p.compaction;
        prof_begin(ctx, FLR_KERNEL_DESCRIPTOR, st);
        s = launch_desc(ctx, nl, pos, species, n, st, nullptr, nullptr, nullptr, skip32);
        prof_end(ctx, FLR_KERNEL_DESCRIPTOR, st);
        if (s == FLR_OK) s = gate_outputs(ctx, st);
        if (s != FLR_OK) return s;
        prof_begin(ctx, FLR_KERNEL_QFORM, st);
        if (ctx->var_mode == FLR_VAR_AUTO) {
            e = cudaMemsetAsync(ctx->ref_count, 0, sizeof(int), st);
            if (e != cudaSuccess) return cuda_fail(e, "clear variance queue");
        }
        s = launch_qform(ctx, nl, out, st);
        if (s == FLR_OK && ctx->var_mode == FLR_VAR_AUTO) {
            // the FP64 variance reads FP32 descriptor rows: write them for the queued atoms
            if (skip32) s = launch_desc(ctx, nl, pos, species, ctx->ws_n, st, ctx->ref_list, ctx->ref_count);
            if (s == FLR_OK) s = launch_variance_fp64(ctx, nl, out, st);
        }
        prof_end(ctx, FLR_KERNEL_QFORM, st);
        if (s != FLR_OK) return s;
    }
    prof_begin(ctx, FLR_KERNEL_FORCE, st);
    s = launch_force(ctx, nl, pos, species, n, out, seg_totals ? ctx->vir_atom : nullptr, nullptr, st);
    prof_end(ctx, FLR_KERNEL_FORCE, st);
    if (s != FLR_OK) return s;
    prof_begin(ctx, FLR_KERNEL_FINALIZE, st);
    if (seg_totals) {
        // a batch: each structure gets its own totals
        flr_outputs o = *out;
        o.totals = nullptr;
        s = launch_finalize(ctx, nl, n, &o, kick, 1.f, st);
        if (s == FLR_OK) s = launch_seg_totals(ctx, nl, out, ctx->vir_atom, seg_totals, st);
    } else {
        s = launch_finalize(ctx, nl, n, out, kick, 1.f, st);
    }
    prof_end(ctx, FLR_KERNEL_FINALIZE, st);
    return s;
}

// Neighbour lists of a batch of structures (one structure for the
// single-system calls); synchronizes.
int build_batch(flr_ctx *c, flr_nbrlist *nl, int n_structs, const int32_t *offsets, const double *cells,
                const int32_t *pbc, const float4 *pos, const int32_t *species, int n, cudaStream_t st)
{
    nl->n = n;
    int s = plan_batch(c, nl, n_structs, offsets, cells, pbc, pos, n, st);
    if (s != FLR_OK || n == 0) return s;
    s = launch_set_rebuild(c, nl, st);
    if (s == FLR_OK) s = launch_rebuild(c, nl, pos, species, n, st, false, nullptr);
    if (s != FLR_OK) return s;
    s = cuda_fail(cudaStreamSynchronize(st), "neighbour build");
    if (s != FLR_OK) return s;
    int dst[4];
    GroupTab gt;
    s = cuda_fail(cudaMemcpy(dst, c->status, sizeof(dst), cudaMemcpyDeviceToHost), "status");
    if (s == FLR_OK) s = cuda_fail(cudaMemcpy(&gt, nl->gtab, sizeof(gt), cudaMemcpyDeviceToHost), "status");
    if (s != FLR_OK) return s;
    if (dst[0]) {
        cudaMemset(c->status, 0, 4 * sizeof(int));
        s = status_to_code(dst[0]);
        if (s == FLR_ENBR_OVERFLOW)
            set_error("neighbour list overflow: an atom has " + std::to_string(gt.max_count) +
                      " neighbours, max_nbr is " + std::to_string(nl->max_nbr));
        return s;
    }
    return FLR_OK;
}

int check_batch(const flr_ctx *ctx, const flr_nbrlist *nl, const flr_batch *b)
{
    if (!b || !nl || nl->ctx != ctx || b->n_structs < 1 || b->n_atoms < 0 || b->n_atoms > nl->n_cap || !b->offsets ||
        !b->cells || !b->pbc) {
        set_error("invalid batch (n_structs >= 1, n_atoms within the list capacity, host offsets/cells/pbc)");
        return FLR_EINVAL;
    }
    if (b->n_atoms > 0 && (!b->pos || !b->species || reinterpret_cast<uintptr_t>(b->pos) % 16)) {
        set_error("batch pos must be 16-byte aligned float[n][4]; species required");
        return FLR_EINVAL;
    }
    return FLR_OK;
}

}  // namespace

// Entry points of the serving loop (server.cu) into this file's helpers.
int srv_reserve_workspace(flr_ctx *ctx, int n) { return ensure_workspace(ctx, n); }

int srv_evaluate(flr_ctx *ctx, const flr_nbrlist *nl, const float4 *pos, const int *species, int n,
                 flr_outputs *out, double *seg_totals, cudaStream_t st)
{
    KickArgs none;
    std::memset(&none, 0, sizeof(none));
    return evaluate(ctx, nl, pos, species, n, out, none, st, seg_totals);
}

int srv_status_code(int st) { return status_to_code(st); }

int srv_check_model(const flr_ctx *ctx) { return check_model(ctx); }

// Device bytes per atom of one evaluation, in two parts: the context's
// workspace (ensure_workspace) and what each batch slot of the serving loop
// holds (a neighbour-list row and its per-atom tables, flr_nbrlist_create,
// and the I/O arrays: positions, species, E, F, V, sigma).
void bytes_per_atom_parts(const flr_ctx *ctx, int64_t *workspace, int64_t *slot)
{
    const Dims &D = ctx->dims;
    int64_t w = 4 * (int64_t)D.nA + 4;
    for (int r = 0; r < 2; ++r) w += 4 * (int64_t)D.kp32[r] + 2 * 2 * (int64_t)D.kp64[r] + 4 * 3 * (int64_t)D.K[r];
    w += 8 * 3 + 4 * 9 + 4 * 3 + 4;
    int64_t l = 4 * (int64_t)ctx->p.max_nbr + 4 * 8 + 16 + 16 + 1;
    l += 16 * (int64_t)ctx->p.max_nbr + 4;   // pair records
    l += 16 + 4 + 4 * 4;                      // I/O arrays
    *workspace = w;
    *slot = l;
}

}  // namespace flr

using namespace flr;

// Copy streams, events and device staging rows of flr_md_step_host.
constexpr int kHostChunks = 8;
struct HostIO {
    cudaStream_t up, down;
    cudaEvent_t ev_up;                  // this step's inputs are in the staging rows (up)
    cudaEvent_t ev_packed;              // positions or velocities are in the staging rows (compute stream)
    cudaEvent_t ev_down[2][kHostChunks];   // chunk c of the positions [0] / velocities [1] has reached the host (down)
    cudaEvent_t ev_read;                // the last read-back of a call has landed (down)
    cudaEvent_t ev_join;                // everything enqueued on down so far (flr_host_join)
    float *stage;                       // [2][cap][3] positions, then velocities
    int cap;
    int last_n;                         // atoms of the previous call (-1: no copies in flight yet)
};

namespace {
void free_hostio(flr_ctx *c);   // host-state MD buffers (below)
}

extern "C" {

const char *flr_last_error(void) { return g_err.c_str(); }

const char *flr_version(void) { return "flare_gb 0.1 (sm_103a)"; }

int flr_create(const flr_params *p, int device, flr_ctx **out)
{
    if (!p || !out) {
        set_error("flr_create: null argument");
        return FLR_EINVAL;
    }
    *out = nullptr;
    if (p->n_species != kSpecies || (p->n_max != 7 && p->n_max != 8) || p->l_max != kL) {
        set_error("flr_create: supported hyperparameters are n_species = 2, n_max in {7, 8}, l_max = 3");
        return FLR_EINVAL;
    }
    if (p->max_nbr < 32 || p->max_nbr > 512 || p->max_nbr % 32) {
        set_error("flr_create: max_nbr must be a multiple of 32 in [32, 512]");
        return FLR_EINVAL;
    }
    if (!(p->r_cut > 0.0) || !(p->skin >= 0.0) || p->precision < 0 || p->precision > 2) {
        set_error("flr_create: invalid r_cut, skin or precision");
        return FLR_EINVAL;
    }
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    flr_ctx *c = new flr_ctx();
    std::memset(static_cast<void *>(c), 0, sizeof(flr_ctx));
    c->use_fused = 0;   // the separate kernels are faster on GB300 so far
    c->overlap = 1;
    c->p = *p;
    c->device = device;
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    Dims &D = c->dims;
    D.N = p->n_max;
    D.C = kSpecies * D.N;
    D.nA = D.C * kNLM;
    D.d_full = D.C * (D.C + 1) / 2 * (kL + 1);
    D.d_single = D.N * (D.N + 1) / 2 * (kL + 1);
    D.K[0] = D.d_full;
    D.K[1] = D.d_single;
    for (int r = 0; r < 2; ++r) {
        D.kp32[r] = round_up(D.K[r], 32);
        D.kp64[r] = round_up(D.K[r], 64);
        D.nrows_pad[r] = round_up(2 * D.K[r], 288);
    }
    int s = dev_alloc(&c->status, 4, "status word");
    if (s == FLR_OK) s = dev_alloc(&c->ref_count, 1, "variance queue counter");
    if (s == FLR_OK) s = dev_alloc(&c->sched, 8, "work counters");
    if (s == FLR_OK) s = dev_alloc(&c->md_sc, 8 + 256, "MD scalars");
    if (s == FLR_OK) s = dev_alloc(&c->md_totals, FLR_NTOTALS, "MD totals");
    if (s == FLR_OK) s = dev_alloc(&c->md_cnt, 2, "MD counters");
    if (s == FLR_OK) s = cuda_fail(cudaMemset(c->ref_count, 0, sizeof(int)), "variance queue counter");
    if (s == FLR_OK) s = cuda_fail(cudaMemset(c->status, 0, 4 * sizeof(int)), "status word");
    // index tables
    std::vector<int32_t> tf, ts;
    for (int a = 0; a < D.C; ++a)
        for (int b = a; b < D.C; ++b)
            for (int l = 0; l <= kL; ++l) tf.push_back(a | (b << 8) | (l << 16));
    for (int a = 0; a < D.N; ++a)
        for (int b = a; b < D.N; ++b)
            for (int l = 0; l <= kL; ++l) ts.push_back(a | (b << 8) | (l << 16));
    for (int t = 0; t < kSpecies; ++t)
        for (int a = 0; a < D.N; ++a)
            for (int b = a; b < D.N; ++b)
                for (int l = 0; l <= kL; ++l) ts.push_back(tri(t * D.N + a, t * D.N + b, D.C) * (kL + 1) + l);
    if (s == FLR_OK) s = dev_alloc(&c->tab_full, tf.size(), "tables");
    if (s == FLR_OK) s = dev_alloc(&c->tab_single, ts.size(), "tables");
    if (s == FLR_OK)
        s = cuda_fail(cudaMemcpy(c->tab_full, tf.data(), tf.size() * 4, cudaMemcpyHostToDevice), "tables");
    if (s == FLR_OK)
        s = cuda_fail(cudaMemcpy(c->tab_single, ts.data(), ts.size() * 4, cudaMemcpyHostToDevice), "tables");
    if (s != FLR_OK) {
        flr_destroy(c);
        return s;
    }
    *out = c;
    return FLR_OK;
}

int flr_destroy(flr_ctx *c)
{
    if (!c) return FLR_OK;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    free_workspace(c);
    for (int g = 0; g < kGroups; ++g) {
        cudaFree(c->W32[g]);
        cudaFree(c->Whi[g]);
        cudaFree(c->Wlo[g]);
        cudaFree(c->Wtf[g]);
        cudaFree(c->S64[g]);
    }
    for (int s = 0; s < kSpecies; ++s) {
        delete[] c->beta_h[s];
        delete[] c->sigma_h[s];
    }
    free_fused_maps(c);
    free_q1_maps(c);
    free_hostio(c);
    cudaFree(c->tab_full);
    cudaFree(c->tab_single);
    cudaFree(c->status);
    cudaFree(c->ref_count);
    cudaFree(c->sched);
    cudaFree(c->md_sc);
    cudaFree(c->md_totals);
    cudaFree(c->md_cnt);
    delete c->maps;
    if (c->prof) {
        prof_drain(c->prof);
        for (int k = 0; k < c->prof->n_pool; ++k) cudaEventDestroy(c->prof->pool[k]);
        delete[] c->prof->pool;
        delete[] c->prof->recs;
        delete c->prof;
    }
    delete c;
    return FLR_OK;
}

int flr_descriptor_dims(const flr_ctx *c, int32_t *d_full, int32_t *d_single)
{
    if (!c) return FLR_EINVAL;
    if (d_full) *d_full = c->dims.d_full;
    if (d_single) *d_single = c->dims.d_single;
    return FLR_OK;
}

int flr_set_precision(flr_ctx *c, int32_t precision)
{
    if (!c || precision < 0 || precision > 2) {
        set_error("flr_set_precision: invalid argument");
        return FLR_EINVAL;
    }
    c->p.precision = precision;
    return FLR_OK;
}

int flr_set_option(flr_ctx *c, int32_t option, int32_t value)
{
    if (!c || (option != FLR_OPT_FUSED_ONE_SPECIES && option != FLR_OPT_OVERLAP_TWO_SPECIES) ||
        (value != 0 && value != 1)) {
        set_error("flr_set_option: invalid option or value");
        return FLR_EINVAL;
    }
    if (option == FLR_OPT_FUSED_ONE_SPECIES)
        c->use_fused = value;
    else
        c->overlap = value;
    return FLR_OK;
}

}  // extern "C"

namespace flr {
namespace {

// Cholesky factor L (lower, row-major K x K) of a symmetric positive
// semi-definite matrix, in FP64.  On a non-positive pivot the diagonal is
// shifted by 1e-14, 1e-12, then 1e-10 of the trace and the factorization
// restarted; false if it still fails.  pivot_ratio = max pivot / min pivot
// (pivots lie inside the spectrum, so this bounds the condition number from
// below).
bool cholesky(const std::vector<double> &S, int K, std::vector<double> &L, double &pivot_ratio)
{
    double tr = 0.0;
    for (int i = 0; i < K; ++i) tr += S[(size_t)i * K + i];
    for (double rel : {0.0, 1e-14, 1e-12, 1e-10}) {
        const double tau = rel * tr;
        L.assign((size_t)K * K, 0.0);
        bool ok = true;
        double pmin = 1e300, pmax = 0.0;
        for (int j = 0; j < K && ok; ++j) {
            double s = S[(size_t)j * K + j] + tau;
            for (int k = 0; k < j; ++k) s -= L[(size_t)j * K + k] * L[(size_t)j * K + k];
            if (!(s > 0.0)) {
                ok = false;
                break;
            }
            const double ljj = std::sqrt(s);
            L[(size_t)j * K + j] = ljj;
            pmin = std::min(pmin, s);
            pmax = std::max(pmax, s);
            for (int i = j + 1; i < K; ++i) {
                double t = S[(size_t)i * K + j];
                for (int k = 0; k < j; ++k) t -= L[(size_t)i * K + k] * L[(size_t)j * K + k];
                L[(size_t)i * K + j] = t / ljj;
            }
        }
        if (ok) {
            pivot_ratio = pmax / pmin;
            return true;
        }
    }
    return false;
}

// Build and upload the B operands of one species' three compaction groups:
// rows [beta_c ; Sigma_c] (DIRECT) or [beta_c ; L_c^T] (FACTORED), restricted
// to the class block c, as FP32 and as BF16 hi / lo parts.
int upload_species(flr_ctx *c, int species)
{
    const Dims &D = c->dims;
    const int d = D.d_full;
    const double *bh = c->beta_h[species], *sh = c->sigma_h[species];
    std::vector<int> idx_full(d), idx_single[kSpecies];
    for (int k = 0; k < d; ++k) idx_full[k] = k;
    for (int t = 0; t < kSpecies; ++t)
        for (int a = 0; a < D.N; ++a)
            for (int b = a; b < D.N; ++b)
                for (int l = 0; l <= kL; ++l) idx_single[t].push_back(tri(t * D.N + a, t * D.N + b, D.C) * (kL + 1) + l);
    for (int cls = 0; cls < 3; ++cls) {
        const int g = species * 3 + cls, r = group_region(g);
        const std::vector<int> &idx = cls == 0 ? idx_full : idx_single[cls - 1];
        const int K = D.K[r], rows = D.nrows_pad[r];
        // the class block of Sigma and, when needed, its Cholesky factor
        bool factored = c->var_mode == FLR_VAR_FACTORED;
        std::vector<double> Lf;
        if (c->var_mode != FLR_VAR_DIRECT) {
            std::vector<double> Sc((size_t)K * K);
            for (int i = 0; i < K; ++i)
                for (int k = 0; k < K; ++k) Sc[(size_t)i * K + k] = sh[(size_t)idx[i] * d + idx[k]];
            double ratio = 0.0;
            if (!cholesky(Sc, K, Lf, ratio)) {
                set_error("flr_set_model: Sigma of species " + std::to_string(species) +
                          " is not positive semi-definite (Cholesky factorization failed)");
                return FLR_EINVAL;
            }
            (void)ratio;
        }
        c->var_factored[g] = factored ? 1 : 0;
        {
            // FP64 copy of the class block of Sigma for the FP64 variance
            std::vector<double> S64((size_t)K * K);
            for (int i = 0; i < K; ++i)
                for (int k = 0; k < K; ++k) S64[(size_t)i * K + k] = sh[(size_t)idx[i] * d + idx[k]];
            int s = FLR_OK;
            if (!c->S64[g]) s = dev_alloc(&c->S64[g], S64.size(), "model");
            if (s == FLR_OK)
                s = cuda_fail(cudaMemcpy(c->S64[g], S64.data(), S64.size() * 8, cudaMemcpyHostToDevice), "model upload");
            if (s != FLR_OK) return s;
            // largest eigenvalue of the block by power iteration (PSD: |Sigma|_2)
            std::vector<double> x(K, 1.0), y(K);
            double lam = 0.0;
            for (int it = 0; it < 40; ++it) {
                double ny = 0.0;
                for (int i = 0; i < K; ++i) {
                    double t = 0.0;
                    for (int k = 0; k < K; ++k) t += S64[(size_t)i * K + k] * x[k];
                    y[i] = t;
                    ny += t * t;
                }
                ny = std::sqrt(ny);
                double nx = 0.0;
                for (int i = 0; i < K; ++i) nx += x[i] * x[i];
                lam = ny / std::sqrt(nx);
                if (!(ny > 0.0)) break;
                for (int i = 0; i < K; ++i) x[i] = y[i] / ny;
            }
            c->sigma_norm[g] = (float)lam;
        }
        std::vector<float> w32((size_t)rows * D.kp32[r], 0.f), wtf((size_t)rows * D.kp32[r], 0.f);
        std::vector<uint16_t> whi((size_t)rows * D.kp64[r], 0), wlo((size_t)rows * D.kp64[r], 0);
        for (int n = 0; n < 2 * K; ++n) {
            for (int k = 0; k < K; ++k) {
                double v;
                if (n < K) v = bh[(size_t)idx[n] * d + idx[k]];
                else if (!factored) v = sh[(size_t)idx[n - K] * d + idx[k]];
                else v = Lf[(size_t)k * K + (n - K)];   // row n-K of L^T
                const float v32 = (float)v;
                w32[(size_t)n * D.kp32[r] + k] = v32;
                uint32_t u;
                std::memcpy(&u, &v32, 4);
                u = tf32_round_bits(u);
                std::memcpy(&wtf[(size_t)n * D.kp32[r] + k], &u, 4);
                const uint16_t h = f2bf((float)v);
                whi[(size_t)n * D.kp64[r] + k] = h;
                wlo[(size_t)n * D.kp64[r] + k] = f2bf((float)(v - (double)bf2f(h)));
            }
        }
        int s = FLR_OK;
        if (!c->W32[g]) {
            s = dev_alloc(&c->W32[g], w32.size(), "model");
            if (s == FLR_OK) s = dev_alloc(&c->Whi[g], whi.size(), "model");
            if (s == FLR_OK) s = dev_alloc(&c->Wlo[g], wlo.size(), "model");
            if (s == FLR_OK) s = dev_alloc(&c->Wtf[g], wtf.size(), "model");
            if (s != FLR_OK) return s;
        }
        s = cuda_fail(cudaMemcpy(c->W32[g], w32.data(), w32.size() * 4, cudaMemcpyHostToDevice), "model upload");
        if (s == FLR_OK)
            s = cuda_fail(cudaMemcpy(c->Wtf[g], wtf.data(), wtf.size() * 4, cudaMemcpyHostToDevice), "model upload");
        if (s == FLR_OK)
            s = cuda_fail(cudaMemcpy(c->Whi[g], whi.data(), whi.size() * 2, cudaMemcpyHostToDevice), "model upload");
        if (s == FLR_OK)
            s = cuda_fail(cudaMemcpy(c->Wlo[g], wlo.data(), wlo.size() * 2, cudaMemcpyHostToDevice), "model upload");
        if (s != FLR_OK) return s;
    }
    return FLR_OK;
}

}  // namespace
}  // namespace flr

extern "C" {

int flr_set_model(flr_ctx *c, int32_t species, const double *beta, const double *sigma)
{
    if (!c || !beta || !sigma || species < 0 || species >= kSpecies) {
        set_error("flr_set_model: invalid argument");
        return FLR_EINVAL;
    }
    cudaSetDevice(c->device);
    const int d = c->dims.d_full;
    double *bh = new double[(size_t)d * d], *sh = new double[(size_t)d * d];
    for (int r = 0; r < d; ++r)
        for (int q = 0; q < d; ++q) {
            bh[(size_t)r * d + q] = 0.5 * (beta[(size_t)r * d + q] + beta[(size_t)q * d + r]);
            sh[(size_t)r * d + q] = 0.5 * (sigma[(size_t)r * d + q] + sigma[(size_t)q * d + r]);
        }
    delete[] c->beta_h[species];
    delete[] c->sigma_h[species];
    c->beta_h[species] = bh;
    c->sigma_h[species] = sh;
    c->model_set[species] = false;
    const int s = upload_species(c, species);
    if (s != FLR_OK) return s;
    c->model_set[species] = true;
    c->maps_n = -1;   // B maps point at the (possibly new) buffers
    return FLR_OK;
}

int flr_set_variance_mode(flr_ctx *c, int32_t mode)
{
    if (!c || mode < FLR_VAR_AUTO || mode > FLR_VAR_FACTORED) {
        set_error("flr_set_variance_mode: invalid argument");
        return FLR_EINVAL;
    }
    cudaSetDevice(c->device);
    c->var_mode = mode;
    for (int sp = 0; sp < kSpecies; ++sp)
        if (c->model_set[sp]) {
            const int s = upload_species(c, sp);
            if (s != FLR_OK) {
                c->model_set[sp] = false;
                return s;
            }
        }
    c->maps_n = -1;
    return FLR_OK;
}

int flr_nbrlist_create(flr_ctx *c, int32_t n_atoms, flr_nbrlist **out)
{
    if (!c || !out || n_atoms < 0 || n_atoms >= (1 << 24)) {
        set_error("flr_nbrlist_create: invalid argument (n_atoms must be < 2^24)");
        return FLR_EINVAL;
    }
    cudaSetDevice(c->device);
    flr_nbrlist *nl = new flr_nbrlist();
    std::memset(static_cast<void *>(nl), 0, sizeof(flr_nbrlist));
    nl->ctx = c;
    nl->n_cap = n_atoms;
    nl->max_nbr = c->p.max_nbr;
    nl->status = c->status;
    nl->sched = c->sched + 2;
    const size_t N = (size_t)std::max(n_atoms, 1);
    int s = dev_alloc(&nl->entries, N * nl->max_nbr, "nbrlist");
    if (s == FLR_OK) s = dev_alloc(&nl->count, N, "nbrlist");
    if (s == FLR_OK) s = dev_alloc(&nl->group, N, "nbrlist");
    if (s == FLR_OK) s = dev_alloc(&nl->row, N, "nbrlist");
    if (s == FLR_OK) s = dev_alloc(&nl->atom_of_row, 2 * N, "nbrlist");
    if (s == FLR_OK) s = dev_alloc(&nl->pos_ref, N, "nbrlist");
    if (s == FLR_OK) s = dev_alloc(&nl->img, N, "nbrlist");
    if (s == FLR_OK) s = dev_alloc(&nl->atom_bin, N, "nbrlist");
    if (s == FLR_OK) s = dev_alloc(&nl->bin_atoms, N, "nbrlist");
    if (s == FLR_OK) s = dev_alloc(&nl->pos_bin, N, "nbrlist");
    if (s == FLR_OK) s = dev_alloc(&nl->blk_group, 8 * ((N + 511) / 512 + 1) + 65536 + 1024, "nbrlist");
    if (s == FLR_OK) s = dev_alloc(&nl->gtab, 1, "nbrlist");
    if (s == FLR_OK) s = dev_alloc(&nl->flags, 4, "nbrlist");
    if (s == FLR_OK) s = dev_alloc(&nl->struct_of, N, "nbrlist");
    if (s == FLR_OK) s = dev_alloc(&nl->pair_rec, N * nl->max_nbr, "nbrlist pair records");
    if (s == FLR_OK) s = dev_alloc(&nl->pair_cnt, N, "nbrlist pair records");
    if (s == FLR_OK) s = cuda_fail(cudaMemset(nl->gtab, 0, sizeof(GroupTab)), "nbrlist");
    if (s == FLR_OK) s = cuda_fail(cudaMemset(nl->flags, 0, 4 * sizeof(int32_t)), "nbrlist");
    if (s == FLR_OK) s = cuda_fail(cudaMemset(nl->group, 0xff, N * sizeof(int32_t)), "nbrlist");
    if (s != FLR_OK) {
        flr_nbrlist_destroy(nl);
        return s;
    }
    *out = nl;
    return FLR_OK;
}

int flr_nbrlist_destroy(flr_nbrlist *nl)
{
    if (!nl) return FLR_OK;
    cudaSetDevice(nl->ctx->device);
    cudaDeviceSynchronize();
    free_rebuild_graph(nl);
    cudaFree(nl->entries);
    cudaFree(nl->count);
    cudaFree(nl->group);
    cudaFree(nl->row);
    cudaFree(nl->atom_of_row);
    cudaFree(nl->pos_ref);
    cudaFree(nl->img);
    cudaFree(nl->atom_bin);
    cudaFree(nl->bin_atoms);
    cudaFree(nl->pos_bin);
    cudaFree(nl->bin_start);
    cudaFree(nl->bin_fill);
    cudaFree(nl->blk_group);
    cudaFree(nl->gtab);
    cudaFree(nl->flags);
    cudaFree(nl->bbox);
    cudaFree(nl->struct_of);
    cudaFree(nl->pair_rec);
    cudaFree(nl->pair_cnt);
    cudaFree(nl->offsets_d);
    cudaFree(nl->shift_d);
    cudaFree(nl->plans_d);
    delete[] nl->plans_h;
    delete[] nl->offsets_h;
    delete nl;
    return FLR_OK;
}

int flr_nbrlist_view(const flr_nbrlist *nl, int32_t **entries, int32_t **count, int32_t **group, int32_t *max_nbr)
{
    if (!nl) return FLR_EINVAL;
    if (entries) *entries = nl->entries;
    if (count) *count = nl->count;
    if (group) *group = nl->group;
    if (max_nbr) *max_nbr = nl->max_nbr;
    return FLR_OK;
}

int flr_build_neighbors(flr_ctx *c, const flr_system *sys, flr_nbrlist *nl, flr_stream_t stream)
{
    if (!c) return FLR_EINVAL;
    int s = check_system(c, nl, sys);
    if (s != FLR_OK) return s;
    cudaSetDevice(c->device);
    const int32_t offsets[2] = {0, sys->n_atoms};
    return build_batch(c, nl, 1, offsets, sys->cell, sys->pbc, reinterpret_cast<const float4 *>(sys->pos),
                       sys->species, sys->n_atoms, reinterpret_cast<cudaStream_t>(stream));
}

int flr_build_neighbors_batch(flr_ctx *c, const flr_batch *b, flr_nbrlist *nl, flr_stream_t stream)
{
    if (!c) return FLR_EINVAL;
    int s = check_batch(c, nl, b);
    if (s != FLR_OK) return s;
    cudaSetDevice(c->device);
    return build_batch(c, nl, b->n_structs, b->offsets, b->cells, b->pbc, reinterpret_cast<const float4 *>(b->pos),
                       b->species, b->n_atoms, reinterpret_cast<cudaStream_t>(stream));
}

int flr_energy_forces_uncertainty_batch(flr_ctx *c, const flr_batch *b, const flr_nbrlist *nl, flr_outputs *out,
                                        flr_stream_t stream)
{
    if (!c || !out) return FLR_EINVAL;
    int s = check_batch(c, nl, b);
    if (s == FLR_OK) s = check_model(c);
    if (s != FLR_OK) return s;
    if (b->n_atoms != nl->n || b->n_structs != nl->n_structs) {
        set_error("batch differs from the neighbour list's last build");
        return FLR_EINVAL;
    }
    if (b->n_atoms > 0 && (!out->forces || !out->energy)) {
        set_error("flr_energy_forces_uncertainty_batch: energy and forces are required");
        return FLR_EINVAL;
    }
    cudaSetDevice(c->device);
    s = ensure_workspace(c, b->n_atoms);
    if (s != FLR_OK) return s;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (b->n_atoms == 0) {
        if (out->totals)
            return cuda_fail(cudaMemsetAsync(out->totals, 0, sizeof(double) * FLR_NTOTALS * b->n_structs, st), "totals");
        return FLR_OK;
    }
    KickArgs kick;
    std::memset(&kick, 0, sizeof(kick));
    if (!out->totals) return evaluate(c, nl, reinterpret_cast<const float4 *>(b->pos), b->species, b->n_atoms, out, kick, st);
    return evaluate(c, nl, reinterpret_cast<const float4 *>(b->pos), b->species, b->n_atoms, out, kick, st, out->totals);
}

int flr_energy_backward(flr_ctx *c, const flr_batch *b, const flr_nbrlist *nl, const float *grad_energy,
                        float *grad_pos, float *grad_beta, flr_stream_t stream)
{
    if (!c) return FLR_EINVAL;
    int s = check_batch(c, nl, b);
    if (s == FLR_OK) s = check_model(c);
    if (s != FLR_OK) return s;
    if (b->n_atoms != nl->n || b->n_structs != nl->n_structs) {
        set_error("batch differs from the neighbour list's last build");
        return FLR_EINVAL;
    }
    if (b->n_atoms > 0 && (!grad_energy || !grad_pos)) {
        set_error("flr_energy_backward: grad_energy and grad_pos are required");
        return FLR_EINVAL;
    }
    cudaSetDevice(c->device);
    s = ensure_workspace(c, b->n_atoms);
    if (s != FLR_OK) return s;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int n = b->n_atoms;
    if (n == 0) {
        if (grad_beta)
            return cuda_fail(cudaMemsetAsync(grad_beta, 0,
                                             sizeof(float) * (size_t)kSpecies * c->dims.d_full * c->dims.d_full, st),
                             "clear dL/dbeta");
        return FLR_OK;
    }
    const float4 *pos = reinterpret_cast<const float4 *>(b->pos);
    // recompute the forward intermediates (descriptors, g); nothing is kept from the forward call
    flr_outputs o;
    o.energy = c->scratch_out;
    o.variance = c->scratch_out + n;
    o.sigma = c->scratch_out + 2 * (size_t)n;
    o.forces = grad_pos;
    o.totals = nullptr;
    s = cuda_fail(cudaMemsetAsync(c->Facc, 0, sizeof(long long) * 3 * (size_t)n, st), "clear force accumulators");
    if (s == FLR_OK) s = launch_desc(c, nl, pos, b->species, n, st);
    if (s == FLR_OK)
        s = launch_qform(c, nl, &o, st);
    // dL/dr = -(forces of sum_i u_i E_i): the force kernel with g_i scaled by u_i
    if (s == FLR_OK) s = launch_force(c, nl, pos, b->species, n, &o, nullptr, grad_energy, st);
    KickArgs none;
    std::memset(&none, 0, sizeof(none));
    if (s == FLR_OK) s = launch_finalize(c, nl, n, &o, none, -1.f, st);
    if (s == FLR_OK && grad_beta) s = launch_dbeta(c, nl, grad_energy, grad_beta, st);
    return s;
}

int flr_compute_descriptors(flr_ctx *c, const flr_system *sys, const flr_nbrlist *nl, float *d_hat, float *norm,
                            flr_stream_t stream)
{
    if (!c || !d_hat) {
        set_error("flr_compute_descriptors: null argument");
        return FLR_EINVAL;
    }
    int s = check_system(c, nl, sys);
    if (s != FLR_OK) return s;
    if (sys->n_atoms != nl->n) {
        set_error("system size differs from the neighbour list's last build");
        return FLR_EINVAL;
    }
    cudaSetDevice(c->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    s = ensure_workspace(c, sys->n_atoms);
    if (s != FLR_OK || sys->n_atoms == 0) return s;
    s = launch_desc(c, nl, reinterpret_cast<const float4 *>(sys->pos), sys->species, sys->n_atoms, st);
    if (s != FLR_OK) return s;
    return launch_expand_desc(c, nl, sys->n_atoms, d_hat, norm, st);
}

int flr_energy_forces_uncertainty(flr_ctx *c, const flr_system *sys, const flr_nbrlist *nl, flr_outputs *out,
                                  flr_stream_t stream)
{
    if (!c || !out || (sys && sys->n_atoms > 0 && (!out->forces || !out->energy))) {
        set_error("flr_energy_forces_uncertainty: null argument (energy and forces are required)");
        return FLR_EINVAL;
    }
    int s = check_system(c, nl, sys);
    if (s == FLR_OK) s = check_model(c);
    if (s != FLR_OK) return s;
    if (sys->n_atoms != nl->n) {
        set_error("system size differs from the neighbour list's last build");
        return FLR_EINVAL;
    }
    cudaSetDevice(c->device);
    s = ensure_workspace(c, sys->n_atoms);
    if (s != FLR_OK) return s;
    KickArgs kick;
    std::memset(&kick, 0, sizeof(kick));
    if (sys->n_atoms == 0) {
        if (out->totals)
            return cuda_fail(cudaMemsetAsync(out->totals, 0, sizeof(double) * FLR_NTOTALS,
                                             reinterpret_cast<cudaStream_t>(stream)),
                             "totals");
        return FLR_OK;
    }
    return evaluate(c, nl, reinterpret_cast<const float4 *>(sys->pos), sys->species, sys->n_atoms, out, kick,
                    reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"

namespace {

// Copy streams, events and staging rows for n atoms (created on first use,
// the rows grown when too small; cudaFree waits for the copies in flight).
int ensure_hostio(flr_ctx *c, int n)
{
    if (!c->hio) {
        HostIO *io = new HostIO();
        std::memset(static_cast<void *>(io), 0, sizeof(HostIO));
        io->last_n = -1;
        c->hio = io;
        cudaError_t e = cudaStreamCreateWithFlags(&io->up, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&io->down, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&io->ev_up, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&io->ev_packed, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&io->ev_read, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&io->ev_join, cudaEventDisableTiming);
        for (int k = 0; k < 2 * kHostChunks && e == cudaSuccess; ++k)
            e = cudaEventCreateWithFlags(&io->ev_down[k / kHostChunks][k % kHostChunks], cudaEventDisableTiming);
        if (e != cudaSuccess) {
            const int r = cuda_fail(e, "host-state streams and events");
            free_hostio(c);   // nothing half-made stays behind for the next call
            return r;
        }
    }
    HostIO *io = c->hio;
    if (io->cap < n) {
        cudaFree(io->stage);
        io->stage = nullptr;
        io->cap = 0;
        io->last_n = -1;   // the copies of earlier calls have landed
        const cudaError_t e = cudaMalloc(&io->stage, sizeof(float) * 6 * (size_t)n);
        if (e != cudaSuccess) return cuda_fail(e, "host-state staging rows");
        io->cap = n;
    }
    return FLR_OK;
}

void free_hostio(flr_ctx *c)
{
    HostIO *io = c->hio;
    if (!io) return;
    if (io->up) cudaStreamSynchronize(io->up);
    if (io->down) cudaStreamSynchronize(io->down);
    cudaFree(io->stage);
    if (io->up) cudaStreamDestroy(io->up);
    if (io->down) cudaStreamDestroy(io->down);
    cudaEvent_t evs[4] = {io->ev_up, io->ev_packed, io->ev_read, io->ev_join};
    for (cudaEvent_t ev : evs)
        if (ev) cudaEventDestroy(ev);
    for (int k = 0; k < 2 * kHostChunks; ++k)
        if (io->ev_down[k / kHostChunks][k % kHostChunks]) cudaEventDestroy(io->ev_down[k / kHostChunks][k % kHostChunks]);
    delete io;
    c->hio = nullptr;
    c->out_gate = nullptr;
}

// Atoms [lo, hi) of chunk k of n.
inline void chunk_range(int n, int k, size_t &lo, size_t &hi)
{
    lo = (size_t)n * k / kHostChunks;
    hi = (size_t)n * (k + 1) / kHostChunks;
}

// Host state -> staging rows -> working copies on `st`.  Each chunk's
// upload waits only for the previous download of the same chunk, and all
// position chunks go before the velocity chunks: the positions of a step are
// final (and downloaded) once its drift and rebuild are done, so the next
// step's position uploads run while the step's kernels still do, and only
// the velocities' round trip remains between two steps.
int host_upload(flr_ctx *c, const flr_host_state *h, flr_md_state *md, cudaStream_t st)
{
    HostIO *io = c->hio;
    const int n = md->n_atoms;
    float *rows[2] = {io->stage, io->stage + 3 * (size_t)io->cap};
    const float *src[2] = {h->pos, h->vel};
    cudaError_t e = cudaSuccess;
    for (int q = 0; q < 2; ++q)
        for (int k = 0; k < kHostChunks && e == cudaSuccess; ++k) {
            size_t lo, hi;
            chunk_range(n, k, lo, hi);
            if (io->last_n >= 0)
                e = cudaStreamWaitEvent(io->up, io->ev_down[q][io->last_n == n ? k : kHostChunks - 1], 0);
            if (e == cudaSuccess && hi > lo)
                e = cudaMemcpyAsync(rows[q] + 3 * lo, src[q] + 3 * lo, 12 * (hi - lo), cudaMemcpyHostToDevice, io->up);
        }
    if (e == cudaSuccess) e = cudaEventRecord(io->ev_up, io->up);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, io->ev_up, 0);
    if (e != cudaSuccess) return cuda_fail(e, "upload host state");
    return launch_state_unpack(c, rows[0], rows[1], reinterpret_cast<float4 *>(md->pos),
                               reinterpret_cast<float4 *>(md->vel), n, st);
}

// Positions (q = 0) or velocities (q = 1) of the working copies -> staging
// rows on `st` -> host, in chunks on the download stream.
int host_download(flr_ctx *c, const flr_host_state *h, flr_md_state *md, int q, cudaStream_t st)
{
    HostIO *io = c->hio;
    const int n = md->n_atoms;
    float *rows = io->stage + (q ? 3 * (size_t)io->cap : 0);
    float *dst = q ? h->vel : h->pos;
    int s = launch_state_pack(c, reinterpret_cast<const float4 *>(q ? md->vel : md->pos), rows, n, st);
    if (s != FLR_OK) return s;
    cudaError_t e = cudaEventRecord(io->ev_packed, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(io->down, io->ev_packed, 0);
    for (int k = 0; k < kHostChunks && e == cudaSuccess; ++k) {
        size_t lo, hi;
        chunk_range(n, k, lo, hi);
        if (hi > lo) e = cudaMemcpyAsync(dst + 3 * lo, rows + 3 * lo, 12 * (hi - lo), cudaMemcpyDeviceToHost, io->down);
        if (e == cudaSuccess) e = cudaEventRecord(io->ev_down[q][k], io->down);
    }
    if (e != cudaSuccess) return cuda_fail(e, "download host state");
    if (q == 1) io->last_n = n;
    return FLR_OK;
}

// The requested results of the call's last step, on the download stream
// after the state; the next call's outputs wait for ev_read.
int host_results(flr_ctx *c, const flr_host_state *h, const flr_outputs &o, int n, cudaStream_t st)
{
    HostIO *io = c->hio;
    cudaError_t e = cudaEventRecord(io->ev_packed, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(io->down, io->ev_packed, 0);
    struct {
        void *dst;
        const void *src;
        size_t bytes;
    } cp[5] = {{h->energy, o.energy, 4 * (size_t)n},
               {h->forces, o.forces, 12 * (size_t)n},
               {h->variance, o.variance, 4 * (size_t)n},
               {h->sigma, o.sigma, 4 * (size_t)n},
               {h->totals, o.totals, sizeof(double) * FLR_NTOTALS}};
    for (auto &x : cp)
        if (e == cudaSuccess && x.dst && x.src && x.bytes)
            e = cudaMemcpyAsync(x.dst, x.src, x.bytes, cudaMemcpyDeviceToHost, io->down);
    if (e == cudaSuccess) e = cudaEventRecord(io->ev_read, io->down);
    if (e != cudaSuccess) return cuda_fail(e, "read back results");
    c->out_gate = io->ev_read;   // stays set: later evaluations of this context wait for it
    return FLR_OK;
}

// n_steps of velocity Verlet (flr_md_step); with h, every step's state goes
// through the host arrays of h (flr_md_step_host).
int md_run(flr_ctx *c, flr_md_state *md, flr_nbrlist *nl, int32_t n_steps, flr_outputs *out, flr_stream_t stream,
           const flr_host_state *h)
{
    if (!c || !md || !nl || !out || !out->forces || !out->energy || n_steps < 0) {
        set_error("flr_md_step: invalid argument");
        return FLR_EINVAL;
    }
    int s = check_model(c);
    if (s != FLR_OK) return s;
    if (md->n_atoms != nl->n || !nl->planned || md->rebuild_every < 1 || !(md->dt > 0.0)) {
        set_error("flr_md_step: build the list with flr_build_neighbors first; rebuild_every >= 1, dt > 0");
        return FLR_EINVAL;
    }
    if (reinterpret_cast<uintptr_t>(md->pos) % 16 || reinterpret_cast<uintptr_t>(md->vel) % 16) {
        set_error("flr_md_step: pos and vel must be 16-byte aligned float[n][4]");
        return FLR_EINVAL;
    }
    const bool nvt = md->temperature > 0.0;
    const bool stop = md->sigma_stop > 0.0;
    const bool cn = md->cn_species >= 0;
    if (nvt && !(md->tau > 0.0)) {
        set_error("flr_md_step: the thermostat needs tau > 0");
        return FLR_EINVAL;
    }
    if (stop && !out->sigma) {
        set_error("flr_md_step: sigma_stop needs the sigma output");
        return FLR_EINVAL;
    }
    if (cn && (md->cn_species >= kSpecies || !(md->cn_cutoff > 0.0) || md->cn_cutoff > c->p.r_cut)) {
        set_error("flr_md_step: cn_species must be a species and 0 < cn_cutoff <= r_cut");
        return FLR_EINVAL;
    }
    md->halted = 0;
    cudaSetDevice(c->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int n = md->n_atoms;
    s = ensure_workspace(c, n);
    if (s == FLR_OK && h) s = ensure_hostio(c, n);
    if (s != FLR_OK || n == 0) return s;
    const double ftm2v = 1.0 / 1.0364269e-4;   // (eV/A)/amu -> A/ps^2
    const double kB = 8.617333262e-5;           // eV/K
    KickArgs kick;
    std::memset(&kick, 0, sizeof(kick));
    kick.vel = reinterpret_cast<float4 *>(md->vel);
    kick.species = md->species;
    for (int sp = 0; sp < kSpecies; ++sp) {
        if (!(md->masses[sp] > 0.0)) {
            set_error("flr_md_step: masses must be positive");
            return FLR_EINVAL;
        }
        kick.half_dt_over_m[sp] = (float)(0.5 * md->dt * ftm2v / md->masses[sp]);
        kick.half_m[sp] = (float)(0.5 * md->masses[sp] / ftm2v);
    }
    // the thermostat reads the kinetic energy from the totals: use the
    // context's own totals when the caller passes none
    flr_outputs o = *out;
    if (!o.totals) o.totals = c->md_totals;
    double *tot = o.totals;
    float4 *pos = reinterpret_cast<float4 *>(md->pos);
    const float skin = (float)c->p.skin;
    const float disp2 = 0.25f * skin * skin;
    const double gkT = 3.0 * n * kB * md->temperature;          // g kB T, g = 3n degrees of freedom
    const double Q = gkT * md->tau * md->tau;                     // thermostat mass (eV ps^2)
    s = launch_clear_rebuild_counter(c, nl, st);
    if (s == FLR_OK && h && n_steps > 0) s = host_upload(c, h, md, st);   // the first step's inputs
    if (s != FLR_OK) return s;
    if (!md->forces_valid) {
        KickArgs none;
        std::memset(&none, 0, sizeof(none));
        s = evaluate(c, nl, pos, md->species, n, &o, none, st);
        if (s != FLR_OK) return s;
        md->forces_valid = 1;
    }
    if (nvt) {
        const double init[2] = {md->xi, md->eta};
        s = cuda_fail(cudaMemcpyAsync(c->md_sc, init, sizeof(init), cudaMemcpyHostToDevice, st), "thermostat state");
        if (s == FLR_OK) s = launch_kinetic(c, kick.vel, md->species, n, md->masses, c->md_sc + 8, c->md_sc + 2, st);
        if (s != FLR_OK) return s;
        kick.scale = c->md_sc + 3;
    }
    kick.enabled = 1;
    for (int k = 0; k < n_steps; ++k) {
        if (h && k > 0) s = host_upload(c, h, md, st);
        if (s == FLR_OK && nvt) s = launch_thermo_half(c, c->md_sc, nullptr, gkT, Q, md->dt, nullptr, st);
        prof_begin(c, FLR_KERNEL_DRIFT, st);
        if (s == FLR_OK)
            s = launch_md_drift(c, nl, pos, kick.vel, o.forces, md->species, n, kick, (float)md->dt, disp2, st);
        prof_end(c, FLR_KERNEL_DRIFT, st);
        if (s == FLR_OK && (md->step + 1) % md->rebuild_every == 0) s = launch_set_rebuild(c, nl, st);
        prof_begin(c, FLR_KERNEL_REBUILD, st);
        if (s == FLR_OK) s = launch_rebuild_cond(c, nl, pos, md->species, n, st, true, pos);
        prof_end(c, FLR_KERNEL_REBUILD, st);
        // the step's positions are final here (drift, wrap at a rebuild)
        if (s == FLR_OK && h) s = host_download(c, h, md, 0, st);
        if (s == FLR_OK) s = evaluate(c, nl, pos, md->species, n, &o, kick, st);
        if (s == FLR_OK && nvt) {
            // second half step from the kinetic energy after the final kick
            s = launch_thermo_half(c, c->md_sc, tot + FLR_TOT_KINETIC, gkT, Q, md->dt, tot, st);
            if (s == FLR_OK) s = launch_scale_vel(c, kick.vel, n, c->md_sc + 3, st);
        }
        if (s == FLR_OK && cn)
            s = launch_cn_count(c, nl, md->species, n, md->cn_species, (float)md->cn_cutoff, c->md_cnt + 1, tot, st);
        if (s != FLR_OK) return s;
        md->step += 1;
        if (stop) {
            s = launch_count_above(c, o.sigma, n, (float)md->sigma_stop, c->md_cnt, tot, st);
            int cnt = 0;
            if (s == FLR_OK) s = cuda_fail(cudaMemcpyAsync(&cnt, c->md_cnt, sizeof(int), cudaMemcpyDeviceToHost, st),
                                           "uncertainty count");
            if (s == FLR_OK) s = cuda_fail(cudaStreamSynchronize(st), "uncertainty count");
            if (s != FLR_OK) return s;
            if (cnt > 0) md->halted = 1;
        }
        if (h) s = host_download(c, h, md, 1, st);
        if (s != FLR_OK) return s;
        if (md->halted) break;
    }
    s = launch_copy_rebuilds(c, nl, tot, st);
    if (s == FLR_OK && h && n_steps > 0) s = host_results(c, h, o, n, st);
    if (s == FLR_OK && nvt) {
        double fin[2];
        s = cuda_fail(cudaMemcpyAsync(fin, c->md_sc, sizeof(fin), cudaMemcpyDeviceToHost, st), "thermostat state");
        if (s == FLR_OK) s = cuda_fail(cudaStreamSynchronize(st), "thermostat state");
        if (s == FLR_OK) {
            md->xi = fin[0];
            md->eta = fin[1];
        }
    }
    return s;
}

}  // namespace

extern "C" {

int flr_md_step(flr_ctx *c, flr_md_state *md, flr_nbrlist *nl, int32_t n_steps, flr_outputs *out,
                flr_stream_t stream)
{
    return md_run(c, md, nl, n_steps, out, stream, nullptr);
}

int flr_md_step_host(flr_ctx *c, flr_md_state *md, flr_nbrlist *nl, int32_t n_steps, flr_outputs *out,
                     const flr_host_state *host, flr_stream_t stream)
{
    if (!host || !host->pos || !host->vel) {
        set_error("flr_md_step_host: host pos and vel are required");
        return FLR_EINVAL;
    }
    return md_run(c, md, nl, n_steps, out, stream, host);
}

int flr_host_join(flr_ctx *c, flr_stream_t stream)
{
    if (!c) return FLR_EINVAL;
    if (!c->hio || c->hio->last_n < 0) return FLR_OK;
    cudaSetDevice(c->device);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    // every upload is followed on the compute stream by its unpack, which the
    // caller's stream orders itself against; the down stream's work (state
    // downloads and read-backs) is waited for here
    cudaError_t e = cudaEventRecord(c->hio->ev_join, c->hio->down);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, c->hio->ev_join, 0);
    return cuda_fail(e, "flr_host_join");
}

int flr_sync(flr_ctx *c, flr_stream_t stream)
{
    if (!c) return FLR_EINVAL;
    cudaSetDevice(c->device);
    int s = cuda_fail(cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)), "flr_sync");
    if (s == FLR_OK && c->hio) s = cuda_fail(cudaStreamSynchronize(c->hio->up), "flr_sync (host uploads)");
    if (s == FLR_OK && c->hio) s = cuda_fail(cudaStreamSynchronize(c->hio->down), "flr_sync (host downloads)");
    if (s != FLR_OK) return s;
    int st[4];
    s = cuda_fail(cudaMemcpy(st, c->status, sizeof(st), cudaMemcpyDeviceToHost), "flr_sync status");
    if (s != FLR_OK) return s;
    if (st[0]) {
        cudaMemset(c->status, 0, sizeof(st));
        return status_to_code(st[0]);
    }
    return FLR_OK;
}

int64_t flr_launch_count(const flr_ctx *c) { return c ? c->launches : 0; }

int flr_profile_enable(flr_ctx *c, int32_t on)
{
    if (!c) return FLR_EINVAL;
    cudaSetDevice(c->device);
    if (!c->prof) {
        c->prof = new ProfState();
        std::memset(static_cast<void *>(c->prof), 0, sizeof(ProfState));
    }
    ProfState *p = c->prof;
    prof_drain(p);
    if (on) {
        for (int k = 0; k < FLR_KERNEL_CLASSES; ++k) {
            p->ms[k] = 0.0;
            p->count[k] = 0;
        }
    }
    p->on = on != 0;
    return FLR_OK;
}

int flr_profile_read(flr_ctx *c, int32_t cls, double *total_ms, int64_t *launches)
{
    if (!c || cls < 0 || cls >= FLR_KERNEL_CLASSES) {
        set_error("flr_profile_read: invalid argument");
        return FLR_EINVAL;
    }
    cudaSetDevice(c->device);
    if (!c->prof) {
        if (total_ms) *total_ms = 0.0;
        if (launches) *launches = 0;
        return FLR_OK;
    }
    prof_drain(c->prof);
    if (total_ms) *total_ms = c->prof->ms[cls];
    if (launches) *launches = c->prof->count[cls];
    return FLR_OK;
}

}  // extern "C"
