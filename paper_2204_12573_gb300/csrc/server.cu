// Continuous-batching evaluation service (flr_server_*).
//
// One worker thread per server drives one CUDA stream.  Each turn of its
// loop: take queued requests in arrival order into a batch while the batch's
// device memory fits the budget, pack their inputs into a pinned arena and
// compute each structure's fractional bounding box on the host (so the bin
// grids are planned without a device round trip), then wait for the batch
// in flight, enqueue the new batch (one host-to-device copy per array,
// neighbour build, evaluation, one device-to-host copy per array and the
// status word, one event), and unpack the finished batch into the requests'
// output arrays while the GPU works on the new one.  Two arenas alternate.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "internal.cuh"

namespace flr {
namespace {

int64_t now_ns()
{
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Pending {
    flr_request req;
    std::vector<float> pos;      // copied inputs
    std::vector<int32_t> species;
    int64_t t_submit;
};

// Host side of one batch.
struct Slot {
    std::vector<Pending> reqs;
    int n_atoms = 0, n_structs = 0;
    int64_t t_start = 0;
    int status = FLR_OK;
    std::string error;
    // pinned arena
    size_t cap_atoms = 0, cap_structs = 0;
    float4 *pos = nullptr;
    int32_t *species = nullptr;
    float *energy = nullptr, *forces = nullptr, *variance = nullptr, *sigma = nullptr;
    double *totals = nullptr;
    int32_t *offsets = nullptr, *pbc = nullptr;
    double *cells = nullptr;
    float *bb = nullptr;
    int *dev_status = nullptr;   // pinned copy of the device status word
    cudaEvent_t done = nullptr;
};

void free_slot(Slot &s)
{
    cudaFreeHost(s.pos);
    cudaFreeHost(s.species);
    cudaFreeHost(s.energy);
    cudaFreeHost(s.forces);
    cudaFreeHost(s.variance);
    cudaFreeHost(s.sigma);
    cudaFreeHost(s.totals);
    cudaFreeHost(s.offsets);
    cudaFreeHost(s.pbc);
    cudaFreeHost(s.cells);
    cudaFreeHost(s.bb);
    s.pos = nullptr;
    s.species = nullptr;
    s.energy = s.forces = s.variance = s.sigma = nullptr;
    s.totals = nullptr;
    s.offsets = s.pbc = nullptr;
    s.cells = nullptr;
    s.bb = nullptr;
    s.cap_atoms = s.cap_structs = 0;
}

template <typename T>
cudaError_t host_alloc(T **p, size_t count)
{
    return cudaHostAlloc(reinterpret_cast<void **>(p), sizeof(T) * std::max<size_t>(count, 1), cudaHostAllocDefault);
}

// Grow a slot's pinned arena to hold n atoms and m structures.
int reserve_slot(Slot &s, size_t n, size_t m)
{
    if (n <= s.cap_atoms && m <= s.cap_structs) return FLR_OK;
    const size_t na = std::max(n, s.cap_atoms + s.cap_atoms / 2), ns = std::max(m, s.cap_structs + s.cap_structs / 2);
    int *st = s.dev_status;
    s.dev_status = nullptr;
    free_slot(s);
    cudaError_t e = host_alloc(&s.pos, na);
    if (e == cudaSuccess) e = host_alloc(&s.species, na);
    if (e == cudaSuccess) e = host_alloc(&s.energy, na);
    if (e == cudaSuccess) e = host_alloc(&s.forces, 3 * na);
    if (e == cudaSuccess) e = host_alloc(&s.variance, na);
    if (e == cudaSuccess) e = host_alloc(&s.sigma, na);
    if (e == cudaSuccess) e = host_alloc(&s.totals, FLR_NTOTALS * ns);
    if (e == cudaSuccess) e = host_alloc(&s.offsets, ns + 1);
    if (e == cudaSuccess) e = host_alloc(&s.pbc, 3 * ns);
    if (e == cudaSuccess) e = host_alloc(&s.cells, 9 * ns);
    if (e == cudaSuccess) e = host_alloc(&s.bb, 8 * ns);
    s.dev_status = st;
    if (e != cudaSuccess) {
        free_slot(s);
        return cuda_fail(e, "server: pinned host arena");
    }
    s.cap_atoms = na;
    s.cap_structs = ns;
    return FLR_OK;
}

}  // namespace
}  // namespace flr

using namespace flr;

struct flr_server {
    flr_ctx *ctx = nullptr;
    flr_server_params p{};
    int64_t bpa = 0;             // bytes per atom
    int64_t per_struct = 0;      // bytes per structure (totals, plans, a bin grid's worth of counters)
    cudaStream_t st = nullptr;
    flr_nbrlist *nl = nullptr;
    // device I/O, grown on demand
    size_t dcap_atoms = 0, dcap_structs = 0;
    float4 *d_pos = nullptr;
    int32_t *d_species = nullptr;
    float *d_energy = nullptr, *d_forces = nullptr, *d_variance = nullptr, *d_sigma = nullptr;
    double *d_totals = nullptr;
    Slot slot[2];
    // queue and completions
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Pending> queue;
    std::deque<flr_completion> done;
    bool stop = false;
    std::thread worker;
    // statistics (under mu)
    int64_t n_requests = 0, n_batches = 0, n_atoms = 0, max_batch_seen = 0;
    std::string last_error;

    int64_t batch_bytes(int64_t atoms, int64_t structs) const { return atoms * bpa + structs * per_struct; }
    int64_t reserved_bytes() const
    {
        return (int64_t)dcap_atoms * bpa + (int64_t)dcap_structs * per_struct;
    }
};

namespace flr {
namespace {

void free_device_io(flr_server *s)
{
    cudaFree(s->d_pos);
    cudaFree(s->d_species);
    cudaFree(s->d_energy);
    cudaFree(s->d_forces);
    cudaFree(s->d_variance);
    cudaFree(s->d_sigma);
    cudaFree(s->d_totals);
    s->d_pos = nullptr;
    s->d_species = nullptr;
    s->d_energy = s->d_forces = s->d_variance = s->d_sigma = nullptr;
    s->d_totals = nullptr;
    s->dcap_atoms = s->dcap_structs = 0;
}

// Device capacity for n atoms and m structures: the context's workspace,
// the neighbour list and the I/O arrays, grown by half again (never past the
// budget) so a slowly growing load does not reallocate every batch.
int reserve_device(flr_server *s, size_t n, size_t m)
{
    if (n <= s->dcap_atoms && m <= s->dcap_structs) return FLR_OK;
    const int64_t budget = (int64_t)s->p.hbm_budget_bytes;
    size_t na = std::max(n, s->dcap_atoms + s->dcap_atoms / 2);
    size_t ns = std::max(m, s->dcap_structs + s->dcap_structs / 2);
    if (s->batch_bytes((int64_t)na, (int64_t)ns) > budget) {
        na = n;
        ns = m;
    }
    cudaStreamSynchronize(s->st);
    free_device_io(s);
    if (s->nl) {
        flr_nbrlist_destroy(s->nl);
        s->nl = nullptr;
    }
    int r = flr_nbrlist_create(s->ctx, (int32_t)na, &s->nl);
    if (r == FLR_OK) r = srv_reserve_workspace(s->ctx, (int)na);
    cudaError_t e = cudaSuccess;
    if (r == FLR_OK) {
        e = cudaMalloc(&s->d_pos, sizeof(float4) * std::max<size_t>(na, 1));
        if (e == cudaSuccess) e = cudaMalloc(&s->d_species, sizeof(int32_t) * std::max<size_t>(na, 1));
        if (e == cudaSuccess) e = cudaMalloc(&s->d_energy, sizeof(float) * std::max<size_t>(na, 1));
        if (e == cudaSuccess) e = cudaMalloc(&s->d_forces, sizeof(float) * 3 * std::max<size_t>(na, 1));
        if (e == cudaSuccess) e = cudaMalloc(&s->d_variance, sizeof(float) * std::max<size_t>(na, 1));
        if (e == cudaSuccess) e = cudaMalloc(&s->d_sigma, sizeof(float) * std::max<size_t>(na, 1));
        if (e == cudaSuccess) e = cudaMalloc(&s->d_totals, sizeof(double) * FLR_NTOTALS * std::max<size_t>(ns, 1));
        if (e != cudaSuccess) r = cuda_fail(e, "server: device I/O arrays");
    }
    if (r != FLR_OK) {
        free_device_io(s);
        return r;
    }
    s->dcap_atoms = na;
    s->dcap_structs = ns;
    return FLR_OK;
}

// Admit queued requests (FIFO) into `out` while the batch fits.
void admit(flr_server *s, std::vector<Pending> &out)
{
    int64_t atoms = 0, structs = 0;
    const int64_t max_s = s->p.max_batch_structs > 0 ? s->p.max_batch_structs : INT64_MAX;
    const int64_t max_a = s->p.max_batch_atoms > 0 ? s->p.max_batch_atoms : INT64_MAX;
    while (!s->queue.empty()) {
        const Pending &q = s->queue.front();
        const int64_t a = atoms + q.req.n_atoms, m = structs + 1;
        if (m > max_s || a > max_a || a >= (1 << 24) || s->batch_bytes(a, m) > (int64_t)s->p.hbm_budget_bytes)
            break;
        out.push_back(std::move(s->queue.front()));
        s->queue.pop_front();
        atoms = a;
        structs = m;
    }
}

// Pack a batch's inputs into the slot's pinned arena (host work only).
int pack(Slot &sl)
{
    size_t n = 0;
    for (const Pending &q : sl.reqs) n += (size_t)q.req.n_atoms;
    const size_t m = sl.reqs.size();
    int r = reserve_slot(sl, n, m);
    if (r != FLR_OK) return r;
    size_t off = 0;
    for (size_t k = 0; k < m; ++k) {
        const Pending &q = sl.reqs[k];
        const int na = q.req.n_atoms;
        sl.offsets[k] = (int32_t)off;
        std::memcpy(sl.pos + off, q.pos.data(), sizeof(float4) * (size_t)na);
        std::memcpy(sl.species + off, q.species.data(), sizeof(int32_t) * (size_t)na);
        std::memcpy(sl.cells + 9 * k, q.req.cell, sizeof(double) * 9);
        for (int d = 0; d < 3; ++d) sl.pbc[3 * k + d] = q.req.pbc[d] ? 1 : 0;
        host_frac_bbox(q.req.cell, q.pos.data(), na, sl.bb + 8 * k);
        off += (size_t)na;
    }
    sl.offsets[m] = (int32_t)off;
    sl.n_atoms = (int)off;
    sl.n_structs = (int)m;
    return FLR_OK;
}

// Enqueue one packed batch on the server's stream.
int enqueue(flr_server *s, Slot &sl)
{
    const int n = sl.n_atoms, m = sl.n_structs;
    int r = reserve_device(s, (size_t)n, (size_t)m);
    if (r != FLR_OK) return r;
    cudaStream_t st = s->st;
    flr_ctx *c = s->ctx;
    if (n > 0) {
        r = cuda_fail(cudaMemcpyAsync(s->d_pos, sl.pos, sizeof(float4) * n, cudaMemcpyHostToDevice, st), "server H2D");
        if (r == FLR_OK)
            r = cuda_fail(cudaMemcpyAsync(s->d_species, sl.species, sizeof(int32_t) * n, cudaMemcpyHostToDevice, st),
                          "server H2D");
        s->nl->n = n;
        if (r == FLR_OK) r = plan_batch(c, s->nl, m, sl.offsets, sl.cells, sl.pbc, s->d_pos, n, st, sl.bb);
        if (r == FLR_OK) r = launch_set_rebuild(c, s->nl, st);
        if (r == FLR_OK) r = launch_rebuild(c, s->nl, s->d_pos, s->d_species, n, st, false, nullptr);
        flr_outputs o;
        o.energy = s->d_energy;
        o.forces = s->d_forces;
        o.variance = s->d_variance;
        o.sigma = s->d_sigma;
        o.totals = nullptr;
        if (r == FLR_OK) r = srv_evaluate(c, s->nl, s->d_pos, s->d_species, n, &o, s->d_totals, st);
        if (r != FLR_OK) return r;
        const size_t fb = sizeof(float) * (size_t)n;
        r = cuda_fail(cudaMemcpyAsync(sl.energy, s->d_energy, fb, cudaMemcpyDeviceToHost, st), "server D2H");
        if (r == FLR_OK) r = cuda_fail(cudaMemcpyAsync(sl.forces, s->d_forces, 3 * fb, cudaMemcpyDeviceToHost, st), "server D2H");
        if (r == FLR_OK) r = cuda_fail(cudaMemcpyAsync(sl.variance, s->d_variance, fb, cudaMemcpyDeviceToHost, st), "server D2H");
        if (r == FLR_OK) r = cuda_fail(cudaMemcpyAsync(sl.sigma, s->d_sigma, fb, cudaMemcpyDeviceToHost, st), "server D2H");
        if (r == FLR_OK)
            r = cuda_fail(cudaMemcpyAsync(sl.totals, s->d_totals, sizeof(double) * FLR_NTOTALS * m,
                                          cudaMemcpyDeviceToHost, st),
                          "server D2H");
        if (r == FLR_OK)
            r = cuda_fail(cudaMemcpyAsync(sl.dev_status, c->status, sizeof(int) * 4, cudaMemcpyDeviceToHost, st),
                          "server D2H");
        if (r == FLR_OK) r = cuda_fail(cudaMemsetAsync(c->status, 0, sizeof(int) * 4, st), "server status");
    } else {
        std::memset(sl.totals, 0, sizeof(double) * FLR_NTOTALS * m);
        std::memset(sl.dev_status, 0, sizeof(int) * 4);
    }
    if (r == FLR_OK) r = cuda_fail(cudaEventRecord(sl.done, st), "server event");
    return r;
}

// Wait for a slot's batch, write every request's outputs, report completions.
void finish(flr_server *s, Slot &sl)
{
    if (sl.status == FLR_OK) {
        sl.status = cuda_fail(cudaEventSynchronize(sl.done), "server batch");
        if (sl.status == FLR_OK && sl.dev_status[0]) sl.status = srv_status_code(sl.dev_status[0]);
        if (sl.status != FLR_OK) sl.error = flr_last_error();
    }
    std::vector<flr_completion> out(sl.reqs.size());
    for (size_t k = 0; k < sl.reqs.size(); ++k) {
        const flr_request &q = sl.reqs[k].req;
        if (sl.status == FLR_OK) {
            const size_t o = (size_t)sl.offsets[k], na = (size_t)q.n_atoms;
            if (q.energy) std::memcpy(q.energy, sl.energy + o, sizeof(float) * na);
            if (q.forces) std::memcpy(q.forces, sl.forces + 3 * o, sizeof(float) * 3 * na);
            if (q.variance) std::memcpy(q.variance, sl.variance + o, sizeof(float) * na);
            if (q.sigma) std::memcpy(q.sigma, sl.sigma + o, sizeof(float) * na);
            if (q.totals) std::memcpy(q.totals, sl.totals + FLR_NTOTALS * k, sizeof(double) * FLR_NTOTALS);
        }
        flr_completion &c = out[k];
        c.tag = q.tag;
        c.status = sl.status;
        c.batch_structs = sl.n_structs;
        c.batch_atoms = sl.n_atoms;
        c.t_submit_ns = sl.reqs[k].t_submit;
        c.t_start_ns = sl.t_start;
    }
    const int64_t t = now_ns();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (flr_completion &c : out) {
            c.t_done_ns = t;
            s->done.push_back(c);
        }
        s->n_requests += (int64_t)out.size();
        s->n_batches += 1;
        s->n_atoms += sl.n_atoms;
        s->max_batch_seen = std::max<int64_t>(s->max_batch_seen, sl.n_atoms);
        if (sl.status != FLR_OK) s->last_error = sl.error;
    }
    s->cv_done.notify_all();
    sl.reqs.clear();
}

void worker_loop(flr_server *s)
{
    cudaSetDevice(s->ctx->device);
    int cur = 0;
    bool inflight = false;
    for (;;) {
        Slot &sl = s->slot[cur];
        Slot &prev = s->slot[1 - cur];
        sl.reqs.clear();
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (!inflight) s->cv_work.wait(lk, [s] { return s->stop || !s->queue.empty(); });
            if (s->stop && !inflight) break;
            if (!s->stop) admit(s, sl.reqs);
        }
        if (!sl.reqs.empty()) {
            sl.status = pack(sl);
            if (sl.status != FLR_OK) sl.error = flr_last_error();
        }
        if (inflight) {
            // the GPU is (nearly) done with the previous batch: wait for it,
            // start the new one, then unpack the previous one
            cudaEventSynchronize(prev.done);
        }
        if (!sl.reqs.empty() && sl.status == FLR_OK) {
            sl.t_start = now_ns();
            sl.status = enqueue(s, sl);
            if (sl.status != FLR_OK) sl.error = flr_last_error();
        }
        if (inflight) {
            finish(s, prev);
            inflight = false;
        }
        if (!sl.reqs.empty()) {
            if (sl.status == FLR_OK) {
                inflight = true;
                cur = 1 - cur;
            } else {
                finish(s, sl);
            }
        }
    }
}

}  // namespace
}  // namespace flr

extern "C" {

int flr_bytes_per_atom(const flr_ctx *ctx, int64_t *bytes)
{
    if (!ctx || !bytes) {
        set_error("flr_bytes_per_atom: null argument");
        return FLR_EINVAL;
    }
    *bytes = bytes_per_atom(ctx);
    return FLR_OK;
}

int flr_server_create(flr_ctx *ctx, const flr_server_params *params, flr_server **out)
{
    if (!ctx || !params || !out) {
        set_error("flr_server_create: null argument");
        return FLR_EINVAL;
    }
    int r = srv_check_model(ctx);
    if (r != FLR_OK) return r;
    flr_server *s = new flr_server();
    s->ctx = ctx;
    s->p = *params;
    s->bpa = bytes_per_atom(ctx);
    s->per_struct = (int64_t)(sizeof(double) * FLR_NTOTALS + sizeof(Plan) + sizeof(double) * 9 + 16 + 4096 * 8);
    if (s->batch_bytes(1, 1) > (int64_t)params->hbm_budget_bytes) {
        set_error("flr_server_create: the memory budget cannot hold one atom (" + std::to_string(s->batch_bytes(1, 1)) +
                  " bytes)");
        delete s;
        return FLR_EBUDGET;
    }
    cudaSetDevice(ctx->device);
    r = cuda_fail(cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking), "server stream");
    for (int k = 0; k < 2 && r == FLR_OK; ++k) {
        r = cuda_fail(cudaEventCreateWithFlags(&s->slot[k].done, cudaEventDisableTiming), "server event");
        if (r == FLR_OK)
            r = cuda_fail(cudaHostAlloc(reinterpret_cast<void **>(&s->slot[k].dev_status), sizeof(int) * 4,
                                        cudaHostAllocDefault),
                          "server status");
    }
    if (r != FLR_OK) {
        flr_server_destroy(s);
        return r;
    }
    s->worker = std::thread(worker_loop, s);
    *out = s;
    return FLR_OK;
}

int flr_server_submit(flr_server *s, const flr_request *req)
{
    if (!s || !req || req->n_atoms < 0 || (req->n_atoms > 0 && (!req->pos || !req->species))) {
        set_error("flr_server_submit: invalid request");
        return FLR_EINVAL;
    }
    const int64_t max_a = s->p.max_batch_atoms > 0 ? s->p.max_batch_atoms : INT64_MAX;
    if (req->n_atoms > max_a || s->batch_bytes(req->n_atoms, 1) > (int64_t)s->p.hbm_budget_bytes ||
        req->n_atoms >= (1 << 24)) {
        set_error("flr_server_submit: " + std::to_string(req->n_atoms) + " atoms exceed the server's budget");
        return FLR_EBUDGET;
    }
    for (int k = 0; k < 9; ++k)
        if (!std::isfinite(req->cell[k])) {
            set_error("flr_server_submit: non-finite cell");
            return FLR_EINVAL;
        }
    Pending p;
    p.req = *req;
    p.pos.assign(req->pos, req->pos + 4 * (size_t)req->n_atoms);
    p.species.assign(req->species, req->species + (size_t)req->n_atoms);
    for (int32_t v : p.species)
        if (v < 0 || v >= s->ctx->p.n_species) {
            set_error("flr_server_submit: species index out of range");
            return FLR_EINVAL;
        }
    p.req.pos = nullptr;
    p.req.species = nullptr;
    p.t_submit = now_ns();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->queue.push_back(std::move(p));
    }
    s->cv_work.notify_one();
    return FLR_OK;
}

int flr_server_poll(flr_server *s, flr_completion *out, int32_t max, int32_t *n_out, double wait_seconds)
{
    if (!s || !n_out || (max > 0 && !out)) {
        set_error("flr_server_poll: invalid argument");
        return FLR_EINVAL;
    }
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->done.empty() && wait_seconds > 0)
        s->cv_done.wait_for(lk, std::chrono::duration<double>(wait_seconds), [s] { return !s->done.empty(); });
    int32_t k = 0;
    while (k < max && !s->done.empty()) {
        out[k++] = s->done.front();
        s->done.pop_front();
    }
    *n_out = k;
    return FLR_OK;
}

int flr_server_stats_read(flr_server *s, flr_server_stats *st)
{
    if (!s || !st) {
        set_error("flr_server_stats_read: null argument");
        return FLR_EINVAL;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(st, 0, sizeof(*st));
    st->requests = s->n_requests;
    st->batches = s->n_batches;
    st->atoms = s->n_atoms;
    st->max_batch_atoms_seen = s->max_batch_seen;
    st->queued = (int64_t)s->queue.size();
    st->reserved_bytes = s->reserved_bytes();
    st->bytes_per_atom = s->bpa;
    std::strncpy(st->last_error, s->last_error.c_str(), sizeof(st->last_error) - 1);
    return FLR_OK;
}

int flr_server_destroy(flr_server *s)
{
    if (!s) return FLR_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    cudaSetDevice(s->ctx->device);
    if (s->st) cudaStreamSynchronize(s->st);
    free_device_io(s);
    if (s->nl) flr_nbrlist_destroy(s->nl);
    for (int k = 0; k < 2; ++k) {
        free_slot(s->slot[k]);
        cudaFreeHost(s->slot[k].dev_status);
        if (s->slot[k].done) cudaEventDestroy(s->slot[k].done);
    }
    if (s->st) cudaStreamDestroy(s->st);
    delete s;
    return FLR_OK;
}

}  // extern "C"
