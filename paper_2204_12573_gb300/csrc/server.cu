// Continuous-batching evaluation service (flr_server_*).
//
// One worker thread per server drives two batch slots.  Each slot owns a
// CUDA stream, a pinned host arena, device input/output arrays and a
// neighbour list (with its own device status word and work counter), so the
// batches of the two slots overlap on the device: while one batch is being
// evaluated, the next one is copied in and its neighbour lists are built.
// The evaluation kernels share the context's workspace, so evaluations run
// one at a time: each waits for an event recorded after the previous
// batch's evaluation.
//
// One batch, on its slot's stream: one host-to-device copy per input array,
// the bin-grid plan (computed on the host from each structure's fractional
// bounding box, so no device round trip), the neighbour build, a wait for
// the workspace, the evaluation, the status words copied back and cleared,
// the workspace event, one device-to-host copy per output array, and a host
// callback that wakes the worker.  The worker admits queued requests in
// arrival order into a free slot while the batch fits the budget, packs them
// into the slot's arena and enqueues the batch; when a slot's batch is done
// it writes every request's outputs and reports the completions.
//
// Device memory is reserved up front (flr_server_params.reserve_atoms) or
// grown by doubling when a batch does not fit; growing synchronizes the
// device, and the stats count how often it happened and how long it took.
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

constexpr int kSlots = 2;

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

// One batch slot: host arena, device arrays, neighbour list and stream.
struct Slot {
    flr_server *srv = nullptr;
    int index = 0;
    std::vector<Pending> reqs;
    int n_atoms = 0, n_structs = 0;
    int64_t t_start = 0;
    int status = FLR_OK;
    std::string error;
    bool inflight = false;       // a batch was enqueued and not yet finished
    bool gpu_done = false;       // set by the stream callback (under the server mutex)
    // pinned arena
    size_t cap_atoms = 0, cap_structs = 0;
    float4 *pos = nullptr;
    int32_t *species = nullptr;
    float *energy = nullptr, *forces = nullptr, *variance = nullptr, *sigma = nullptr;
    double *totals = nullptr;
    int32_t *offsets = nullptr, *pbc = nullptr;
    double *cells = nullptr;
    float *bb = nullptr;
    int *dev_status = nullptr;   // pinned copies of the status words: [0..3] evaluation, [4..7] list build
    // device side
    cudaStream_t st = nullptr;
    flr_nbrlist *nl = nullptr;
    int *d_words = nullptr;      // [8]: list-build status word [0..3], list-build work counter [4]
    size_t dcap_atoms = 0, dcap_structs = 0;
    float4 *d_pos = nullptr;
    int32_t *d_species = nullptr;
    float *d_energy = nullptr, *d_forces = nullptr, *d_variance = nullptr, *d_sigma = nullptr;
    double *d_totals = nullptr;
    // timing events of the last batch (device clock): H2D start, build end, evaluation start / end, done
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
};

void free_host(Slot &s)
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

// Pinned arena for n atoms and m structures (grown by doubling).
int reserve_host(Slot &s, size_t n, size_t m)
{
    if (n <= s.cap_atoms && m <= s.cap_structs) return FLR_OK;
    const size_t na = std::max(n, 2 * s.cap_atoms), ns = std::max(m, 2 * s.cap_structs);
    free_host(s);
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
    if (e != cudaSuccess) {
        free_host(s);
        return cuda_fail(e, "server: pinned host arena");
    }
    s.cap_atoms = na;
    s.cap_structs = ns;
    return FLR_OK;
}

void free_device(Slot &s)
{
    cudaFree(s.d_pos);
    cudaFree(s.d_species);
    cudaFree(s.d_energy);
    cudaFree(s.d_forces);
    cudaFree(s.d_variance);
    cudaFree(s.d_sigma);
    cudaFree(s.d_totals);
    s.d_pos = nullptr;
    s.d_species = nullptr;
    s.d_energy = s.d_forces = s.d_variance = s.d_sigma = nullptr;
    s.d_totals = nullptr;
    if (s.nl) flr_nbrlist_destroy(s.nl);
    s.nl = nullptr;
    s.dcap_atoms = s.dcap_structs = 0;
}

}  // namespace
}  // namespace flr

using namespace flr;

struct flr_server {
    flr_ctx *ctx = nullptr;
    flr_server_params p{};
    int64_t ws_bpa = 0;          // workspace bytes per atom (one batch evaluates at a time)
    int64_t slot_bpa = 0;        // neighbour list and I/O bytes per atom (each slot)
    int64_t per_struct = 0;      // bytes per structure (totals, plans, a bin grid's worth of counters)
    Slot slot[kSlots];
    cudaEvent_t ws_free = nullptr;   // recorded after each evaluation (the shared workspace)
    bool ws_used = false;
    cudaEvent_t t0 = nullptr;        // origin of the device timestamps
    std::deque<int> order;           // slots in flight, oldest first
    // queue and completions
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Pending> queue;
    std::deque<flr_completion> done;
    bool stop = false;
    std::thread worker;
    // statistics (under mu)
    int64_t n_requests = 0, n_batches = 0, n_atoms = 0, max_batch_seen = 0, n_overlapped = 0;
    int64_t grow_events = 0, ns_grow = 0, ns_pack = 0, ns_enqueue = 0, ns_finish = 0;
    std::string last_error;

    // device bytes of a batch of `atoms` atoms and `structs` structures: the
    // workspace once, the neighbour lists and I/O of both slots
    int64_t batch_bytes(int64_t atoms, int64_t structs) const
    {
        return atoms * (ws_bpa + kSlots * slot_bpa) + kSlots * structs * per_struct;
    }
    int64_t reserved_bytes() const
    {
        int64_t b = (int64_t)ctx->ws_n * ws_bpa;
        for (int k = 0; k < kSlots; ++k)
            b += (int64_t)slot[k].dcap_atoms * slot_bpa + (int64_t)slot[k].dcap_structs * per_struct;
        return b;
    }
};

namespace flr {
namespace {

// The stream callback of a finished batch (no CUDA calls allowed here).
void CUDART_CB on_batch_done(void *arg)
{
    Slot *sl = static_cast<Slot *>(arg);
    flr_server *s = sl->srv;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        sl->gpu_done = true;
    }
    s->cv_work.notify_all();
}

// Device capacity of a slot for n atoms and m structures: its neighbour list,
// its I/O arrays and, shared by the slots, the context's workspace.  Grows
// by doubling (never past what the budget allows for one batch); growing
// synchronizes the device.
int reserve_device(flr_server *s, Slot &sl, size_t n, size_t m)
{
    flr_ctx *c = s->ctx;
    const bool slot_ok = n <= sl.dcap_atoms && m <= sl.dcap_structs;
    const bool ws_ok = (int64_t)n <= (int64_t)c->ws_n;
    if (slot_ok && ws_ok) return FLR_OK;
    const int64_t t0 = now_ns();
    const int64_t budget = (int64_t)s->p.hbm_budget_bytes;
    size_t na = std::max(n, 2 * sl.dcap_atoms), ns = std::max(m, 2 * sl.dcap_structs);
    if (s->batch_bytes((int64_t)na, (int64_t)ns) > budget) {
        na = std::max(n, sl.dcap_atoms);
        ns = std::max(m, sl.dcap_structs);
    }
    int r = FLR_OK;
    if (!slot_ok) {
        cudaStreamSynchronize(sl.st);
        free_device(sl);
        r = flr_nbrlist_create(c, (int32_t)na, &sl.nl);
        if (r == FLR_OK) {
            sl.nl->status = sl.d_words;
            sl.nl->sched = sl.d_words + 4;
        }
        cudaError_t e = cudaSuccess;
        if (r == FLR_OK) {
            e = cudaMalloc(&sl.d_pos, sizeof(float4) * std::max<size_t>(na, 1));
            if (e == cudaSuccess) e = cudaMalloc(&sl.d_species, sizeof(int32_t) * std::max<size_t>(na, 1));
            if (e == cudaSuccess) e = cudaMalloc(&sl.d_energy, sizeof(float) * std::max<size_t>(na, 1));
            if (e == cudaSuccess) e = cudaMalloc(&sl.d_forces, sizeof(float) * 3 * std::max<size_t>(na, 1));
            if (e == cudaSuccess) e = cudaMalloc(&sl.d_variance, sizeof(float) * std::max<size_t>(na, 1));
            if (e == cudaSuccess) e = cudaMalloc(&sl.d_sigma, sizeof(float) * std::max<size_t>(na, 1));
            if (e == cudaSuccess) e = cudaMalloc(&sl.d_totals, sizeof(double) * FLR_NTOTALS * std::max<size_t>(ns, 1));
            if (e != cudaSuccess) r = cuda_fail(e, "server: device I/O arrays");
        }
        if (r != FLR_OK) {
            free_device(sl);
            return r;
        }
        sl.dcap_atoms = na;
        sl.dcap_structs = ns;
    }
    if (!ws_ok) {
        int64_t nw = std::max<int64_t>((int64_t)n, 2 * (int64_t)c->ws_n);
        if (s->batch_bytes(nw, (int64_t)ns) > budget) nw = (int64_t)n;
        r = srv_reserve_workspace(c, (int)nw);   // synchronizes the device
        if (r != FLR_OK) return r;
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->grow_events += 1;
        s->ns_grow += now_ns() - t0;
    }
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

// Pack a batch's inputs into the slot's pinned arena and compute each
// structure's fractional bounding box (host work only).
int pack(Slot &sl)
{
    size_t n = 0;
    for (const Pending &q : sl.reqs) n += (size_t)q.req.n_atoms;
    const size_t m = sl.reqs.size();
    int r = reserve_host(sl, n, m);
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

// Enqueue one packed batch on its slot's stream (see the file comment).
int enqueue(flr_server *s, Slot &sl)
{
    const int n = sl.n_atoms, m = sl.n_structs;
    int r = reserve_device(s, sl, (size_t)n, (size_t)m);
    if (r != FLR_OK) return r;
    cudaStream_t st = sl.st;
    flr_ctx *c = s->ctx;
    cudaEventRecord(sl.ev[0], st);
    if (n > 0) {
        r = cuda_fail(cudaMemcpyAsync(sl.d_pos, sl.pos, sizeof(float4) * n, cudaMemcpyHostToDevice, st), "server H2D");
        if (r == FLR_OK)
            r = cuda_fail(cudaMemcpyAsync(sl.d_species, sl.species, sizeof(int32_t) * n, cudaMemcpyHostToDevice, st),
                          "server H2D");
        sl.nl->n = n;
        if (r == FLR_OK) r = plan_batch(c, sl.nl, m, sl.offsets, sl.cells, sl.pbc, sl.d_pos, n, st, sl.bb);
        if (r == FLR_OK) r = launch_set_rebuild(c, sl.nl, st);
        if (r == FLR_OK) r = launch_rebuild(c, sl.nl, sl.d_pos, sl.d_species, n, st, false, nullptr);
        if (r == FLR_OK) r = cuda_fail(cudaEventRecord(sl.ev[1], st), "server event");
        // the workspace is free once the previous batch's evaluation is done
        if (r == FLR_OK && s->ws_used) r = cuda_fail(cudaStreamWaitEvent(st, s->ws_free, 0), "server event");
        if (r == FLR_OK) r = cuda_fail(cudaEventRecord(sl.ev[2], st), "server event");
        flr_outputs o;
        o.energy = sl.d_energy;
        o.forces = sl.d_forces;
        o.variance = sl.d_variance;
        o.sigma = sl.d_sigma;
        o.totals = nullptr;
        if (r == FLR_OK) r = srv_evaluate(c, sl.nl, sl.d_pos, sl.d_species, n, &o, sl.d_totals, st);
        if (r == FLR_OK)
            r = cuda_fail(cudaMemcpyAsync(sl.dev_status, c->status, sizeof(int) * 4, cudaMemcpyDeviceToHost, st),
                          "server D2H");
        if (r == FLR_OK) r = cuda_fail(cudaMemsetAsync(c->status, 0, sizeof(int) * 4, st), "server status");
        if (r == FLR_OK) r = cuda_fail(cudaEventRecord(sl.ev[3], st), "server event");
        if (r == FLR_OK) r = cuda_fail(cudaEventRecord(s->ws_free, st), "server event");
        if (r != FLR_OK) return r;
        s->ws_used = true;
        const size_t fb = sizeof(float) * (size_t)n;
        r = cuda_fail(cudaMemcpyAsync(sl.energy, sl.d_energy, fb, cudaMemcpyDeviceToHost, st), "server D2H");
        if (r == FLR_OK) r = cuda_fail(cudaMemcpyAsync(sl.forces, sl.d_forces, 3 * fb, cudaMemcpyDeviceToHost, st), "server D2H");
        if (r == FLR_OK) r = cuda_fail(cudaMemcpyAsync(sl.variance, sl.d_variance, fb, cudaMemcpyDeviceToHost, st), "server D2H");
        if (r == FLR_OK) r = cuda_fail(cudaMemcpyAsync(sl.sigma, sl.d_sigma, fb, cudaMemcpyDeviceToHost, st), "server D2H");
        if (r == FLR_OK)
            r = cuda_fail(cudaMemcpyAsync(sl.totals, sl.d_totals, sizeof(double) * FLR_NTOTALS * m,
                                          cudaMemcpyDeviceToHost, st),
                          "server D2H");
        if (r == FLR_OK)
            r = cuda_fail(cudaMemcpyAsync(sl.dev_status + 4, sl.d_words, sizeof(int) * 4, cudaMemcpyDeviceToHost, st),
                          "server D2H");
        if (r == FLR_OK) r = cuda_fail(cudaMemsetAsync(sl.d_words, 0, sizeof(int) * 4, st), "server status");
    } else {
        std::memset(sl.totals, 0, sizeof(double) * FLR_NTOTALS * m);
        std::memset(sl.dev_status, 0, sizeof(int) * 8);
        for (int k = 1; k < 4 && r == FLR_OK; ++k) r = cuda_fail(cudaEventRecord(sl.ev[k], st), "server event");
    }
    if (r == FLR_OK) r = cuda_fail(cudaEventRecord(sl.ev[4], st), "server event");
    if (r == FLR_OK) r = cuda_fail(cudaLaunchHostFunc(st, on_batch_done, &sl), "server callback");
    return r;
}

float event_ms(flr_server *s, cudaEvent_t e)
{
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, s->t0, e) != cudaSuccess) ms = -1.f;
    return ms;
}

// Write every request's outputs of a finished slot and report completions.
void finish(flr_server *s, Slot &sl)
{
    const int64_t t_f0 = now_ns();
    float tms[5] = {-1.f, -1.f, -1.f, -1.f, -1.f};
    if (sl.status == FLR_OK) {
        sl.status = cuda_fail(cudaEventSynchronize(sl.ev[4]), "server batch");
        if (sl.status == FLR_OK) {
            const int st = sl.dev_status[0] | sl.dev_status[4];
            if (st) sl.status = srv_status_code(st);
            for (int k = 0; k < 5; ++k) tms[k] = event_ms(s, sl.ev[k]);
        }
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
        std::memset(&c, 0, sizeof(c));
        c.tag = q.tag;
        c.status = sl.status;
        c.batch_structs = sl.n_structs;
        c.batch_atoms = sl.n_atoms;
        c.t_submit_ns = sl.reqs[k].t_submit;
        c.t_start_ns = sl.t_start;
        c.slot = sl.index;
        c.gpu_start_ms = tms[0];
        c.gpu_built_ms = tms[1];
        c.gpu_eval_start_ms = tms[2];
        c.gpu_eval_end_ms = tms[3];
        c.gpu_done_ms = tms[4];
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
        s->ns_finish += t - t_f0;
        if (sl.status != FLR_OK) s->last_error = sl.error;
        sl.inflight = false;
        sl.gpu_done = false;
    }
    s->cv_done.notify_all();
    sl.reqs.clear();
}

void worker_loop(flr_server *s)
{
    cudaSetDevice(s->ctx->device);
    for (;;) {
        // the oldest batch in flight, once its stream callback has run
        int ready = -1, free_slot = -1;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            auto have_work = [&] {
                if (!s->order.empty() && s->slot[s->order.front()].gpu_done) return true;
                if (s->stop) return s->order.empty() || s->slot[s->order.front()].gpu_done;
                if (s->queue.empty()) return false;
                for (int k = 0; k < kSlots; ++k)
                    if (!s->slot[k].inflight) return true;
                return false;
            };
            s->cv_work.wait(lk, have_work);
            if (!s->order.empty() && s->slot[s->order.front()].gpu_done) {
                ready = s->order.front();
                s->order.pop_front();
            } else if (s->stop) {
                break;
            } else {
                for (int k = 0; k < kSlots && free_slot < 0; ++k)
                    if (!s->slot[k].inflight) free_slot = k;
                admit(s, s->slot[free_slot].reqs);
            }
        }
        if (ready >= 0) {
            finish(s, s->slot[ready]);
            continue;
        }
        Slot &sl = s->slot[free_slot];
        const int64_t t0 = now_ns();
        sl.status = pack(sl);
        if (sl.status != FLR_OK) sl.error = flr_last_error();
        const int64_t t1 = now_ns();
        if (sl.status == FLR_OK) {
            sl.t_start = t1;
            sl.status = enqueue(s, sl);
            if (sl.status != FLR_OK) sl.error = flr_last_error();
        }
        const int64_t t2 = now_ns();
        bool overlapped = false;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->ns_pack += t1 - t0;
            s->ns_enqueue += t2 - t1;
            for (int k = 0; k < kSlots; ++k)
                if (k != free_slot && s->slot[k].inflight) overlapped = true;
            if (overlapped) s->n_overlapped += 1;
            if (sl.status == FLR_OK) {
                sl.inflight = true;
                s->order.push_back(free_slot);
            }
        }
        if (sl.status != FLR_OK) {
            // nothing of this batch is left running once its stream is idle
            cudaStreamSynchronize(sl.st);
            finish(s, sl);
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
    int64_t ws = 0, sl = 0;
    bytes_per_atom_parts(ctx, &ws, &sl);
    *bytes = ws + kSlots * sl;
    return FLR_OK;
}

int flr_server_destroy(flr_server *s);

int flr_server_create(flr_ctx *ctx, const flr_server_params *params, flr_server **out)
{
    if (!ctx || !params || !out || params->reserve_atoms < 0 || params->reserve_structs < 0) {
        set_error("flr_server_create: invalid argument");
        return FLR_EINVAL;
    }
    int r = srv_check_model(ctx);
    if (r != FLR_OK) return r;
    flr_server *s = new flr_server();
    s->ctx = ctx;
    s->p = *params;
    bytes_per_atom_parts(ctx, &s->ws_bpa, &s->slot_bpa);
    s->per_struct = (int64_t)(sizeof(double) * FLR_NTOTALS + sizeof(Plan) + sizeof(double) * 9 + 16 + 4096 * 8);
    if (s->batch_bytes(1, 1) > (int64_t)params->hbm_budget_bytes) {
        set_error("flr_server_create: the memory budget cannot hold one atom (" + std::to_string(s->batch_bytes(1, 1)) +
                  " bytes)");
        delete s;
        return FLR_EBUDGET;
    }
    if (params->reserve_atoms > 0 &&
        s->batch_bytes(params->reserve_atoms, std::max(params->reserve_structs, 1)) > (int64_t)params->hbm_budget_bytes) {
        set_error("flr_server_create: reserve_atoms exceeds the memory budget");
        delete s;
        return FLR_EBUDGET;
    }
    cudaSetDevice(ctx->device);
    r = cuda_fail(cudaEventCreateWithFlags(&s->ws_free, cudaEventDisableTiming), "server event");
    if (r == FLR_OK) r = cuda_fail(cudaEventCreate(&s->t0), "server event");
    if (r == FLR_OK) r = cuda_fail(cudaEventRecord(s->t0, 0), "server event");
    for (int k = 0; k < kSlots && r == FLR_OK; ++k) {
        Slot &sl = s->slot[k];
        sl.srv = s;
        sl.index = k;
        r = cuda_fail(cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking), "server stream");
        for (int e = 0; e < 5 && r == FLR_OK; ++e) r = cuda_fail(cudaEventCreate(&sl.ev[e]), "server event");
        if (r == FLR_OK)
            r = cuda_fail(cudaHostAlloc(reinterpret_cast<void **>(&sl.dev_status), sizeof(int) * 8, cudaHostAllocDefault),
                          "server status");
        if (r == FLR_OK) r = cuda_fail(cudaMalloc(&sl.d_words, sizeof(int) * 8), "server status");
        if (r == FLR_OK) r = cuda_fail(cudaMemset(sl.d_words, 0, sizeof(int) * 8), "server status");
        if (r == FLR_OK && params->reserve_atoms > 0) {
            const size_t na = (size_t)params->reserve_atoms, ns = (size_t)std::max(params->reserve_structs, 1);
            r = reserve_host(sl, na, ns);
            if (r == FLR_OK) r = reserve_device(s, sl, na, ns);
            if (r == FLR_OK) {
                // the bin-grid and per-structure tables of the slot's list too
                r = nbrlist_reserve_batch(ctx, sl.nl, (int)ns, (long long)ns * 4096 + (long long)na);
            }
        }
    }
    if (r == FLR_OK) {
        s->grow_events = 0;   // the reservation is not growth under load
        s->ns_grow = 0;
        r = cuda_fail(cudaDeviceSynchronize(), "server reservation");
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
    s->cv_work.notify_all();
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
    st->bytes_per_atom = s->ws_bpa + kSlots * s->slot_bpa;
    std::strncpy(st->last_error, s->last_error.c_str(), sizeof(st->last_error) - 1);
    st->batches_overlapped = s->n_overlapped;
    st->grow_events = s->grow_events;
    st->grow_ms = s->ns_grow * 1e-6;
    st->pack_ms = s->ns_pack * 1e-6;
    st->enqueue_ms = s->ns_enqueue * 1e-6;
    st->finish_ms = s->ns_finish * 1e-6;
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
    for (int k = 0; k < kSlots; ++k)
        if (s->slot[k].st) cudaStreamSynchronize(s->slot[k].st);
    for (int k = 0; k < kSlots; ++k) {
        Slot &sl = s->slot[k];
        free_device(sl);
        free_host(sl);
        cudaFreeHost(sl.dev_status);
        cudaFree(sl.d_words);
        for (int e = 0; e < 5; ++e)
            if (sl.ev[e]) cudaEventDestroy(sl.ev[e]);
        if (sl.st) cudaStreamDestroy(sl.st);
    }
    if (s->ws_free) cudaEventDestroy(s->ws_free);
    if (s->t0) cudaEventDestroy(s->t0);
    delete s;
    return FLR_OK;
}

}  // extern "C"
