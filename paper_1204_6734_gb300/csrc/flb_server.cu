// flb_server.cu -- continuous-batching request server for simulation requests.
//
// A request is one periodic FP32 lattice (parameters, number of steps,
// sampling schedule); its result is its correlation sums. Requests wait in a
// FIFO queue and are admitted, in order, whenever a slot and a range of the
// device pool (the HBM budget) are free. Admitted requests run together:
//
//  * batched mode: all running requests are replicas of one batch
//    (flb_batch.cu), stepped by one persistent launch per step, in chunks of
//    `chunk` steps replayed from a CUDA graph;
//  * per-lattice mode (the comparison): each running request is its own
//    lattice handle on a workspace carved from the same pool, stepped by one
//    launch per lattice and step.
//
// The host runs ahead of the GPU by up to kDepth chunks. A request that ends
// inside a chunk is known on the host when the chunk is enqueued: the copy of
// its sums and error record into page-locked memory is enqueued right after
// the chunk, and its slot and pool range are returned at once (later users
// are ordered after the copy on the same stream). When the chunk's event has
// completed, its finished requests become results.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <cstring>
#include <deque>
#include <new>
#include <unordered_map>
#include <vector>

#include "../../include/flb.h"
#include "flb_arena.h"
#include "flb_host.h"
#include "flb_kernels.cuh"
#include "flb_runtime.h"

using namespace flb;

namespace {

constexpr int kDepth = 2;   // chunks in flight

struct alignas(64) PinnedResult {
    double acc[kSums];
    DevError err;
};

struct Req {
    int64_t id = 0;
    flb_params p;
    int64_t nsteps = 0, warmup = 0, every = 0;
    double t_submit = 0, t_admit = 0;
    int slot = -1;                  // batch slot (batched mode)
    flb_lattice lat = nullptr;      // handle (per-lattice mode)
    size_t off = 0;                 // pool range (per-lattice mode)
    int64_t done = 0;               // steps enqueued (per-lattice mode)
};

struct Finished {
    int64_t id;
    int record;                     // index into the page-locked results
    int64_t steps, nsamp;
};

struct Chunk {
    cudaEvent_t start = nullptr, end = nullptr;
    std::vector<Finished> fin;
    int64_t replica_steps = 0, node_steps = 0;
};

}  // namespace

struct flb_server_s {
    int mode = FLB_SERVE_BATCHED;
    int basis = 0, max_slots = 0, chunk = 0;
    cudaStream_t stream = nullptr;
    std::chrono::steady_clock::time_point t0;
    // batched mode
    flb_batch batch = nullptr;
    // per-lattice mode
    char* pool = nullptr;
    Arena arena;
    int running_lat = 0;
    int64_t live = 0;                            // admitted and not yet at their last step
    // requests
    int64_t next_id = 0;
    std::deque<int64_t> queue;
    std::unordered_map<int64_t, Req> reqs;      // queued and running
    std::deque<Chunk> inflight;
    std::vector<cudaEvent_t> spare_events;
    PinnedResult* pinned = nullptr;
    std::vector<int> free_records;
    std::deque<flb_result> done;
    flb_serve_stats st;
};

namespace {

double now_s(const flb_server_s* s) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

cudaError_t take_event(flb_server_s* s, cudaEvent_t* e) {
    if (!s->spare_events.empty()) {
        *e = s->spare_events.back();
        s->spare_events.pop_back();
        return cudaSuccess;
    }
    return cudaEventCreate(e);
}

void to_result(const PinnedResult& r, const Req& q, const Finished& f, double t_done,
               flb_result* out) {
    std::memset(out, 0, sizeof(*out));
    out->id = q.id;
    out->status = map_status(r.err.code);
    out->steps = f.steps;
    out->n_samples = f.nsamp;
    for (int i = 0; i < 9; ++i) out->S1[i] = r.acc[i];
    int k = 9;
    for (int i = 0; i < 9; ++i)
        for (int j = i; j < 9; ++j, ++k) out->S2[i * 9 + j] = out->S2[j * 9 + i] = r.acc[k];
    out->t_submit = q.t_submit;
    out->t_admit = q.t_admit;
    out->t_done = t_done;
}

// Move the chunks whose work has completed to the results (all of them when
// wait, else as far as they have completed in order).
int retire(flb_server_s* s, bool wait) {
    while (!s->inflight.empty()) {
        Chunk& c = s->inflight.front();
        cudaError_t ce = wait ? cudaEventSynchronize(c.end) : cudaEventQuery(c.end);
        if (ce == cudaErrorNotReady) return FLB_OK;
        if (ce != cudaSuccess) {
            cudaGetLastError();
            return FLB_ERR_CUDA;
        }
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c.start, c.end) == cudaSuccess) s->st.gpu_busy_s += ms * 1e-3;
        const double t = now_s(s);
        for (const Finished& f : c.fin) {
            auto it = s->reqs.find(f.id);
            if (it == s->reqs.end()) continue;
            flb_result r;
            to_result(s->pinned[f.record], it->second, f, t, &r);
            s->done.push_back(r);
            s->free_records.push_back(f.record);
            s->reqs.erase(it);
            s->st.completed += 1;
            s->st.finishing -= 1;
        }
        s->st.replica_steps += c.replica_steps;
        s->st.node_steps += c.node_steps;
        s->st.chunks += 1;
        s->spare_events.push_back(c.start);
        s->spare_events.push_back(c.end);
        s->inflight.pop_front();
        wait = false;
    }
    return FLB_OK;
}

// Admit queued requests in order while a slot and pool memory are free.
int admit(flb_server_s* s) {
    while (!s->queue.empty()) {
        Req& q = s->reqs[s->queue.front()];
        int rc = FLB_OK;
        if (s->mode == FLB_SERVE_BATCHED) {
            int32_t slot = -1;
            rc = flb_batch_add(s->batch, &q.p, q.nsteps, &slot);
            if (rc == FLB_ERR_OOM) return FLB_OK;
            if (rc == FLB_OK) rc = flb_batch_set_sampling(s->batch, slot, q.warmup, q.every);
            if (rc != FLB_OK) return rc;
            q.slot = slot;
            size_t used = 0;
            flb_batch_info(s->batch, nullptr, nullptr, &used, nullptr);
            s->st.pool_used = (int64_t)used;
        } else {
            if (s->running_lat >= s->max_slots) return FLB_OK;
            const size_t ws = flb_workspace_bytes(&q.p);
            size_t off = 0;
            if (ws == 0) return FLB_ERR_ARG;
            if (!s->arena.alloc(ws, &off)) return FLB_OK;
            rc = lattice_create(&q.p, s->pool + off, Arena::round_up(ws), s->stream, false, &q.lat);
            if (rc == FLB_OK) rc = flb_set_option(q.lat, FLB_OPT_KERNEL, FLB_KERNEL_PIPELINED);
            if (rc == FLB_OK) rc = flb_set_sampling(q.lat, q.warmup, q.every);
            if (rc != FLB_OK) {
                if (q.lat) lattice_forget(q.lat);
                q.lat = nullptr;
                s->arena.release(off);
                return rc;
            }
            q.off = off;
            s->running_lat += 1;
            s->st.pool_used = (int64_t)s->arena.used();
        }
        q.t_admit = now_s(s);
        s->live += 1;
        s->queue.pop_front();
        s->st.queued -= 1;
        s->st.running += 1;
    }
    return FLB_OK;
}

// Enqueue the next chunk of steps of every running request.
int enqueue_chunk(flb_server_s* s) {
    if (s->live <= 0) return FLB_OK;
    Chunk c;
    cudaError_t ce = take_event(s, &c.start);
    if (ce == cudaSuccess) ce = take_event(s, &c.end);
    if (ce == cudaSuccess) ce = cudaEventRecord(c.start, s->stream);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return FLB_ERR_CUDA;
    }
    std::vector<int64_t> ending;
    if (s->mode == FLB_SERVE_BATCHED) {
        int64_t step0 = 0;
        flb_batch_time(s->batch, &step0);
        for (auto& kv : s->reqs) {
            const Req& q = kv.second;
            if (q.slot < 0) continue;
            const int64_t t = batch_replica_time(s->batch, q.slot);
            const int64_t n = std::min<int64_t>(s->chunk, q.nsteps - t);
            c.replica_steps += n;
            c.node_steps += n * (int64_t)q.p.Lx * q.p.Ly;
            if (t + n >= q.nsteps) ending.push_back(q.id);
        }
        int rc = flb_batch_step(s->batch, s->chunk);
        if (rc != FLB_OK) return rc;
    } else {
        for (auto& kv : s->reqs) {
            Req& q = kv.second;
            if (!q.lat) continue;
            const int64_t n = std::min<int64_t>(s->chunk, q.nsteps - q.done);
            int rc = flb_step(q.lat, n);
            if (rc != FLB_OK) return rc;
            q.done += n;
            c.replica_steps += n;
            c.node_steps += n * (int64_t)q.p.Lx * q.p.Ly;
            if (q.done >= q.nsteps) ending.push_back(q.id);
        }
    }
    for (int64_t id : ending) {
        Req& q = s->reqs[id];
        if (s->free_records.empty()) return FLB_ERR_STATE;
        const int rec = s->free_records.back();
        s->free_records.pop_back();
        Finished f{id, rec, q.nsteps, 0};
        int rc;
        if (s->mode == FLB_SERVE_BATCHED) {
            f.nsamp = batch_samples(s->batch, q.slot);
            rc = batch_enqueue_readout(s->batch, q.slot, s->pinned[rec].acc, &s->pinned[rec].err);
            if (rc == FLB_OK) rc = flb_batch_remove(s->batch, q.slot);
            q.slot = -1;
            size_t used = 0;
            flb_batch_info(s->batch, nullptr, nullptr, &used, nullptr);
            s->st.pool_used = (int64_t)used;
        } else {
            f.nsamp = lattice_samples(q.lat);
            rc = lattice_enqueue_readout(q.lat, s->pinned[rec].acc, &s->pinned[rec].err);
            lattice_forget(q.lat);     // workspace reuse is ordered after the copy
            q.lat = nullptr;
            s->arena.release(q.off);
            s->running_lat -= 1;
            s->st.pool_used = (int64_t)s->arena.used();
        }
        if (rc != FLB_OK) return rc;
        s->live -= 1;
        s->st.running -= 1;
        s->st.finishing += 1;
        c.fin.push_back(f);
    }
    ce = cudaEventRecord(c.end, s->stream);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return FLB_ERR_CUDA;
    }
    s->inflight.push_back(std::move(c));
    return FLB_OK;
}

}  // namespace

extern "C" {

int flb_server_create(int32_t mode, int32_t basis, size_t pool_bytes, int32_t max_slots,
                      int32_t chunk_steps, void* stream, flb_server* out) {
    if (!out) return FLB_ERR_ARG;
    *out = nullptr;
    if ((mode != FLB_SERVE_BATCHED && mode != FLB_SERVE_PER_LATTICE) || max_slots < 1 ||
        max_slots > 16384 || chunk_steps < 1 || chunk_steps > 100000 || pool_bytes < 4096 ||
        (basis != FLB_BASIS_STANDARD && basis != FLB_BASIS_LOCAL && basis != FLB_BASIS_LOCAL_LUT))
        return FLB_ERR_ARG;
    flb_server s = new (std::nothrow) flb_server_s();
    if (!s) return FLB_ERR_OOM;
    s->mode = mode;
    s->basis = basis;
    s->max_slots = max_slots;
    s->chunk = chunk_steps;
    s->stream = (cudaStream_t)stream;
    s->t0 = std::chrono::steady_clock::now();
    std::memset(&s->st, 0, sizeof(s->st));
    int rc = FLB_OK;
    if (mode == FLB_SERVE_BATCHED) {
        rc = flb_batch_open(basis, max_slots, pool_bytes, stream, &s->batch);
        if (rc == FLB_OK) rc = flb_batch_set_graph(s->batch, chunk_steps);
        // narrow tiles waste least on a mix of small and uneven lattices
        if (rc == FLB_OK) rc = flb_batch_set_tile(s->batch, FLB_TILE_64x8);
    } else {
        void* p = nullptr;
        if (cudaMalloc(&p, pool_bytes) != cudaSuccess) {
            cudaGetLastError();
            rc = FLB_ERR_OOM;
        } else {
            s->pool = (char*)p;
            s->arena.reset(pool_bytes);
        }
    }
    const int nrec = max_slots * (kDepth + 1);
    if (rc == FLB_OK) {
        void* p = nullptr;
        if (cudaMallocHost(&p, sizeof(PinnedResult) * nrec) != cudaSuccess) {
            cudaGetLastError();
            rc = FLB_ERR_OOM;
        } else {
            s->pinned = (PinnedResult*)p;
            for (int k = nrec - 1; k >= 0; --k) s->free_records.push_back(k);
        }
    }
    if (rc != FLB_OK) {
        flb_server_destroy(s);
        return rc;
    }
    s->st.pool_size = (int64_t)pool_bytes;
    *out = s;
    return FLB_OK;
}

int flb_server_destroy(flb_server s) {
    if (!s) return FLB_OK;
    cudaError_t ce = cudaStreamSynchronize(s->stream);
    for (auto& kv : s->reqs)
        if (kv.second.lat) lattice_forget(kv.second.lat);
    int rc = s->batch ? flb_batch_destroy(s->batch) : FLB_OK;
    if (s->pool) cudaFree(s->pool);
    if (s->pinned) cudaFreeHost(s->pinned);
    for (auto& c : s->inflight) {
        cudaEventDestroy(c.start);
        cudaEventDestroy(c.end);
    }
    for (cudaEvent_t e : s->spare_events) cudaEventDestroy(e);
    delete s;
    if (ce != cudaSuccess) {
        cudaGetLastError();
        return FLB_ERR_CUDA;
    }
    return rc;
}

int flb_server_submit(flb_server s, const flb_params* p, int64_t nsteps, int64_t warmup,
                      int64_t every, int64_t* id) {
    if (!s || !p || !id || nsteps < 1 || nsteps >= INT_MAX || warmup < 0 || every < 0 ||
        warmup >= INT_MAX || every >= INT_MAX)
        return FLB_ERR_ARG;
    if (!valid_params(p) || p->precision != FLB_FP32 || p->basis != s->basis) return FLB_ERR_ARG;
    const size_t need = s->mode == FLB_SERVE_BATCHED ? flb_batch_replica_bytes(p)
                                                     : Arena::round_up(flb_workspace_bytes(p));
    if (need == 0) return FLB_ERR_ARG;
    if (need > (size_t)s->st.pool_size) return FLB_ERR_OOM;   // could never be admitted
    Req q;
    q.id = s->next_id++;
    q.p = *p;
    q.nsteps = nsteps;
    q.warmup = warmup;
    q.every = every;
    q.t_submit = now_s(s);
    s->reqs[q.id] = q;
    s->queue.push_back(q.id);
    s->st.submitted += 1;
    s->st.queued += 1;
    *id = q.id;
    return FLB_OK;
}

int flb_server_poll(flb_server s, int32_t wait, int32_t max_results, flb_result* results,
                    int32_t* n_results) {
    if (!s || max_results < 0 || (max_results > 0 && !results) || !n_results) return FLB_ERR_ARG;
    *n_results = 0;
    int rc = retire(s, false);
    if (rc == FLB_OK) rc = admit(s);
    while (rc == FLB_OK && (int)s->inflight.size() < kDepth && s->live > 0) {
        rc = enqueue_chunk(s);
        if (rc == FLB_OK) rc = admit(s);   // slots freed by requests ending in that chunk
    }
    if (rc == FLB_OK && wait && s->done.empty() && !s->inflight.empty()) {
        rc = retire(s, true);
        if (rc == FLB_OK) rc = admit(s);
        while (rc == FLB_OK && (int)s->inflight.size() < kDepth && s->live > 0) {
            rc = enqueue_chunk(s);
            if (rc == FLB_OK) rc = admit(s);
        }
    }
    int32_t n = 0;
    while (n < max_results && !s->done.empty()) {
        results[n++] = s->done.front();
        s->done.pop_front();
    }
    *n_results = n;
    return rc;
}

int flb_server_set_tile(flb_server s, int32_t tile) {
    if (!s) return FLB_ERR_ARG;
    if (s->mode != FLB_SERVE_BATCHED) return FLB_ERR_STATE;
    return flb_batch_set_tile(s->batch, tile);
}

int flb_server_stats(flb_server s, flb_serve_stats* out) {
    if (!s || !out) return FLB_ERR_ARG;
    *out = s->st;
    out->clock_s = now_s(s);
    out->pending_results = (int64_t)s->done.size();
    return FLB_OK;
}

}  // extern "C"
