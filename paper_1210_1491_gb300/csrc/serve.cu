// serve.cu -- continuous-batching request server over dtn_solve_patches.
//
// A worker thread owns `max_inflight` slots; each slot has its own stream, its
// own clone of the geometry object (so its workspace is private) and pinned
// staging buffers.  Queries wait in a FIFO.  Whenever a slot is free the worker
// merges queued queries into one batch (up to max_batch_patches patches and the
// memory budget), copies it to the device, enqueues the solve and the copies
// back, and records an event.  Queries that arrive while other batches run are
// admitted as soon as a slot and memory free up, so batches overlap on the
// device.  Every random number of a patch is fixed by its own patch id and the
// walk sums use per-node fixed-point scales, so a query's result does not
// depend on what it was batched with.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <thread>
#include <unordered_map>
#include <vector>

#include "dtn_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct QueryRec {
    int64_t n = 0;
    std::vector<double> centers, radius;
    std::vector<int32_t> nt, nph, nr, ns;
    std::vector<int64_t> walks;
    std::vector<uint32_t> pid;
    int64_t gamma_total = 0, panels_total = 0, matrix_total = 0;
    int64_t bytes = 0;
    std::vector<double> neumann, u;
    bool done = false;
    Clock::time_point t_submit, t_done;
};

template <typename T>
struct Pinned {
    T *p = nullptr;
    size_t n = 0;
    cudaError_t reserve(size_t k) {
        if (k <= n && p) return cudaSuccess;
        if (p) cudaFreeHost(p);
        p = nullptr;
        n = 0;
        cudaError_t e = cudaMallocHost((void **)&p, std::max<size_t>(k, 16) * sizeof(T));
        if (e == cudaSuccess) n = std::max<size_t>(k, 16);
        return e;
    }
    void release() {
        if (p) cudaFreeHost(p);
        p = nullptr;
        n = 0;
    }
};

struct Slot {
    dtn_geometry *g = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    dtn::DevBuf d_centers, d_radius, d_u, d_q;
    Pinned<double> h_centers, h_radius, h_u, h_q;
    std::vector<int32_t> nt, nph, nr, ns;
    std::vector<int64_t> walks;
    std::vector<uint32_t> pid;
    std::vector<int64_t> tickets;
    bool busy = false;
    int64_t bytes = 0;
};

int64_t estimate_bytes(int64_t gamma_total, int64_t panels_total, int64_t matrix_total) {
    // assembled matrix + LU scratch + node and panel arrays
    return matrix_total * 12 + gamma_total * 8 * 12 + panels_total * 8 * 24 + (1 << 16);
}

}  // namespace

struct dtn_server {
    dtn_server_config cfg{};
    dtn_geometry *geom = nullptr;
    std::vector<Slot> slots;
    std::deque<int64_t> queue;
    std::unordered_map<int64_t, QueryRec> recs;
    std::mutex mu;
    std::condition_variable cv;
    std::thread worker;
    bool stop = false;
    int64_t next_ticket = 1;
    int64_t mem_in_use = 0;
    int device = 0;
    dtn_status error = DTN_OK;
};

namespace {

dtn_status launch_batch(dtn_server *S, Slot &sl, const std::vector<int64_t> &tick) {
    int64_t n = 0, gt = 0, pt = 0;
    for (int64_t t : tick) {
        const QueryRec &q = S->recs[t];
        n += q.n;
        gt += q.gamma_total;
        pt += q.panels_total;
    }
    cudaError_t e;
    if ((e = sl.h_centers.reserve(3 * n)) != cudaSuccess || (e = sl.h_radius.reserve(n)) != cudaSuccess ||
        (e = sl.h_u.reserve(gt)) != cudaSuccess || (e = sl.h_q.reserve(pt)) != cudaSuccess ||
        (e = sl.d_centers.reserve(3 * n * 8)) != cudaSuccess || (e = sl.d_radius.reserve(n * 8)) != cudaSuccess ||
        (e = sl.d_u.reserve(gt * 8)) != cudaSuccess || (e = sl.d_q.reserve(pt * 8)) != cudaSuccess)
        return DTN_E_OUT_OF_MEMORY;
    sl.nt.clear(); sl.nph.clear(); sl.nr.clear(); sl.ns.clear(); sl.walks.clear(); sl.pid.clear();
    int64_t k = 0;
    for (int64_t t : tick) {
        const QueryRec &q = S->recs[t];
        std::memcpy(sl.h_centers.p + 3 * k, q.centers.data(), 3 * q.n * sizeof(double));
        std::memcpy(sl.h_radius.p + k, q.radius.data(), q.n * sizeof(double));
        sl.nt.insert(sl.nt.end(), q.nt.begin(), q.nt.end());
        sl.nph.insert(sl.nph.end(), q.nph.begin(), q.nph.end());
        sl.nr.insert(sl.nr.end(), q.nr.begin(), q.nr.end());
        sl.ns.insert(sl.ns.end(), q.ns.begin(), q.ns.end());
        sl.walks.insert(sl.walks.end(), q.walks.begin(), q.walks.end());
        sl.pid.insert(sl.pid.end(), q.pid.begin(), q.pid.end());
        k += q.n;
    }
    cudaMemcpyAsync(sl.d_centers.p, sl.h_centers.p, 3 * n * 8, cudaMemcpyHostToDevice, sl.s);
    cudaMemcpyAsync(sl.d_radius.p, sl.h_radius.p, n * 8, cudaMemcpyHostToDevice, sl.s);
    dtn_patch_batch b{};
    b.n_patches = n;
    b.centers = sl.d_centers.as<double>();
    b.radius = sl.h_radius.p;   // per-patch shape parameter: host array
    b.n_theta = sl.nt.data();
    b.n_phi = sl.nph.data();
    b.n_rings = sl.nr.data();
    b.n_sectors = sl.ns.data();
    b.walks_per_point = sl.walks.data();
    b.patch_ids = sl.pid.data();
    dtn_patch_result r{};
    r.u_gamma_mean = sl.d_u.as<double>();
    r.neumann = sl.d_q.as<double>();
    dtn_status st = dtn_solve_patches(sl.g, &b, &S->cfg.opts, &r, sl.s);
    if (st != DTN_OK) return st;
    cudaMemcpyAsync(sl.h_q.p, sl.d_q.p, pt * 8, cudaMemcpyDeviceToHost, sl.s);
    cudaMemcpyAsync(sl.h_u.p, sl.d_u.p, gt * 8, cudaMemcpyDeviceToHost, sl.s);
    if ((e = cudaEventRecord(sl.ev, sl.s)) != cudaSuccess) return DTN_E_CUDA;
    sl.tickets = tick;
    sl.busy = true;
    return DTN_OK;
}

void finish_batch(dtn_server *S, Slot &sl) {
    int64_t go = 0, po = 0;
    const auto now = Clock::now();
    for (int64_t t : sl.tickets) {
        QueryRec &q = S->recs[t];
        q.neumann.assign(sl.h_q.p + po, sl.h_q.p + po + q.panels_total);
        q.u.assign(sl.h_u.p + go, sl.h_u.p + go + q.gamma_total);
        po += q.panels_total;
        go += q.gamma_total;
        q.done = true;
        q.t_done = now;
    }
    sl.tickets.clear();
    sl.busy = false;
    S->mem_in_use -= sl.bytes;
    sl.bytes = 0;
}

void worker_main(dtn_server *S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        bool any_busy = false;
        for (Slot &sl : S->slots) {
            if (!sl.busy) continue;
            const cudaError_t q = cudaEventQuery(sl.ev);
            if (q == cudaSuccess) finish_batch(S, sl);
            else if (q != cudaErrorNotReady) { S->error = DTN_E_CUDA; finish_batch(S, sl); }
            else any_busy = true;
        }
        for (Slot &sl : S->slots) {
            if (sl.busy || S->queue.empty()) continue;
            std::vector<int64_t> tick;
            int64_t n = 0, bytes = 0;
            while (!S->queue.empty()) {
                const QueryRec &q = S->recs[S->queue.front()];
                const bool first = tick.empty();
                if (!first && n + q.n > S->cfg.max_batch_patches) break;
                if (S->mem_in_use + bytes + q.bytes > S->cfg.memory_budget && !(first && S->mem_in_use == 0)) break;
                tick.push_back(S->queue.front());
                S->queue.pop_front();
                n += q.n;
                bytes += q.bytes;
            }
            if (tick.empty()) break;
            sl.bytes = bytes;
            S->mem_in_use += bytes;
            const dtn_status st = launch_batch(S, sl, tick);
            if (st != DTN_OK) {
                S->error = st;
                for (int64_t t : tick) {
                    S->recs[t].done = true;
                    S->recs[t].t_done = Clock::now();
                }
                S->mem_in_use -= bytes;
                sl.bytes = 0;
                sl.busy = false;
            } else {
                any_busy = true;
            }
        }
        S->cv.notify_all();
        if (S->stop && S->queue.empty() && !any_busy) break;
        S->cv.wait_for(lk, std::chrono::microseconds(any_busy ? 50 : 500));
    }
}

}  // namespace

extern "C" {

dtn_status dtn_server_create(dtn_geometry *geom, const dtn_server_config *cfg, dtn_server **out) {
    if (!geom || !cfg || !out || cfg->max_inflight < 1 || cfg->max_batch_patches < 1) return DTN_E_INVALID_ARG;
    if (!geom->has_data) return DTN_E_INVALID_ARG;
    *out = nullptr;
    dtn_server *S = new dtn_server();
    S->cfg = *cfg;
    if (S->cfg.memory_budget <= 0) S->cfg.memory_budget = (int64_t)1 << 34;
    S->geom = geom;
    S->device = geom->device;
    S->slots.resize(cfg->max_inflight);
    for (Slot &sl : S->slots) {
        dtn_status st = dtn_create_geometry(&geom->host.desc, &sl.g);
        if (st == DTN_OK) st = dtn_set_dirichlet(sl.g, &geom->host.data);
        if (st != DTN_OK || cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess) {
            for (Slot &t : S->slots) {
                if (t.g) dtn_destroy_geometry(t.g);
                if (t.s) cudaStreamDestroy(t.s);
                if (t.ev) cudaEventDestroy(t.ev);
            }
            delete S;
            return st != DTN_OK ? st : DTN_E_CUDA;
        }
    }
    S->worker = std::thread(worker_main, S);
    *out = S;
    return DTN_OK;
}

dtn_status dtn_server_submit(dtn_server *S, const dtn_query *q, int64_t *ticket) {
    if (!S || !q || !ticket || q->n_patches < 1 || !q->centers || !q->radius || !q->n_theta || !q->n_phi ||
        !q->n_rings || !q->n_sectors || !q->walks_per_point || !q->patch_ids)
        return DTN_E_INVALID_ARG;
    QueryRec r;
    const int64_t n = q->n_patches;
    r.n = n;
    r.centers.assign(q->centers, q->centers + 3 * n);
    r.radius.assign(q->radius, q->radius + n);
    r.nt.assign(q->n_theta, q->n_theta + n);
    r.nph.assign(q->n_phi, q->n_phi + n);
    r.nr.assign(q->n_rings, q->n_rings + n);
    r.ns.assign(q->n_sectors, q->n_sectors + n);
    r.walks.assign(q->walks_per_point, q->walks_per_point + n);
    r.pid.assign(q->patch_ids, q->patch_ids + n);
    dtn_patch_batch b{};
    b.n_patches = n;
    b.n_theta = r.nt.data();
    b.n_phi = r.nph.data();
    b.n_rings = r.nr.data();
    b.n_sectors = r.ns.data();
    dtn_status st = dtn_query_patch_sizes(&b, &r.panels_total, &r.gamma_total, &r.matrix_total);
    if (st != DTN_OK) return st;
    for (int64_t p = 0; p < n; ++p)
        if (r.walks[p] < 2 || r.walks[p] > 0xFFFFFFFFll) return DTN_E_INVALID_ARG;
    r.bytes = estimate_bytes(r.gamma_total, r.panels_total, r.matrix_total);
    r.t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        const int64_t t = S->next_ticket++;
        S->recs.emplace(t, std::move(r));
        S->queue.push_back(t);
        *ticket = t;
    }
    S->cv.notify_all();
    return DTN_OK;
}

dtn_status dtn_server_poll(dtn_server *S, int64_t ticket, int32_t *done, double *neumann, double *u_mean,
                           double *latency_s) {
    if (!S || !done) return DTN_E_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->recs.find(ticket);
    if (it == S->recs.end()) return DTN_E_INVALID_ARG;
    QueryRec &q = it->second;
    *done = q.done ? 1 : 0;
    if (!q.done) return DTN_OK;
    if (S->error != DTN_OK && q.neumann.empty()) return S->error;
    if (neumann) std::memcpy(neumann, q.neumann.data(), q.neumann.size() * sizeof(double));
    if (u_mean) std::memcpy(u_mean, q.u.data(), q.u.size() * sizeof(double));
    if (latency_s) *latency_s = std::chrono::duration<double>(q.t_done - q.t_submit).count();
    return DTN_OK;
}

dtn_status dtn_server_drain(dtn_server *S) {
    if (!S) return DTN_E_INVALID_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    S->cv.wait(lk, [S] {
        if (!S->queue.empty()) return false;
        for (const Slot &sl : S->slots)
            if (sl.busy) return false;
        return true;
    });
    return S->error;
}

dtn_status dtn_server_destroy(dtn_server *S) {
    if (!S) return DTN_E_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (Slot &sl : S->slots) {
        if (sl.s) cudaStreamSynchronize(sl.s);
        sl.d_centers.release(); sl.d_radius.release(); sl.d_u.release(); sl.d_q.release();
        sl.h_centers.release(); sl.h_radius.release(); sl.h_u.release(); sl.h_q.release();
        if (sl.g) dtn_destroy_geometry(sl.g);
        if (sl.s) cudaStreamDestroy(sl.s);
        if (sl.ev) cudaEventDestroy(sl.ev);
    }
    delete S;
    return DTN_OK;
}

}  // extern "C"
