// serve.cu -- continuous-batching request server over dtn_solve_patches.
//
// A worker thread owns `max_inflight` slots; each slot has its own stream, its
// own clone of the geometry object (so its workspace is private) and pinned
// staging buffers.  Queries wait in a FIFO.  Whenever a slot is free the worker
// merges queued queries into one batch (up to max_batch_patches patches and
// what device memory allows), copies it to the device, enqueues the solve and
// the copies back, and records events around it.  Queries that arrive while
// other batches run are admitted as soon as a slot and memory free up, so
// batches overlap on the device; with split_sms each slot's walk launch takes
// a share of the resident walk blocks, so the walks of different slots run side
// by side instead of one after the other.  Every random number of a patch is
// fixed by its own patch id and the walk sums use per-node fixed-point scales,
// so a query's result does not depend on what it was batched with.
//
// Admission by device memory: the budget is the device's free memory at
// creation less a reserve (or the configured budget, if smaller).  The ledger
// holds what each slot's workspace holds now (its buffers only grow, stream-
// ordered, and are kept for the next batch) and, for a batch about to start,
// the workspace its solve reserves (computed from its layout); a batch starts
// only if the slots' total stays within the budget.  Idle slots give their
// workspace back when a batch would not fit otherwise; a query that cannot fit
// even in an empty server fails with DTN_E_OUT_OF_MEMORY.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <thread>
#include <unordered_map>
#include <utility>
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
    int64_t bytes = 0;                 // workspace its solve reserves alone
    std::vector<double> neumann, u;
    std::vector<int32_t> patch_status;
    dtn_status status = DTN_OK;        // the query's result status (dtn_server_poll)
    bool filled = false;               // neumann / u / patch_status hold the result
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
        const size_t want = std::max<size_t>(k + k / 2, 16);
        cudaError_t e = cudaMallocHost((void **)&p, want * sizeof(T));
        if (e == cudaSuccess) n = want;
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
    cudaEvent_t ev_start = nullptr, ev_end = nullptr;   // around a batch, on s
    dtn_solve_opts opts{};
    dtn::DevBuf d_centers, d_u, d_q, d_st;
    Pinned<double> h_centers, h_radius, h_u, h_q;
    Pinned<int32_t> h_st;
    std::vector<int32_t> nt, nph, nr, ns;
    std::vector<int64_t> walks;
    std::vector<uint32_t> pid;
    std::vector<int64_t> tickets;
    bool busy = false;
    int64_t need = 0;   // ledger entry while busy: max(held, the batch's workspace)
};

int64_t slot_held(const Slot &sl) {
    return (int64_t)(dtn::workspace_bytes(sl.g) + sl.d_centers.bytes + sl.d_u.bytes + sl.d_q.bytes +
                     sl.d_st.bytes);
}

// staging the batch needs on the device besides the solve's workspace
int64_t staging_bytes(int64_t n, int64_t gt, int64_t pt) { return (3 * n + gt + pt) * 8 + n * 4 + 4096; }

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
    int device = 0;
    dtn_status error = DTN_OK;
    bool caps = false;                 // ball regions: cap patches (workspace estimate)
    int64_t budget = 0, device_free = 0, peak_held = 0;
    int64_t batches = 0, queries_done = 0, rejected = 0;
    cudaEvent_t epoch = nullptr;
    std::vector<std::pair<float, float>> intervals;   // device ms of finished batches, from epoch
};

namespace {

int64_t ledger(const dtn_server *S, const Slot *except) {
    int64_t t = 0;
    for (const Slot &sl : S->slots)
        if (&sl != except) t += sl.busy ? std::max(sl.need, slot_held(sl)) : slot_held(sl);
    return t;
}

void finish_query(dtn_server *S, QueryRec &q, dtn_status st) {
    q.status = st;
    q.done = true;
    q.t_done = Clock::now();
    S->queries_done += 1;
}

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
        (e = sl.h_st.reserve(n)) != cudaSuccess || (e = sl.d_centers.reserve(3 * n * 8, sl.s)) != cudaSuccess ||
        (e = sl.d_u.reserve(gt * 8, sl.s)) != cudaSuccess || (e = sl.d_q.reserve(pt * 8, sl.s)) != cudaSuccess ||
        (e = sl.d_st.reserve(n * 4, sl.s)) != cudaSuccess)
        return dtn::to_status(e);
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
    if ((e = cudaEventRecord(sl.ev_start, sl.s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(sl.d_centers.p, sl.h_centers.p, 3 * n * 8, cudaMemcpyHostToDevice, sl.s)) != cudaSuccess)
        return dtn::to_status(e);
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
    r.patch_status = sl.d_st.as<int32_t>();
    dtn_status st = dtn_solve_patches(sl.g, &b, &sl.opts, &r, sl.s);
    if (st != DTN_OK) return st;
    if ((e = cudaMemcpyAsync(sl.h_q.p, sl.d_q.p, pt * 8, cudaMemcpyDeviceToHost, sl.s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(sl.h_u.p, sl.d_u.p, gt * 8, cudaMemcpyDeviceToHost, sl.s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(sl.h_st.p, sl.d_st.p, n * 4, cudaMemcpyDeviceToHost, sl.s)) != cudaSuccess ||
        (e = cudaEventRecord(sl.ev_end, sl.s)) != cudaSuccess)
        return dtn::to_status(e);
    sl.tickets = tick;
    sl.busy = true;
    return DTN_OK;
}

// A batch has completed (ok) or its stream reported an error (!ok: its queries
// get DTN_E_CUDA and no result).
void finish_batch(dtn_server *S, Slot &sl, bool ok) {
    int64_t go = 0, po = 0, ko = 0;
    for (int64_t t : sl.tickets) {
        QueryRec &q = S->recs[t];
        dtn_status st = ok ? DTN_OK : DTN_E_CUDA;
        if (ok) {
            q.neumann.assign(sl.h_q.p + po, sl.h_q.p + po + q.panels_total);
            q.u.assign(sl.h_u.p + go, sl.h_u.p + go + q.gamma_total);
            q.patch_status.assign(sl.h_st.p + ko, sl.h_st.p + ko + q.n);
            q.filled = true;
            for (int32_t v : q.patch_status)
                if (v != DTN_OK) {
                    st = (dtn_status)v;
                    break;
                }
        }
        po += q.panels_total;
        go += q.gamma_total;
        ko += q.n;
        finish_query(S, q, st);
    }
    if (ok) {
        float t0 = 0.f, t1 = 0.f;
        if (cudaEventElapsedTime(&t0, S->epoch, sl.ev_start) == cudaSuccess &&
            cudaEventElapsedTime(&t1, S->epoch, sl.ev_end) == cudaSuccess)
            S->intervals.emplace_back(t0, t1);
        else
            cudaGetLastError();
    }
    S->batches += 1;
    sl.tickets.clear();
    sl.busy = false;
    sl.need = 0;
    S->peak_held = std::max(S->peak_held, ledger(S, nullptr));
}

void trim_idle(dtn_server *S, Slot *keep) {
    for (Slot &sl : S->slots) {
        if (&sl == keep || sl.busy) continue;
        dtn_release_workspace(sl.g);
        sl.d_centers.release(); sl.d_u.release(); sl.d_q.release(); sl.d_st.release();
    }
}

void worker_main(dtn_server *S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        bool any_busy = false;
        for (Slot &sl : S->slots) {
            if (!sl.busy) continue;
            const cudaError_t q = cudaEventQuery(sl.ev_end);
            if (q == cudaSuccess) {
                finish_batch(S, sl, true);
            } else if (q != cudaErrorNotReady) {
                dtn::set_cuda_error(q);
                cudaGetLastError();
                S->error = DTN_E_CUDA;
                finish_batch(S, sl, false);
            } else {
                any_busy = true;
            }
        }
        for (Slot &sl : S->slots) {
            if (sl.busy || S->queue.empty()) continue;
            std::vector<int64_t> tick;
            int64_t n = 0, gt = 0, pt = 0, bytes = 0;
            const int64_t held = slot_held(sl);
            while (!S->queue.empty()) {
                QueryRec &q = S->recs[S->queue.front()];
                const int64_t others = ledger(S, &sl);
                const int64_t nb = bytes + q.bytes;
                const int64_t need =
                    std::max(held, nb + nb / 2 + staging_bytes(n + q.n, gt + q.gamma_total, pt + q.panels_total));
                if (!tick.empty() && n + q.n > S->cfg.max_batch_patches) break;
                if (others + need > S->budget) {
                    if (!tick.empty()) break;
                    // not even alone in this slot: free idle slots, else wait for
                    // busy ones, else the query can never run
                    bool busy_other = false;
                    for (const Slot &o : S->slots) busy_other |= (o.busy && &o != &sl);
                    if (busy_other) break;
                    if (ledger(S, &sl) > 0) {
                        trim_idle(S, &sl);
                        continue;
                    }
                    S->queue.pop_front();
                    S->rejected += 1;
                    finish_query(S, q, DTN_E_OUT_OF_MEMORY);
                    continue;
                }
                tick.push_back(S->queue.front());
                S->queue.pop_front();
                n += q.n;
                gt += q.gamma_total;
                pt += q.panels_total;
                bytes = nb;
            }
            if (tick.empty()) continue;
            sl.need = std::max(held, bytes + bytes / 2 + staging_bytes(n, gt, pt));
            const dtn_status st = launch_batch(S, sl, tick);
            if (st != DTN_OK) {
                for (int64_t t : tick) finish_query(S, S->recs[t], st);
                sl.tickets.clear();
                sl.busy = false;
                sl.need = 0;
                if (st == DTN_E_CUDA) S->error = st;
            } else {
                any_busy = true;
            }
            S->peak_held = std::max(S->peak_held, ledger(S, nullptr));
        }
        S->cv.notify_all();
        if (S->stop && S->queue.empty() && !any_busy) break;
        S->cv.wait_for(lk, std::chrono::microseconds(any_busy ? 50 : 500));
    }
}

void destroy_slots(dtn_server *S) {
    for (Slot &sl : S->slots) {
        if (sl.s) cudaStreamSynchronize(sl.s);
        sl.d_centers.release(); sl.d_u.release(); sl.d_q.release(); sl.d_st.release();
        sl.h_centers.release(); sl.h_radius.release(); sl.h_u.release(); sl.h_q.release(); sl.h_st.release();
        if (sl.g) dtn_destroy_geometry(sl.g);
        if (sl.s) cudaStreamDestroy(sl.s);
        if (sl.ev_start) cudaEventDestroy(sl.ev_start);
        if (sl.ev_end) cudaEventDestroy(sl.ev_end);
    }
    if (S->epoch) cudaEventDestroy(S->epoch);
}

}  // namespace

extern "C" {

dtn_status dtn_server_create(dtn_geometry *geom, const dtn_server_config *cfg, dtn_server **out) {
    if (!geom || !cfg || !out || cfg->max_inflight < 1 || cfg->max_batch_patches < 1) return DTN_E_INVALID_ARG;
    if (cfg->memory_budget < 0 || !geom->has_data) return DTN_E_INVALID_ARG;
    if (dtn::wrong_device(geom)) return DTN_E_INVALID_ARG;
    *out = nullptr;
    size_t free_b = 0, total_b = 0;
    cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
    if (e != cudaSuccess) return dtn::to_status(e);
    dtn_server *S = new dtn_server();
    S->cfg = *cfg;
    S->geom = geom;
    S->device = geom->device;
    S->caps = (geom->dg.kind == dtn::kBall || geom->dg.kind == dtn::kBallExterior);
    // the budget: free memory now, less a reserve for the caller and the runtime
    const int64_t reserve = std::max<int64_t>((int64_t)1 << 30, (int64_t)(total_b / 20));
    S->device_free = (int64_t)free_b;
    S->budget = std::max<int64_t>(0, (int64_t)free_b - reserve);
    if (cfg->memory_budget > 0) S->budget = std::min(S->budget, cfg->memory_budget);
    S->slots.resize(cfg->max_inflight);
    int split_bps = 0;
    if (cfg->split_sms && cfg->max_inflight > 1 && cfg->opts.wos_blocks_per_sm == 0) {
        const int resident = dtn::wos_resident_blocks(geom, cfg->opts.prec);
        split_bps = std::max(1, resident / cfg->max_inflight);
    }
    dtn_status st = DTN_OK;
    for (Slot &sl : S->slots) {
        sl.opts = cfg->opts;
        if (split_bps) sl.opts.wos_blocks_per_sm = split_bps;
        st = dtn_create_geometry(&geom->host.desc, &sl.g);
        if (st == DTN_OK) st = dtn_set_dirichlet(sl.g, &geom->host.data);
        if (st == DTN_OK && (cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking) != cudaSuccess ||
                             cudaEventCreate(&sl.ev_start) != cudaSuccess || cudaEventCreate(&sl.ev_end) != cudaSuccess))
            st = DTN_E_CUDA;
        if (st != DTN_OK) break;
    }
    if (st == DTN_OK && (cudaEventCreate(&S->epoch) != cudaSuccess || cudaEventRecord(S->epoch, S->slots[0].s) != cudaSuccess ||
                         cudaEventSynchronize(S->epoch) != cudaSuccess))
        st = DTN_E_CUDA;
    if (st != DTN_OK) {
        destroy_slots(S);
        delete S;
        return st;
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
    for (int64_t p = 0; p < n; ++p)
        if (r.walks[p] < 2 || r.walks[p] > 0xFFFFFFFFll || !(r.radius[p] > 0.0)) return DTN_E_INVALID_ARG;
    dtn_patch_batch b{};
    b.n_patches = n;
    b.radius = r.radius.data();
    b.n_theta = r.nt.data();
    b.n_phi = r.nph.data();
    b.n_rings = r.nr.data();
    b.n_sectors = r.ns.data();
    b.walks_per_point = r.walks.data();
    b.patch_ids = r.pid.data();
    dtn_status st = dtn_query_patch_sizes(&b, &r.panels_total, &r.gamma_total, &r.matrix_total);
    if (st != DTN_OK) return st;
    r.bytes = (int64_t)dtn::solve_workspace_bytes(&b, &S->cfg.opts, S->caps);
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
                           double *latency_s, int32_t *patch_status) {
    if (!S || !done) return DTN_E_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->recs.find(ticket);
    if (it == S->recs.end()) return DTN_E_INVALID_ARG;
    QueryRec &q = it->second;
    *done = q.done ? 1 : 0;
    if (!q.done) return DTN_OK;
    if (latency_s) *latency_s = std::chrono::duration<double>(q.t_done - q.t_submit).count();
    if (q.filled) {
        if (neumann) std::memcpy(neumann, q.neumann.data(), q.neumann.size() * sizeof(double));
        if (u_mean) std::memcpy(u_mean, q.u.data(), q.u.size() * sizeof(double));
        if (patch_status) std::memcpy(patch_status, q.patch_status.data(), q.patch_status.size() * sizeof(int32_t));
    }
    return q.status;
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

dtn_status dtn_server_stats(dtn_server *S, dtn_server_info *out) {
    if (!S || !out) return DTN_E_INVALID_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    dtn_server_info I{};
    I.budget_bytes = S->budget;
    I.device_free_bytes = S->device_free;
    I.held_bytes = ledger(S, nullptr);
    I.peak_held_bytes = S->peak_held;
    I.batches = S->batches;
    I.queries = S->queries_done;
    I.rejected = S->rejected;
    // sweep over the finished batches' device intervals
    std::vector<std::pair<float, int>> ev;
    ev.reserve(2 * S->intervals.size());
    for (const auto &iv : S->intervals) {
        ev.emplace_back(iv.first, +1);
        ev.emplace_back(iv.second, -1);
    }
    std::sort(ev.begin(), ev.end(), [](const std::pair<float, int> &a, const std::pair<float, int> &b) {
        return a.first < b.first || (a.first == b.first && a.second < b.second);   // ends before starts
    });
    int cur = 0;
    double last = 0.0;
    for (const auto &e : ev) {
        if (cur >= 1) I.busy_ms += e.first - last;
        if (cur >= 2) I.overlap_ms += e.first - last;
        cur += e.second;
        last = e.first;
        I.max_concurrent = std::max(I.max_concurrent, cur);
    }
    *out = I;
    return DTN_OK;
}

dtn_status dtn_server_destroy(dtn_server *S) {
    if (!S) return DTN_E_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv.notify_all();
    if (S->worker.joinable()) S->worker.join();
    destroy_slots(S);
    delete S;
    return DTN_OK;
}

}  // extern "C"
