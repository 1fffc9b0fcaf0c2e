// Serving loop for several resident graphs (mf_server_* in mf.h).
//
// The method keeps the residual graph on the GPU between batches so that the
// max flow can be maintained indefinitely without host round trips
// (Sec. 1); this runtime serves update batches of several such graphs at
// once.  A scheduler thread admits queued requests as resources free up --
// continuous batching, not a queue drained one request at a time:
//   * one repair at a time per graph (a graph's batches are applied in
//     submission order);
//   * the persistent repair kernels of all requests in flight together use
//     at most `sm_slots` CTAs, so that their cooperative grids are co-resident
//     and their work overlaps on the device (each graph was created with a
//     grid of its own size, mf_options.grid_blocks);
//   * the device staging of the batches in flight stays within the HBM
//     budget left after the resident graphs;
//   * a repair's grid is sized to its batch (the graph's full grid, half or
//     a quarter of it; see grid_class), so that the CTAs left beside a large
//     repair admit small ones.
// Each graph has its own stream; a request is three copies of its batch into
// the graph's device staging, the repair (the policy kernel when the graph
// uses one, and the persistent kernel, both reading the batch size from the
// device), captured once per graph and grid size in a CUDA graph and
// replayed, and the copy of status and value back into pinned host memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "mf.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    int64_t ticket;
    int graph;
    std::vector<int32_t> ids, caps;
    int32_t flags;
    Clock::time_point t_submit;
};

struct Result {
    bool done = false;
    int32_t code = MF_OK;
    int64_t flow = 0;
    double latency_us = 0;
};

// Grid classes of a repair: the graph's full grid, half and a quarter.
constexpr int kGridClasses = 3;

// The class of a request: full for recomputes and batches above 20,000
// entries, half above 2,000, a quarter below (the repair of a small batch on
// a small graph is latency bound: a smaller grid costs it little and frees
// SMs), but never smaller than the graph's size allows (max_class): every
// repair runs at least one BFS over the whole graph, so on a graph of 2^21
// vertices or more a smaller grid only makes it slower.
int grid_class(int64_t k, int32_t flags, int max_class) {
    if ((flags & MF_RECOMPUTE) || k > 20000) return 0;
    const int c = k > 2000 ? 1 : 2;
    return c < max_class ? c : max_class;
}

int graph_max_class(int32_t n) { return n >= (1 << 21) ? 0 : n >= (1 << 19) ? 1 : 2; }

struct Slot {
    mf_graph *g = nullptr;
    int grids[kGridClasses] = {0, 0, 0};   // CTAs of each grid class
    int max_class = 2;                     // smallest class the graph's size allows
    int64_t max_batch = 0;
    cudaStream_t stream = nullptr;
    int32_t *h_stage = nullptr;   // pinned: [k, pad x 3, ids[max_batch], caps[max_batch]]
    int32_t *d_stage = nullptr;   // device copy of the same layout
    int64_t *h_result = nullptr;  // pinned: status, value
    cudaEvent_t done = nullptr;
    cudaGraphExec_t exec[kGridClasses] = {nullptr, nullptr, nullptr};   // repair per grid class
    cudaGraphExec_t exec_recompute = nullptr;                          // (full grid)
    bool busy = false;
    Request cur;
    int64_t cur_bytes = 0;
    int cur_grid = 0;
};

}  // namespace

struct mf_server {
    mf_server_options opt{};
    int dev = 0;
    std::vector<Slot> slots;
    std::deque<Request> queue;
    std::unordered_map<int64_t, Result> results;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    std::atomic<bool> stop{false};
    int64_t next_ticket = 1;
    int64_t resident_bytes = 0;
    int sm_in_use = 0;
    int64_t staging_in_use = 0;
    int inflight = 0;
    // statistics
    int64_t submitted = 0, completed = 0, failed = 0;
    int max_inflight = 0;
    int captured = 0;
    int64_t replays = 0, direct = 0;
    std::vector<double> latencies;
    std::vector<char> held;   // per graph: a request of it is waiting (admission scan)
    Clock::time_point t_first{}, t_last{};
    bool any = false;
    std::string err;
};

namespace {

int64_t stage_words(int64_t max_batch) { return 4 + 2 * max_batch; }

// Capture the repair of one slot: policy (if any) + persistent kernel +
// result copy, reading the batch size and arrays from the device staging.
bool capture(Slot &S, int32_t flags, cudaGraphExec_t *exec) {
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(S.stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const int rc1 = mf_apply_updates_dev(S.g, S.d_stage, S.max_batch, S.d_stage + 4, S.d_stage + 4 + S.max_batch,
                                         flags, S.stream);
    const int rc2 = mf_flow_value_async(S.g, S.h_result, S.stream);
    const cudaError_t e = cudaStreamEndCapture(S.stream, &graph);
    bool ok = rc1 == MF_OK && rc2 == MF_OK && e == cudaSuccess && graph;
    if (ok && cudaGraphInstantiate(exec, graph, 0) != cudaSuccess) ok = false;
    if (graph) cudaGraphDestroy(graph);
    if (!ok) {
        cudaGetLastError();
        *exec = nullptr;
    }
    return ok;
}

int code_of_status(int64_t bits) {
    const int32_t st = int32_t(bits & 0xffffffff);
    if (st & 16) return MF_ECHECK;
    if (st & (2 | 4 | 8)) return MF_ETIMEOUT;
    if (st & 1) return MF_EINVAL;
    return MF_OK;
}

void launch_request(mf_server *S, Slot &sl, Request &&r) {
    const int64_t k = int64_t(r.ids.size());
    sl.h_stage[0] = int32_t(k);
    std::memcpy(sl.h_stage + 4, r.ids.data(), size_t(k) * 4);
    std::memcpy(sl.h_stage + 4 + sl.max_batch, r.caps.data(), size_t(k) * 4);
    cudaMemcpyAsync(sl.d_stage, sl.h_stage, 16, cudaMemcpyHostToDevice, sl.stream);
    if (k > 0) {
        cudaMemcpyAsync(sl.d_stage + 4, sl.h_stage + 4, size_t(k) * 4, cudaMemcpyHostToDevice, sl.stream);
        cudaMemcpyAsync(sl.d_stage + 4 + sl.max_batch, sl.h_stage + 4 + sl.max_batch, size_t(k) * 4,
                        cudaMemcpyHostToDevice, sl.stream);
    }
    const bool rec = (r.flags & MF_RECOMPUTE) != 0;
    const int gc = grid_class(k, r.flags, sl.max_class);
    cudaGraphExec_t ex = rec ? sl.exec_recompute : sl.exec[gc];
    int rc = MF_OK;
    if (ex && !(r.flags & MF_DELTA)) {
        if (cudaGraphLaunch(ex, sl.stream) != cudaSuccess) rc = MF_ECUDA;
        S->replays += 1;
    } else {
        mf_set_grid_blocks(sl.g, sl.grids[gc]);
        rc = mf_apply_updates_dev(sl.g, sl.d_stage, sl.max_batch, sl.d_stage + 4, sl.d_stage + 4 + sl.max_batch,
                                  r.flags & (MF_DELTA | MF_RECOMPUTE), sl.stream);
        if (rc == MF_OK) rc = mf_flow_value_async(sl.g, sl.h_result, sl.stream);
        S->direct += 1;
    }
    if (rc != MF_OK) {
        cudaGetLastError();
        sl.h_result[0] = 4;   // reported as a device failure
    }
    cudaEventRecord(sl.done, sl.stream);
    sl.busy = true;
    sl.cur_bytes = 8 * k;
    sl.cur_grid = sl.grids[gc];
    sl.cur = std::move(r);
    S->sm_in_use += sl.cur_grid;
    S->staging_in_use += sl.cur_bytes;
    S->inflight += 1;
    S->max_inflight = std::max(S->max_inflight, S->inflight);
}

void worker_loop(mf_server *S) {
    cudaSetDevice(S->dev);
    std::unique_lock<std::mutex> lk(S->mu);
    while (!S->stop) {
        bool progress = false;
        // completions
        for (auto &sl : S->slots) {
            if (!sl.busy) continue;
            if (cudaEventQuery(sl.done) != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            Result &res = S->results[sl.cur.ticket];
            res.done = true;
            res.code = code_of_status(sl.h_result[0]);
            res.flow = sl.h_result[1];
            const auto now = Clock::now();
            res.latency_us = std::chrono::duration<double, std::micro>(now - sl.cur.t_submit).count();
            S->latencies.push_back(res.latency_us);
            S->t_last = now;
            S->completed += 1;
            if (res.code != MF_OK) S->failed += 1;
            sl.busy = false;
            S->sm_in_use -= sl.cur_grid;
            S->staging_in_use -= sl.cur_bytes;
            S->inflight -= 1;
            progress = true;
        }
        if (progress) S->cv_done.notify_all();
        // admissions, in arrival order; a request whose graph is busy or that
        // does not fit waits while later ones of other graphs may go ahead.
        // A graph's own requests keep their order (batches carry absolute
        // capacities): once one of them waits, the later ones wait too, even
        // when their smaller grid would fit.
        S->held.assign(S->slots.size(), 0);
        for (auto it = S->queue.begin(); it != S->queue.end();) {
            Slot &sl = S->slots[size_t(it->graph)];
            const int64_t bytes = 8 * int64_t(it->ids.size());
            const int grid = sl.grids[grid_class(int64_t(it->ids.size()), it->flags, sl.max_class)];
            const bool fits = !S->held[size_t(it->graph)] && !sl.busy && S->sm_in_use + grid <= S->opt.sm_slots &&
                              S->staging_in_use + bytes <= S->opt.hbm_budget_bytes - S->resident_bytes;
            if (!fits) {
                S->held[size_t(it->graph)] = 1;
                ++it;
                continue;
            }
            Request r = std::move(*it);
            it = S->queue.erase(it);
            launch_request(S, sl, std::move(r));
            progress = true;
        }
        if (!progress) {
            if (S->inflight > 0) {
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(20));
                lk.lock();
            } else {
                S->cv_work.wait_for(lk, std::chrono::milliseconds(50));
            }
        }
    }
}

}  // namespace

extern "C" {

int mf_server_options_default(mf_server_options *opt) {
    if (!opt) return MF_EINVAL;
    std::memset(opt, 0, sizeof(*opt));
    opt->use_cuda_graphs = 1;
    return MF_OK;
}

int mf_server_create(const mf_server_options *opt, mf_server **out) {
    if (!out) return MF_EINVAL;
    *out = nullptr;
    mf_server *S = new (std::nothrow) mf_server();
    if (!S) return MF_ENOMEM;
    if (opt) S->opt = *opt;
    else mf_server_options_default(&S->opt);
    if (cudaGetDevice(&S->dev) != cudaSuccess) {
        delete S;
        return MF_ECUDA;
    }
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, S->dev);
    if (S->opt.sm_slots <= 0) S->opt.sm_slots = sms;
    if (S->opt.hbm_budget_bytes <= 0) {
        size_t fr = 0, tot = 0;
        cudaMemGetInfo(&fr, &tot);
        S->opt.hbm_budget_bytes = int64_t(tot);
    }
    S->worker = std::thread(worker_loop, S);
    *out = S;
    return MF_OK;
}

int mf_server_add_graph(mf_server *S, mf_graph *g, int64_t max_batch, int32_t *index) {
    if (!S || !g || !index || max_batch <= 0) return MF_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    int64_t bytes = 0;
    int32_t grid = 0;
    mf_device_bytes(g, &bytes);
    mf_grid_blocks(g, &grid);
    const int64_t need = bytes + 4 * stage_words(max_batch);
    if (grid > S->opt.sm_slots) {
        S->err = "graph grid larger than the SM slots";
        return MF_EINVAL;
    }
    if (S->resident_bytes + need > S->opt.hbm_budget_bytes) {
        S->err = "graph does not fit the HBM budget";
        return MF_ENOMEM;
    }
    Slot sl;
    sl.g = g;
    sl.grids[0] = grid;
    sl.grids[1] = std::max(1, grid / 2);
    sl.grids[2] = std::max(1, grid / 4);
    int32_t n = 0;
    mf_sizes(g, &n, nullptr, nullptr);
    sl.max_class = graph_max_class(n);
    sl.max_batch = max_batch;
    if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMallocHost(&sl.h_stage, size_t(4 * stage_words(max_batch))) != cudaSuccess ||
        cudaMalloc(&sl.d_stage, size_t(4 * stage_words(max_batch))) != cudaSuccess ||
        cudaMallocHost(&sl.h_result, 16) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return MF_ECUDA;
    }
    cudaMemset(sl.d_stage, 0, 16);
    // size the graph's batch staging outside any capture with an empty batch
    // (a repair that finds nothing to do), then capture
    int rc = mf_apply_updates_dev(g, sl.d_stage, max_batch, sl.d_stage + 4, sl.d_stage + 4 + max_batch, 0,
                                  sl.stream);
    if (rc == MF_OK) rc = mf_flow_value_async(g, sl.h_result, sl.stream);
    cudaStreamSynchronize(sl.stream);
    if (rc != MF_OK || code_of_status(sl.h_result[0]) != MF_OK) {
        S->err = "graph could not be solved on its server stream";
        return rc != MF_OK ? rc : MF_ECUDA;
    }
    if (S->opt.use_cuda_graphs) {
        // one capture per grid class (the grid size is part of the launch
        // captured), the recompute on the full grid
        for (int c = sl.max_class; c >= 0; --c) {
            if (c < sl.max_class && sl.grids[c] == sl.grids[c + 1]) {
                sl.exec[c] = sl.exec[c + 1];   // the same size: share the capture
                continue;
            }
            mf_set_grid_blocks(g, sl.grids[c]);
            if (capture(sl, 0, &sl.exec[c])) S->captured += 1;
        }
        if (capture(sl, MF_RECOMPUTE, &sl.exec_recompute)) S->captured += 1;
    }
    S->resident_bytes += need;
    S->slots.push_back(sl);
    *index = int32_t(S->slots.size() - 1);
    return MF_OK;
}

int mf_server_submit(mf_server *S, int32_t graph, int64_t k, const int32_t *edge_id, const int32_t *new_cap,
                     int32_t flags, int64_t *ticket) {
    if (!S || !ticket || k < 0 || (k > 0 && (!edge_id || !new_cap))) return MF_EINVAL;
    if (flags & ~(MF_DELTA | MF_RECOMPUTE)) return MF_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    if (graph < 0 || size_t(graph) >= S->slots.size()) return MF_EINVAL;
    if (k > S->slots[size_t(graph)].max_batch) return MF_EINVAL;
    Request r;
    r.ticket = S->next_ticket++;
    r.graph = graph;
    r.ids.assign(edge_id, edge_id + k);
    r.caps.assign(new_cap, new_cap + k);
    r.flags = flags;
    r.t_submit = Clock::now();
    if (!S->any) {
        S->t_first = r.t_submit;
        S->any = true;
    }
    *ticket = r.ticket;
    S->results[r.ticket] = Result{};
    S->queue.push_back(std::move(r));
    S->submitted += 1;
    S->cv_work.notify_one();
    return MF_OK;
}

int mf_server_poll(mf_server *S, int64_t ticket, int32_t *done, int64_t *flow, int32_t *code, double *latency_us) {
    if (!S || !done) return MF_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->results.find(ticket);
    if (it == S->results.end()) return MF_EINVAL;
    *done = it->second.done ? 1 : 0;
    if (flow) *flow = it->second.flow;
    if (code) *code = it->second.code;
    if (latency_us) *latency_us = it->second.latency_us;
    return MF_OK;
}

int mf_server_drain(mf_server *S) {
    if (!S) return MF_EINVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    S->cv_work.notify_one();
    S->cv_done.wait(lk, [S] { return S->completed == S->submitted; });
    return MF_OK;   // each request's own code: mf_server_poll; failures are counted in the stats
}

int mf_server_stats_get(mf_server *S, mf_server_stats *out) {
    if (!S || !out) return MF_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    std::memset(out, 0, sizeof(*out));
    out->submitted = S->submitted;
    out->completed = S->completed;
    out->failed = S->failed;
    out->max_inflight = S->max_inflight;
    out->graphs = int32_t(S->slots.size());
    out->captured_graphs = S->captured;
    out->replays = S->replays;
    out->direct_launches = S->direct;
    std::vector<double> l = S->latencies;
    if (!l.empty()) {
        std::sort(l.begin(), l.end());
        auto q = [&](double p) { return l[std::min(l.size() - 1, size_t(p * double(l.size() - 1) + 0.5))]; };
        out->p50_us = q(0.50);
        out->p99_us = q(0.99);
        double s = 0;
        for (double x : l) s += x;
        out->mean_us = s / double(l.size());
        out->makespan_s = std::chrono::duration<double>(S->t_last - S->t_first).count();
    }
    return MF_OK;
}

void mf_server_reset_stats(mf_server *S) {
    if (!S) return;
    std::lock_guard<std::mutex> lk(S->mu);
    S->latencies.clear();
    S->replays = S->direct = 0;
    S->submitted -= S->completed;
    S->completed = 0;
    S->failed = 0;
    S->max_inflight = S->inflight;
    S->any = false;
}

void mf_server_destroy(mf_server *S) {
    if (!S) return;
    {
        std::unique_lock<std::mutex> lk(S->mu);
        S->cv_done.wait(lk, [S] { return S->completed == S->submitted; });
        S->stop = true;
        S->cv_work.notify_all();
    }
    S->worker.join();
    for (auto &sl : S->slots) {
        cudaStreamSynchronize(sl.stream);
        mf_set_stream(sl.g, nullptr);   // the graph outlives the server's stream
        mf_set_grid_blocks(sl.g, sl.grids[0]);
        for (int c = 0; c < kGridClasses; ++c)
            if (sl.exec[c] && (c == kGridClasses - 1 || sl.exec[c] != sl.exec[c + 1]))
                cudaGraphExecDestroy(sl.exec[c]);   // (classes past max_class were never captured)
        if (sl.exec_recompute) cudaGraphExecDestroy(sl.exec_recompute);
        cudaEventDestroy(sl.done);
        cudaFreeHost(sl.h_stage);
        cudaFreeHost(sl.h_result);
        cudaFree(sl.d_stage);
        cudaStreamDestroy(sl.stream);
    }
    delete S;
}

}  // extern "C"
