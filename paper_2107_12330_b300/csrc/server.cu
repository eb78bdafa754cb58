// server.cu -- serving loop: resident graphs, continuous batching of survey
// requests under a scratch-memory budget.
//
// Requests queue on the host.  A dispatcher thread admits them in arrival
// order while fewer than max_inflight are on the device and their scratch
// (the device accumulator of the result) fits under the budget; each admitted
// request is launched on one of several CUDA streams, so requests of different
// graphs, kinds and windows overlap on the GPU.  A request on a large graph
// (kLargeEdges edges or more) already fills the GPU, and two of them at once
// only evict each other's working sets from L2: large requests run one at a
// time, and small ones behind a waiting large one are admitted past it.  A
// host function enqueued after the result copy marks the request done,
// returns its budget and wakes the dispatcher, which admits whatever arrived
// meanwhile.  Results are the same integer tables tripoll_survey computes for
// the request alone.
#include <chrono>
#include <cstring>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace tp {
namespace {

constexpr uint64_t kLargeEdges = 1ull << 25;  // graphs whose survey alone fills the GPU

uint64_t now_ns() {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Request {
    uint64_t id = 0;
    const tripoll_graph* graph = nullptr;  // read under the lock at submit time
    uint32_t slot = 0, kinds = 0, t_lo = 0, t_hi = 0;
    uint64_t words = 0;
    uint64_t bytes = 0;          // device scratch charged to the budget
    bool view = false;           // survey through a window view of the graph
    bool large = false;          // on a graph of kLargeEdges edges or more
    uint64_t* host = nullptr;    // pinned result buffer
    size_t host_cap = 0;
    uint64_t t_submit = 0, t_done = 0;
    int status = TRIPOLL_OK;
    bool done = false;
    struct tripoll_server* server = nullptr;
};

}  // namespace
}  // namespace tp

struct tripoll_server {
    int device = 0;
    uint64_t cap = 0;
    uint32_t max_inflight = 1;
    std::vector<tripoll_graph*> graphs;
    std::vector<cudaStream_t> streams;
    size_t next_stream = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<uint64_t> pending;
    std::unordered_map<uint64_t, tp::Request*> reqs;
    std::multimap<size_t, uint64_t*> pinned_pool;  // free pinned buffers by capacity
    uint64_t next_id = 1;
    uint32_t inflight = 0, large_inflight = 0;
    uint64_t in_use = 0;
    bool stop = false;
    std::thread dispatcher;
};

namespace tp {
namespace {

void CUDART_CB on_request_done(void* arg) {
    Request* r = static_cast<Request*>(arg);
    tripoll_server* s = r->server;
    std::lock_guard<std::mutex> lk(s->mu);
    r->t_done = now_ns();
    r->done = true;
    s->inflight -= 1;
    s->large_inflight -= r->large ? 1 : 0;
    s->in_use -= r->bytes;
    s->cv.notify_all();
}

// Launch one admitted request on a stream (called by the dispatcher, lock not held).
int launch_request(tripoll_server* s, Request* r, cudaStream_t st) {
    (void)s;
    const tripoll_graph* g = r->graph;
    Scratch acc;
    TP_CUDA(acc.alloc(r->words * 8 + 16, st));
    unsigned long long* a = acc.as<unsigned long long>();
    uint32_t* counters = reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(a) + r->words * 8);
    TP_CUDA(cudaMemsetAsync(a, 0, r->words * 8, st));
    int rc = launch_survey(g, r->kinds, r->t_lo, r->t_hi, 0, g->n, a, counters, st, r->view);
    if (rc) return rc;
    TP_CUDA(cudaMemcpyAsync(r->host, a, r->words * 8, cudaMemcpyDeviceToHost, st));
    acc.release();  // stream-ordered: after the copy
    TP_CUDA(cudaLaunchHostFunc(st, on_request_done, r));
    return TRIPOLL_OK;
}

// May r start now?  (lock held)
bool admissible(const tripoll_server* s, const Request* r) {
    if (r->large && s->large_inflight > 0) return false;
    return s->in_use + r->bytes <= s->cap || s->inflight == 0;
}

void dispatcher_loop(tripoll_server* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        s->cv.wait(lk, [&] {
            if (s->stop) return true;
            if (s->inflight >= s->max_inflight) return false;
            for (uint64_t id : s->pending)
                if (admissible(s, s->reqs[id])) return true;
            return false;
        });
        if (s->stop) break;
        // one admission round: everything that may start now, in arrival order;
        // requests that must wait keep their place in the queue
        std::vector<Request*> round;
        for (auto it = s->pending.begin(); it != s->pending.end() && s->inflight < s->max_inflight;) {
            Request* r = s->reqs[*it];
            if (!admissible(s, r)) {
                if (!r->large) break;  // over budget: keep arrival order
                ++it;                  // a large request waits for the one running; smaller ones pass
                continue;
            }
            it = s->pending.erase(it);
            s->inflight += 1;
            s->large_inflight += r->large ? 1 : 0;
            s->in_use += r->bytes;
            round.push_back(r);
        }
        std::vector<cudaStream_t> lanes;
        for (size_t i = 0; i < round.size(); ++i) {
            lanes.push_back(s->streams[s->next_stream]);
            s->next_stream = (s->next_stream + 1) % s->streams.size();
        }
        lk.unlock();
        for (size_t i = 0; i < round.size(); ++i) {
            int rc = launch_request(s, round[i], lanes[i]);
            if (rc) {
                std::lock_guard<std::mutex> g(s->mu);
                round[i]->status = rc;
                round[i]->t_done = now_ns();
                round[i]->done = true;
                s->inflight -= 1;
                s->large_inflight -= round[i]->large ? 1 : 0;
                s->in_use -= round[i]->bytes;
                s->cv.notify_all();
            }
        }
        lk.lock();
    }
}

}  // namespace
}  // namespace tp

using namespace tp;

extern "C" int tripoll_server_create(uint64_t scratch_cap_bytes, uint32_t max_inflight, tripoll_server_t* out) {
    if (!out || max_inflight == 0 || scratch_cap_bytes == 0)
        return fail(TRIPOLL_ERR_INVALID_ARG, "server needs a non-zero budget and max_inflight");
    tripoll_server* s = new tripoll_server();
    s->cap = scratch_cap_bytes;
    s->max_inflight = max_inflight;
    cudaError_t e = cudaGetDevice(&s->device);
    const uint32_t nstreams = max_inflight < 16 ? max_inflight : 16;
    for (uint32_t i = 0; e == cudaSuccess && i < nstreams; ++i) {
        cudaStream_t st;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e == cudaSuccess) s->streams.push_back(st);
    }
    if (e != cudaSuccess) {
        for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
        delete s;
        return cuda_fail(e, "tripoll_server_create");
    }
    s->dispatcher = std::thread(dispatcher_loop, s);
    *out = s;
    return TRIPOLL_OK;
}

extern "C" int tripoll_server_add_graph(tripoll_server_t s, tripoll_graph_t g, uint32_t* slot) {
    if (!s || !g || !slot) return fail(TRIPOLL_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    s->graphs.push_back(g);
    *slot = (uint32_t)(s->graphs.size() - 1);
    return TRIPOLL_OK;
}

extern "C" int tripoll_server_submit(tripoll_server_t s, uint32_t slot, uint32_t kind_mask, uint32_t t_lo,
                                     uint32_t t_hi, uint64_t* request_id) {
    if (!s || !request_id) return fail(TRIPOLL_ERR_INVALID_ARG, "NULL argument");
    tripoll_graph* g = nullptr;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (slot >= s->graphs.size()) return fail(TRIPOLL_ERR_NOT_FOUND, "unknown graph slot");
        g = s->graphs[slot];
    }
    int rc = check_survey_args(g, kind_mask, t_lo, t_hi, request_id);
    if (rc) return rc;
    Request* r = new Request();
    r->graph = g;
    r->slot = slot;
    r->kinds = kind_mask;
    r->t_lo = t_lo;
    r->t_hi = t_hi;
    r->words = make_layout(kind_mask, g->Lv, g->Le, g->n, g->m).words * g->num_graphs;
    r->bytes = r->words * 8 + 16;
    r->large = g->m >= kLargeEdges;
    r->server = s;
    if (r->bytes > s->cap) {
        delete r;
        return fail(TRIPOLL_ERR_NO_MEMORY, "request needs more scratch than the server budget");
    }
    // the window view when the budget holds it too, else out-of-window edges are skipped in place
    const uint64_t vb = window_view_bytes(g, kind_mask, t_lo, t_hi);
    r->view = vb > 0 && r->bytes + vb <= s->cap;
    if (r->view) r->bytes += vb;
    {  // pinned result buffer from the pool
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->pinned_pool.lower_bound(r->words * 8);
        if (it != s->pinned_pool.end()) {
            r->host = it->second;
            r->host_cap = it->first;
            s->pinned_pool.erase(it);
        }
    }
    if (!r->host) {
        size_t cap = 64;
        while (cap < r->words * 8) cap <<= 1;
        cudaError_t e = cudaHostAlloc((void**)&r->host, cap, cudaHostAllocPortable);
        if (e != cudaSuccess) {
            delete r;
            return cuda_fail(e, "cudaHostAlloc");
        }
        r->host_cap = cap;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    r->id = s->next_id++;
    r->t_submit = now_ns();
    s->reqs[r->id] = r;
    s->pending.push_back(r->id);
    *request_id = r->id;
    s->cv.notify_all();
    return TRIPOLL_OK;
}

extern "C" int tripoll_server_wait(tripoll_server_t s, uint64_t request_id, uint64_t* result, uint64_t* latency_ns,
                                   uint32_t timeout_ms) {
    if (!s) return fail(TRIPOLL_ERR_INVALID_ARG, "NULL server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(request_id);
    if (it == s->reqs.end()) return fail(TRIPOLL_ERR_NOT_FOUND, "unknown request id");
    Request* r = it->second;
    if (!s->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return r->done; }))
        return fail(TRIPOLL_ERR_TIMEOUT, "request not finished in time");
    s->reqs.erase(it);
    const int status = r->status;
    if (status == TRIPOLL_OK) {
        if (result) memcpy(result, r->host, r->words * 8);
        if (latency_ns) *latency_ns = r->t_done - r->t_submit;
    }
    s->pinned_pool.emplace(r->host_cap, r->host);
    delete r;
    if (status != TRIPOLL_OK) return fail(status, "request failed");
    return TRIPOLL_OK;
}

extern "C" void tripoll_server_destroy(tripoll_server_t s) {
    if (!s) return;
    for (cudaStream_t st : s->streams) cudaStreamSynchronize(st);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->cv.notify_all();
    }
    if (s->dispatcher.joinable()) s->dispatcher.join();
    // requests still queued or running: wait for the device, then free
    for (cudaStream_t st : s->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    for (auto& kv : s->reqs) {
        if (kv.second->host) cudaFreeHost(kv.second->host);
        delete kv.second;
    }
    for (auto& kv : s->pinned_pool) cudaFreeHost(kv.second);
    delete s;
}
