// server.cu -- serving loop: resident graphs, continuous batching of survey
// requests under a scratch-memory budget.
//
// Requests queue on the host.  A dispatcher thread forms admission rounds in
// arrival order while fewer than max_inflight requests are on the device and
// the round's scratch fits under the budget.  Within a round, requests on the
// same graph join one batch (up to 64): a batch of several requests is one
// pass over the graph (survey_many: the wedge checks of the union of their
// windows once, each triangle folded once into the cell of the requests'
// window bounds that holds it), a batch of one is an ordinary survey; batches
// of different graphs run at once on different CUDA streams.  A batch is
// charged what it really takes: its record grid, its results, and the window
// view of its union window when that fits too (else the pass skips
// out-of-window edges in place).  A batch on a large graph (kLargeEdges edges
// or more) already fills the GPU, and two at once only evict each other's
// working sets from L2, so large batches run one at a time while requests
// that arrive meanwhile queue up -- the next round takes them all in one pass
// -- and small ones are admitted past a waiting large one.  A host function
// enqueued after a batch's result copies marks its requests done, returns the
// budget and wakes the dispatcher.  Each result equals tripoll_survey's for
// that request alone.
#include <chrono>
#include <cstring>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <algorithm>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace tp {
namespace {

constexpr uint64_t kLargeEdges = 1ull << 25;  // graphs whose survey alone fills the GPU
constexpr size_t kBatchMax = 64;              // requests in one pass (distinct window bounds it can hold)
// A pass over several requests pays for every triangle of the union of their windows, while a request
// alone pays only for those of its own; it wins when several requests share the wedge checks and every
// triangle folds cheaply, i.e. when the whole grid of cell records fits the kernels' on-chip mirror.
constexpr uint64_t kBatchMirrorWords = 4096;
constexpr size_t kBatchMin = 4;               // fewer requests run one by one

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
    uint64_t bytes = 0;          // device scratch of the request surveyed alone
    bool view = false;           // alone: survey through a window view of the graph
    bool large = false;          // on a graph of kLargeEdges edges or more
    bool joins = false;          // may share a pass with other requests on its graph
    uint64_t* host = nullptr;    // pinned result buffer
    size_t host_cap = 0;
    uint64_t t_submit = 0, t_done = 0;
    int status = TRIPOLL_OK;
    bool done = false;
};

// Requests launched together: one pass over one graph.
struct Batch {
    std::vector<Request*> reqs;
    const tripoll_graph* graph = nullptr;
    uint64_t bytes = 0;  // charged to the budget
    bool view = false;   // several requests: through the view of the union window
    bool large = false;
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
    uint32_t inflight = 0, large_inflight = 0;  // requests, and batches on large graphs
    uint64_t in_use = 0;
    uint64_t st_requests = 0, st_batches = 0, st_passes = 0, st_fused = 0;  // tripoll_server_stats
    bool stop = false;
    std::thread dispatcher;
};

namespace tp {
namespace {

// Mark a batch's requests done and return its budget (lock not held by the caller).
void finish_batch(Batch* b, int status) {
    tripoll_server* s = b->server;
    std::lock_guard<std::mutex> lk(s->mu);
    const uint64_t t = now_ns();
    for (Request* r : b->reqs) {
        r->status = status;
        r->t_done = t;
        r->done = true;
    }
    s->inflight -= (uint32_t)b->reqs.size();
    s->large_inflight -= b->large ? 1 : 0;
    s->in_use -= b->bytes;
    s->cv.notify_all();
    delete b;
}

void CUDART_CB on_batch_done(void* arg) { finish_batch(static_cast<Batch*>(arg), TRIPOLL_OK); }

// Launch one request alone on a stream.
int launch_single(const tripoll_graph* g, Request* r, cudaStream_t st) {
    {
        Scratch acc;
        TP_CUDA(acc.alloc(r->words * 8 + 16, st));
        unsigned long long* a = acc.as<unsigned long long>();
        uint32_t* counters = reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(a) + r->words * 8);
        TP_CUDA(cudaMemsetAsync(a, 0, r->words * 8, st));
        int rc = launch_survey(g, r->kinds, r->t_lo, r->t_hi, 0, g->n, a, counters, st, r->view);
        if (rc) return rc;
        TP_CUDA(cudaMemcpyAsync(r->host, a, r->words * 8, cudaMemcpyDeviceToHost, st));
        acc.release();  // stream-ordered: after the copy
    }
    return TRIPOLL_OK;
}

// Launch a batch on a stream (dispatcher thread, lock not held); its host function completes it.
// A batch below kBatchMin requests runs them one after the other on the stream.
int launch_batch(Batch* b, cudaStream_t st) {
    const tripoll_graph* g = b->graph;
    if (b->reqs.size() < kBatchMin) {
        for (Request* r : b->reqs) {
            int rc = launch_single(g, r, st);
            if (rc) return rc;
        }
    } else {
        std::vector<uint32_t> kinds, lo, hi;
        std::vector<uint64_t*> res;
        for (Request* r : b->reqs) {
            kinds.push_back(r->kinds);
            lo.push_back(r->t_lo);
            hi.push_back(r->t_hi);
            res.push_back(r->host);
        }
        // the pinned results are complete when the host function runs: no synchronisation here
        int rc = survey_many(g, (uint32_t)b->reqs.size(), kinds.data(), lo.data(), hi.data(), res.data(), st, b->view,
                             false);
        if (rc) return rc;
    }
    TP_CUDA(cudaLaunchHostFunc(st, on_batch_done, b));
    return TRIPOLL_OK;
}

// Scratch of a batch of several requests, with or without the union window's view (~0 when the
// batch cannot be one pass).  Below kBatchMin the requests run one by one: their own scratch, one
// at a time, plus each one's window view when that is what its alone-estimate holds.
uint64_t batch_bytes(const std::vector<Request*>& reqs, bool view) {
    std::vector<uint32_t> kinds, lo, hi;
    uint32_t all = 0;
    uint64_t single = 0;
    for (Request* r : reqs) {
        kinds.push_back(r->kinds);
        lo.push_back(r->t_lo);
        hi.push_back(r->t_hi);
        all |= r->kinds;
        single = std::max(single, r->bytes);
    }
    // the cell grid must fit on chip: distinct lower x upper bounds x the union layout's words
    std::vector<uint32_t> l(lo), h(hi);
    std::sort(l.begin(), l.end());
    std::sort(h.begin(), h.end());
    const uint64_t cells = (uint64_t)(std::unique(l.begin(), l.end()) - l.begin()) *
                           (uint64_t)(std::unique(h.begin(), h.end()) - h.begin());
    const tripoll_graph* g = reqs[0]->graph;
    if (cells * make_layout(all, g->Lv, g->Le, g->n, g->m).words > kBatchMirrorWords) return ~0ull;
    if (reqs.size() < kBatchMin) return single;
    return survey_many_bytes(g, (uint32_t)reqs.size(), kinds.data(), lo.data(), hi.data(), view);
}

// May r start a batch of its own now?  (lock held)
bool admissible(const tripoll_server* s, const Request* r) {
    if (r->large && s->large_inflight > 0) return false;
    return s->in_use + r->bytes <= s->cap || s->inflight == 0;
}

// Add r to batch b if the budget holds the larger batch (lock held).
bool try_join(tripoll_server* s, Batch* b, Request* r) {
    if (!r->joins || b->reqs.size() >= kBatchMax) return false;
    std::vector<Request*> grown = b->reqs;
    grown.push_back(r);
    const uint64_t others = s->in_use - b->bytes;
    bool view = true;
    uint64_t bytes = batch_bytes(grown, true);
    if (bytes == ~0ull || others + bytes > s->cap) {
        view = false;
        bytes = batch_bytes(grown, false);
    }
    if (bytes == ~0ull || others + bytes > s->cap) return false;
    s->in_use = others + bytes;
    b->bytes = bytes;
    b->view = view;
    b->reqs.push_back(r);
    return true;
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
        // one admission round, in arrival order: a request joins its graph's batch of this round when
        // the budget holds the larger batch, else starts one; requests that must wait keep their place
        std::vector<Batch*> round;
        std::multimap<const tripoll_graph*, Batch*> open;
        for (auto it = s->pending.begin(); it != s->pending.end() && s->inflight < s->max_inflight;) {
            Request* r = s->reqs[*it];
            bool joined = false;
            for (auto ob = open.equal_range(r->graph); ob.first != ob.second && !joined; ++ob.first)
                joined = try_join(s, ob.first->second, r);
            if (joined) {
                it = s->pending.erase(it);
                s->inflight += 1;
                continue;
            }
            if (!admissible(s, r)) {
                if (!r->large) break;  // over budget: keep arrival order
                ++it;                  // a large request waits for the batch running; smaller ones pass
                continue;
            }
            Batch* b = new Batch();
            b->graph = r->graph;
            b->server = s;
            b->large = r->large;
            b->bytes = r->bytes;
            b->view = r->view;
            b->reqs.push_back(r);
            it = s->pending.erase(it);
            s->inflight += 1;
            s->large_inflight += r->large ? 1 : 0;
            s->in_use += r->bytes;
            round.push_back(b);
            if (r->joins) open.emplace(r->graph, b);
        }
        std::vector<cudaStream_t> lanes;
        for (size_t i = 0; i < round.size(); ++i) {
            lanes.push_back(s->streams[s->next_stream]);
            s->next_stream = (s->next_stream + 1) % s->streams.size();
        }
        lk.unlock();
        for (size_t i = 0; i < round.size(); ++i) {
            {
                std::lock_guard<std::mutex> g(s->mu);
                s->st_requests += round[i]->reqs.size();
                s->st_batches += 1;
                const bool fused = round[i]->reqs.size() >= kBatchMin;
                s->st_passes += fused ? 1 : round[i]->reqs.size();
                s->st_fused += fused ? round[i]->reqs.size() : 0;
            }
            int rc = launch_batch(round[i], lanes[i]);
            if (rc) finish_batch(round[i], rc);
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
    // the timestamp histogram that bounds each request's window view for the scratch budget
    if (int rc = ts_histogram(g)) return rc;
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
    r->joins = !g->graph_of && !(kind_mask & (TRIPOLL_VERTEX_LOCAL | TRIPOLL_EDGE_LOCAL));
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

extern "C" int tripoll_server_stats(tripoll_server_t s, uint64_t* stats) {
    if (!s || !stats) return fail(TRIPOLL_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    stats[0] = s->st_requests;
    stats[1] = s->st_batches;
    stats[2] = s->st_passes;
    stats[3] = s->st_fused;
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
