// serve.cu -- tc_submit / tc_poll / tc_drain: continuous batching of
// triangle-count requests.
//
// tc_submit copies the caller's host CSR into library-owned host memory and
// queues the request. A worker thread per context runs the loop:
//   1. admission: queued requests, oldest first, get device memory for their
//      CSR from an arena of mem_budget_bytes (first fit, coalescing frees) as
//      long as it has room; a request that alone exceeds the budget is refused
//      at submission with TC_ERR_BUSY;
//   2. completion: a finished round's per-graph counts are handed to its
//      tickets and the round's arena memory is freed, which admits more;
//   3. launch: whenever a round slot is idle and admitted requests of its
//      class wait, they form a round: their CSRs are copied to the device on
//      the round's stream and counted by the batched path (one padded
//      orientation + one counting pass, batch.cu). Rounds run on separate
//      streams, so a round formed from requests that arrived while others were
//      on the GPU overlaps with them.
// Two request classes keep large graphs from holding up small ones: a graph
// with more than kLargeEntries CSR entries is large and runs alone in the
// large slot, whose stream has the lowest priority and whose persistent
// counting kernels take kLargeGridShare of the SMs; small graphs share the
// other slots, whose streams have the highest priority.
// Each request's count is that of its own graph, whatever else is in its
// round (the batch lays graphs out disjointly).
#include <chrono>
#include <cstring>
#include <map>

#include "api_internal.h"

using namespace tcg;

namespace tcg {

namespace {

constexpr int kRounds = 4;                    // round slots (streams) in flight; the last is for large graphs
constexpr int kLargeSlot = kRounds - 1;
constexpr long long kLargeEntries = 1ll << 24;  // n + nnz above this: a large request
constexpr float kLargeGridShare = 0.75f;
constexpr int kMaxRoundGraphs = 4096;         // graphs per round
constexpr long long kMaxRoundEntries = 1ll << 30;  // CSR entries per round
constexpr size_t kAlign = 256;

enum class ReqState { Queued, Admitted, Running, Done };

struct Request {
    uint64_t ticket = 0;
    int64_t n = 0, nnz = 0;
    int bits = 32;
    std::vector<unsigned char> h_rp;  // library copies (tc_submit)
    std::vector<int32_t> h_col;
    const void* src_rp = nullptr;     // the caller's arrays (tc_submit_borrowed)
    const int32_t* src_col = nullptr;
    size_t off = 0, bytes = 0;  // arena placement
    ReqState state = ReqState::Queued;
    tc_status status = TC_OK;
    uint64_t count = 0;
};

size_t req_bytes(int64_t n, int64_t nnz, int bits) {
    const size_t rp = (size_t)(n + 1) * (bits / 8);
    const size_t a = (rp + kAlign - 1) / kAlign * kAlign;
    return a + ((size_t)nnz * 4 + kAlign - 1) / kAlign * kAlign + kAlign;
}

// First-fit allocator over one device block [0, size).
struct Arena {
    std::map<size_t, size_t> free_;  // offset -> length
    size_t size = 0;
    void reset(size_t sz) {
        free_.clear();
        size = sz;
        if (sz) free_[0] = sz;
    }
    bool alloc(size_t len, size_t* off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= len) {
                *off = it->first;
                const size_t rest = it->second - len, at = it->first + len;
                free_.erase(it);
                if (rest) free_[at] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t len) {
        auto it = free_.emplace(off, len).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

struct Round {
    BatchRunner runner;
    std::vector<Request*> reqs;
    std::vector<uint64_t> counts;
    bool busy = false;
    cudaEvent_t done = nullptr;
};

}  // namespace

struct ServeState {
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    std::deque<Request*> queue;
    std::vector<Request*> admitted;
    std::unordered_map<uint64_t, Request*> tickets;
    uint64_t next_ticket = 1;
    size_t outstanding = 0;  // requests not yet finished
    unsigned char* arena_base = nullptr;
    Arena arena;
    Round rounds[kRounds];
    tc_status fatal = TC_OK;
};

namespace {

void finish_round(tc_ctx* ctx, ServeState& S, Round& r) {
    tc_status st = r.runner.finish(ctx, r.counts.data());
    std::lock_guard<std::mutex> lk(S.mu);
    for (size_t i = 0; i < r.reqs.size(); ++i) {
        Request* q = r.reqs[i];
        q->status = st;
        q->count = st ? 0 : r.counts[i];
        q->state = ReqState::Done;
        S.arena.release(q->off, q->bytes);
        q->h_rp.clear();
        q->h_rp.shrink_to_fit();
        q->h_col.clear();
        q->h_col.shrink_to_fit();
        S.outstanding--;
    }
    r.reqs.clear();
    r.busy = false;
    S.cv_done.notify_all();
}

// Copy the round's CSRs to the device on its stream, then count them.
tc_status start_round(tc_ctx* ctx, ServeState& S, Round& r) {
    std::vector<tc_csr> gs(r.reqs.size());
    cudaStream_t st = r.runner.stream;
    for (size_t i = 0; i < r.reqs.size(); ++i) {
        Request* q = r.reqs[i];
        unsigned char* base = S.arena_base + q->off;
        const size_t rp_bytes = (size_t)(q->n + 1) * (q->bits / 8);
        unsigned char* d_col = base + (rp_bytes + kAlign - 1) / kAlign * kAlign;
        const void* hrp = q->src_rp ? q->src_rp : q->h_rp.data();
        const void* hcol = q->src_col ? (const void*)q->src_col : (const void*)q->h_col.data();
        cudaError_t e = cudaMemcpyAsync(base, hrp, rp_bytes, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess && q->nnz) e = cudaMemcpyAsync(d_col, hcol, (size_t)q->nnz * 4, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_status(ctx, e, "serving: copying a request to the device");
        gs[i] = tc_csr{q->n, q->nnz, base, q->bits, reinterpret_cast<const int32_t*>(d_col)};
    }
    r.counts.assign(r.reqs.size(), 0);
    tc_status s = r.runner.prepare(ctx, gs.data(), (int)gs.size());
    if (!s) s = r.runner.launch(ctx, false);
    if (!s) s = cuda_status(ctx, cudaEventRecord(r.done, st), "serving: cudaEventRecord");
    return s;
}

void worker_loop(tc_ctx* ctx) {
    ServeState& S = *ctx->serve;
    cudaSetDevice(ctx->device);
    for (;;) {
        // completions
        for (Round& r : S.rounds) {
            if (!r.busy) continue;
            const cudaError_t q = cudaEventQuery(r.done);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) cudaGetLastError();
            finish_round(ctx, S, r);
        }
        std::unique_lock<std::mutex> lk(S.mu);
        if (S.stop) {
            lk.unlock();
            break;
        }
        // admission: oldest first, as long as the arena has room
        while (!S.queue.empty()) {
            Request* q = S.queue.front();
            size_t off = 0;
            if (!S.arena.alloc(q->bytes, &off)) break;
            q->off = off;
            q->state = ReqState::Admitted;
            S.admitted.push_back(q);
            S.queue.pop_front();
        }
        // launch: idle round slots take the admitted requests of their class
        bool launched = false;
        for (int slot = 0; slot < kRounds; ++slot) {
            Round& r = S.rounds[slot];
            const bool large_slot = slot == kLargeSlot;
            if (r.busy || S.admitted.empty()) continue;
            // a round holds requests of one class and one offset width, oldest
            // first; a large round holds one graph
            int bits = 0;
            long long entries = 0;
            r.reqs.clear();
            for (size_t i = 0; i < S.admitted.size() && (int)r.reqs.size() < kMaxRoundGraphs;) {
                Request* q = S.admitted[i];
                const long long e2 = entries + q->nnz + q->n;
                const bool large = q->nnz + q->n > kLargeEntries;
                if (large != large_slot || (bits && q->bits != bits) || (!r.reqs.empty() && e2 > kMaxRoundEntries)) {
                    ++i;
                    continue;
                }
                bits = q->bits;
                entries = e2;
                r.reqs.push_back(q);
                S.admitted.erase(S.admitted.begin() + (long)i);
                if (large_slot) break;
            }
            if (r.reqs.empty()) continue;
            for (Request* q : r.reqs) q->state = ReqState::Running;
            r.busy = true;
            lk.unlock();
            const tc_status s = start_round(ctx, S, r);
            if (s) {
                cudaStreamSynchronize(r.runner.stream);
                lk.lock();
                for (Request* q : r.reqs) {
                    q->status = s;
                    q->state = ReqState::Done;
                    S.arena.release(q->off, q->bytes);
                    S.outstanding--;
                }
                r.reqs.clear();
                r.busy = false;
                S.cv_done.notify_all();
                lk.unlock();
            }
            lk.lock();
            launched = true;
        }
        bool any_busy = false;
        for (Round& r : S.rounds) any_busy |= r.busy;
        if (!launched) {
            // busy rounds are polled every 50 us; otherwise sleep until work arrives
            if (any_busy)
                S.cv_work.wait_for(lk, std::chrono::microseconds(50));
            else if (S.queue.empty() && S.admitted.empty())
                S.cv_work.wait_for(lk, std::chrono::milliseconds(20));
        }
    }
    // shutdown: wait for rounds in flight
    for (Round& r : S.rounds)
        if (r.busy) finish_round(ctx, S, r);
}

tc_status serve_start(tc_ctx* ctx) {
    if (ctx->serve) return TC_OK;
    if (ctx->mem_budget == 0) return ctx_fail(ctx, TC_ERR_INVALID_ARG, "serving needs a memory budget (tc_create)");
    ServeState* S = new (std::nothrow) ServeState();
    if (!S) return TC_ERR_OOM;
    void* p = nullptr;
    tc_status s = injected_oom(ctx)
                      ? ctx_fail(ctx, TC_ERR_OOM, "cudaMalloc(serving arena): out of memory (injected by tc_inject_oom)")
                      : cuda_status(ctx, cudaMalloc(&p, ctx->mem_budget), "cudaMalloc(serving arena)");
    if (!s) {
        S->arena_base = static_cast<unsigned char*>(p);
        S->arena.reset(ctx->mem_budget);
        ctx->held_bytes += (long long)ctx->mem_budget;
    }
    int least = 0, greatest = 0;
    if (!s)
        s = cuda_status(ctx, cudaDeviceGetStreamPriorityRange(&least, &greatest),
                        "cudaDeviceGetStreamPriorityRange");
    for (int i = 0; i < kRounds && !s; ++i) {
        S->rounds[i].runner.priority = i == kLargeSlot ? least : greatest;
        S->rounds[i].runner.grid_share = i == kLargeSlot ? kLargeGridShare : 1.0f;
        s = S->rounds[i].runner.init(ctx);
        if (!s) s = cuda_status(ctx, cudaEventCreateWithFlags(&S->rounds[i].done, cudaEventDisableTiming),
                                "cudaEventCreate");
    }
    if (s) {
        for (Round& r : S->rounds) {
            r.runner.release(ctx);
            if (r.done) cudaEventDestroy(r.done);
        }
        if (S->arena_base) cudaFree(S->arena_base);
        delete S;
        return s;
    }
    ctx->serve = S;
    S->worker = std::thread(worker_loop, ctx);
    return TC_OK;
}

}  // namespace

void serve_shutdown(tc_ctx* ctx) {
    ServeState* S = ctx->serve;
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (Round& r : S->rounds) {
        r.runner.release(ctx);
        if (r.done) cudaEventDestroy(r.done);
    }
    if (S->arena_base) {
        cudaFree(S->arena_base);
        ctx->held_bytes -= (long long)ctx->mem_budget;
    }
    for (auto& kv : S->tickets) delete kv.second;
    for (Request* q : S->queue)
        if (!S->tickets.count(q->ticket)) delete q;
    delete S;
    ctx->serve = nullptr;
}

}  // namespace tcg

extern "C" {

}  // extern "C"

namespace {

tc_status submit_common(tc_ctx* ctx, const tc_csr* g, bool borrowed, uint64_t* ticket) {
    if (!ctx || !ticket) return TC_ERR_INVALID_ARG;
    tc_status s = check_csr(ctx, g);
    if (s) return s;
    {
        static std::mutex start_mu;
        std::lock_guard<std::mutex> lk(start_mu);
        DeviceGuard dg(ctx->device);
        if ((s = serve_start(ctx))) return s;
    }
    ServeState& S = *ctx->serve;
    const size_t bytes = req_bytes(g->n, g->nnz, g->offset_bits);
    if (bytes > ctx->mem_budget)
        return ctx_fail(ctx, TC_ERR_BUSY, "request needs %zu bytes, more than the %zu-byte budget", bytes,
                        ctx->mem_budget);
    Request* q = new (std::nothrow) Request();
    if (!q) return TC_ERR_OOM;
    q->n = g->n;
    q->nnz = g->nnz;
    q->bits = g->offset_bits;
    q->bytes = bytes;
    if (borrowed) {
        q->src_rp = g->row_ptr;
        q->src_col = g->col;
    } else {
        try {
            q->h_rp.resize((size_t)(g->n + 1) * (g->offset_bits / 8));
            q->h_col.resize((size_t)g->nnz);
        } catch (...) {
            delete q;
            return ctx_fail(ctx, TC_ERR_OOM, "host memory for the request copy");
        }
        if (g->row_ptr) memcpy(q->h_rp.data(), g->row_ptr, q->h_rp.size());
        if (g->nnz) memcpy(q->h_col.data(), g->col, (size_t)g->nnz * 4);
        // a malformed request is refused here, so it cannot fail the round it would join
        long long prev = 0;
        bool bad = false;
        for (int64_t u = 0; u <= g->n && !bad; ++u) {
            const long long o = q->bits == 64 ? reinterpret_cast<const int64_t*>(q->h_rp.data())[u]
                                              : reinterpret_cast<const int32_t*>(q->h_rp.data())[u];
            bad = (u == 0 ? o != 0 : o < prev) || o > g->nnz || (u == g->n && o != g->nnz);
            prev = o;
        }
        for (int64_t i = 0; i < g->nnz && !bad; ++i) bad = (uint32_t)q->h_col[i] >= (uint64_t)g->n;
        if (bad) {
            delete q;
            return ctx_fail(ctx, TC_ERR_BAD_GRAPH, "malformed CSR: row_ptr not 0..nnz non-decreasing, or a column id "
                                                   "outside [0, n)");
        }
    }
    {
        std::lock_guard<std::mutex> lk(S.mu);
        q->ticket = S.next_ticket++;
        S.tickets[q->ticket] = q;
        S.queue.push_back(q);
        S.outstanding++;
        *ticket = q->ticket;
    }
    S.cv_work.notify_one();
    return TC_OK;
}

}  // namespace

extern "C" {

tc_status tc_submit(tc_ctx* ctx, const tc_csr* g, uint64_t* ticket) { return submit_common(ctx, g, false, ticket); }

tc_status tc_submit_borrowed(tc_ctx* ctx, const tc_csr* g, uint64_t* ticket) {
    return submit_common(ctx, g, true, ticket);
}

tc_status tc_poll(tc_ctx* ctx, uint64_t ticket, uint64_t* count) {
    if (!ctx || !count) return TC_ERR_INVALID_ARG;
    if (!ctx->serve) return ctx_fail(ctx, TC_ERR_INVALID_ARG, "unknown ticket %llu", (unsigned long long)ticket);
    ServeState& S = *ctx->serve;
    std::lock_guard<std::mutex> lk(S.mu);
    auto it = S.tickets.find(ticket);
    if (it == S.tickets.end())
        return ctx_fail(ctx, TC_ERR_INVALID_ARG, "unknown ticket %llu", (unsigned long long)ticket);
    Request* q = it->second;
    if (q->state != ReqState::Done) return TC_ERR_NOT_READY;
    const tc_status st = q->status;
    if (!st) *count = q->count;
    S.tickets.erase(it);
    delete q;
    return st;
}

tc_status tc_drain(tc_ctx* ctx) {
    if (!ctx) return TC_ERR_INVALID_ARG;
    if (!ctx->serve) return TC_OK;
    ServeState& S = *ctx->serve;
    std::unique_lock<std::mutex> lk(S.mu);
    S.cv_work.notify_all();
    S.cv_done.wait(lk, [&] { return S.outstanding == 0; });
    return TC_OK;
}

}  // extern "C"
