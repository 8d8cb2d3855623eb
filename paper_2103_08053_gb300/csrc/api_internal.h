// api_internal.h -- host-side state of a tc_ctx (not installed).
#pragma once

#include <atomic>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "tc_internal.h"

namespace tcg {

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    // Grow-only: (re)allocates when `need` exceeds the current size, after
    // synchronising `st` so no queued kernel still reads the old buffer.
    tc_status ensure(tc_ctx* ctx, size_t need, cudaStream_t st);
    void release(tc_ctx* ctx);
};

// Scratch of one counting pass.
struct Workspace {
    DevBuf deg, kept, partial, dag_ptr, dag_col, warp_list, warp_desc, items, ctr, stats, hubs, kbits, bnd;
    DevBuf pc;  // physical-combination scratch (tc_params.balance == TC_BALANCE_PC only)
    DevBuf okey, ohist;  // ordered warp list: per-vertex locality keys, key histogram / offsets
    DevBuf ikey, items2; // ordered work items (BLOCK_ITEM_ORDER): item keys, items as binned
    void release_all(tc_ctx* ctx) {
        for (DevBuf* b : {&deg, &kept, &partial, &dag_ptr, &dag_col, &warp_list, &warp_desc, &items, &ctr, &stats,
                          &hubs, &kbits, &bnd, &pc, &okey, &ohist, &ikey, &items2})
            b->release(ctx);
    }
};

struct BufPair {
    DevBuf a, b;
    void release_all(tc_ctx* ctx) {
        a.release(ctx);
        b.release(ctx);
    }
};

class DeviceGuard {
   public:
    explicit DeviceGuard(int dev);
    ~DeviceGuard();

   private:
    int prev_ = -1, dev_ = -1;
};

// CUDA events of one timed call: [0] before orientation (or binning), [1]
// after orientation, [2] after binning, [3] after the counting kernels.
struct TimedCall {
    cudaEvent_t ev[4];
    bool oriented;
};

// One batched counting pass (batch.cu): its own stream, workspace, pinned
// staging and a CUDA graph of the whole launch sequence, replayed while the
// batch shape (graph count, padded vertices, entries, offset width, params)
// and the buffers stay the same. Used by tc_count_batch and by serving rounds.
struct BatchRunner {
    cudaStream_t stream = nullptr;
    int priority = 0;          // stream priority (init); 0 = default
    float grid_share = 1.0f;   // fraction of the persistent counting grids this runner launches
    cudaEvent_t ev_in = nullptr, ev_done = nullptr;
    Workspace ws;
    DevBuf graphs, per_vertex, counts, dag_ptr, dag_col;
    GraphRef* h_graphs = nullptr;   // pinned
    uint64_t* h_counts = nullptr;   // pinned
    DevCounters* h_ctr = nullptr;   // pinned
    int h_cap = 0;
    int k = 0, bits = 32;
    bool row_local = false;         // the batch's DAG is row-local (see launch_orient)
    long long total = 0, nnz_total = 0;
    bool moved = true;              // a buffer moved since the graph was captured
    cudaGraphExec_t exec = nullptr;
    int key_k = -1, key_bits = 0;
    long long key_total = 0, key_nnz = 0, key_cfg = -1, captured_launches = 0, enqueued_launches = 0;

    tc_status init(tc_ctx* ctx);
    void release(tc_ctx* ctx);
    void drop_graph();
    tc_status prepare(tc_ctx* ctx, const tc_csr* gs, int k);  // layout + buffers + staging
    tc_status enqueue(tc_ctx* ctx);                           // the launch sequence on `stream`
    tc_status launch(tc_ctx* ctx, bool use_graph);            // capture once, then replay
    tc_status finish(tc_ctx* ctx, uint64_t* counts_host);     // wait, check errors, copy results
};

struct ServeState;  // serve.cu

}  // namespace tcg

struct tc_ctx {
    int device = 0;
    int num_sms = 0;
    int max_smem_optin = 0;
    size_t mem_budget = 0;
    std::atomic<long long> held_bytes{0};
    tc_params params{};
    tcg::CountCfg cfg{};
    char last_error[512] = {0};
    tcg::Workspace ws;
    tcg::DevBuf out_scalars;          // device: count (8 B) + error (4 B)
    tcg::BufPair csr_copy;            // device copy of a host CSR (tc_count_host)
    tcg::DevCounters* host_ctr = nullptr;  // pinned
    std::map<void*, void*> dags;      // tc_orient allocations: dag_ptr -> dag_col
    std::atomic<long long> launches{0};     // kernels launched by this context (any thread)
    std::vector<tcg::TimedCall> timed;      // recorded, not yet read
    std::vector<tcg::TimedCall> timed_free; // event sets to reuse
    long long cfg_version = 0;              // bumped by tc_set_params
    long long cyc_build = 0, cyc_probe = 0; // worker cycles read back by blocking calls (record_timing 2)
    cudaStream_t aux_stream = nullptr;      // tc_count_host: host-to-device copies in pieces
    cudaEvent_t aux_ev[9] = {};             // one per piece, plus the start
    tcg::BatchRunner* batch = nullptr;
    tcg::ServeState* serve = nullptr;
    // tc_inject_oom: the fail_alloc_in-th counted device allocation from now
    // on fails on the host as if the device were out of memory (0: off)
    std::atomic<long long> fail_alloc_in{0};
};

namespace tcg {

tc_status ctx_fail(tc_ctx* ctx, tc_status s, const char* fmt, ...);
// True when this device allocation of ctx is the one tc_inject_oom asked to
// fail (it then counts as made); false otherwise, and always for ctx NULL.
bool injected_oom(tc_ctx* ctx);
tc_status cuda_status(tc_ctx* ctx, cudaError_t e, const char* what);
tc_status err_bits_status(int bits);
const char* err_bits_text(int bits);
tc_status resolve_params(tc_ctx* ctx, const tc_params* in, tc_params* out, CountCfg* cfg);
tc_status check_csr(tc_ctx* ctx, const tc_csr* g);
tc_status ensure_count_ws(tc_ctx* ctx, Workspace& ws, int64_t n, int64_t m, cudaStream_t st);
tc_status ensure_orient_ws(tc_ctx* ctx, Workspace& ws, int64_t n, int64_t nnz, cudaStream_t st);
// Orient g into ctx->ws.dag_ptr / dag_col (blocking on st); *m = DAG edges.
tc_status orient_to_workspace(tc_ctx* ctx, const tc_csr* g, cudaStream_t st, int64_t* m);

void batch_release(tc_ctx* ctx);  // batch.cu
size_t noalloc_scratch_bytes();    // noalloc.cu
// Start a timed call when tc_params.record_timing is set (else returns null);
// mark(i) records event i of it on st.
TimedCall* timing_begin(tc_ctx* ctx, bool oriented);
void timing_mark(TimedCall* tc, int i, cudaStream_t st);
void serve_shutdown(tc_ctx* ctx); // serve.cu

}  // namespace tcg
