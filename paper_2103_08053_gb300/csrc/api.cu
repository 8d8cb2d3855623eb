// api.cu -- the C ABI declared in include/tc.h: contexts, workspace, the
// single-graph entry points, statistics and diagnostics. Batched counting
// lives in batch.cu, serving in serve.cu.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "api_internal.h"

using namespace tcg;

// ---------------------------------------------------------------- helpers

// Failures of calls that have no context yet (tc_create) are kept per thread
// and reported by tc_last_error(NULL).
static thread_local char g_create_error[512];

tc_status tcg::ctx_fail(tc_ctx* ctx, tc_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(ctx ? ctx->last_error : g_create_error, ctx ? sizeof(ctx->last_error) : sizeof(g_create_error), fmt,
              ap);
    va_end(ap);
    return s;
}

tc_status tcg::cuda_status(tc_ctx* ctx, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return TC_OK;
    cudaGetLastError();
    const tc_status s = (e == cudaErrorMemoryAllocation) ? TC_ERR_OOM : TC_ERR_CUDA;
    return ctx_fail(ctx, s, "%s: %s", what, cudaGetErrorString(e));
}

tc_status tcg::err_bits_status(int bits) {
    if (bits & ERRBIT_DAG_TOO_BIG) return TC_ERR_UNSUPPORTED;
    if (bits) return TC_ERR_BAD_GRAPH;
    return TC_OK;
}

const char* tcg::err_bits_text(int bits) {
    if (bits & ERRBIT_DAG_TOO_BIG) return "oriented graph has 2^31 or more edges (int32 DAG offsets)";
    if (bits & ERRBIT_DAG_OVERFLOW) return "more kept edges than nnz/2: the CSR is not symmetric";
    if (bits & ERRBIT_BAD_GRAPH) return "malformed CSR: column id outside [0,n) or row_ptr not monotone within [0,nnz]";
    return "";
}

bool tcg::injected_oom(tc_ctx* ctx) {
    if (!ctx) return false;
    long long k = ctx->fail_alloc_in.load();
    while (k > 0 && !ctx->fail_alloc_in.compare_exchange_weak(k, k - 1)) {
    }
    return k == 1;
}

tc_status tcg::DevBuf::ensure(tc_ctx* ctx, size_t need, cudaStream_t st) {
    if (need <= bytes) return TC_OK;
    if (injected_oom(ctx))
        return ctx_fail(ctx, TC_ERR_OOM, "cudaMalloc(workspace): out of memory (injected by tc_inject_oom)");
    if (p) {
        cudaStreamSynchronize(st);
        cudaFree(p);
        ctx->held_bytes -= bytes;
        p = nullptr;
        bytes = 0;
    }
    size_t want = need + need / 8;  // headroom against repeated growth
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        want = need;
        e = cudaMalloc(&p, want);
    }
    if (e != cudaSuccess) {
        p = nullptr;
        return cuda_status(ctx, e, "cudaMalloc(workspace)");
    }
    bytes = want;
    ctx->held_bytes += want;
    return TC_OK;
}

void tcg::DevBuf::release(tc_ctx* ctx) {
    if (p) {
        cudaFree(p);
        if (ctx) ctx->held_bytes -= bytes;
    }
    p = nullptr;
    bytes = 0;
}

DeviceGuard::DeviceGuard(int dev) {
    cudaGetDevice(&prev_);
    if (prev_ != dev) cudaSetDevice(dev);
    dev_ = dev;
}
DeviceGuard::~DeviceGuard() {
    if (prev_ != dev_ && prev_ >= 0) cudaSetDevice(prev_);
}

static void fill_defaults(tc_params* p) {
    memset(p, 0, sizeof(*p));
    p->warp_max_out_degree = 128;
    p->warp_area_ints = pack_table_ints(128, 16);
    p->warp_min_buckets = 16;
    p->block_threads = 256;
    p->block_smem_bytes = 50 * 1024;
    p->item_neighbors = DEFAULT_ITEM_NEIGHBORS;
    p->chunk = 32;
    p->warps_per_block = 8;
    p->shard_count = 1;
    p->shard_index = 0;
    p->validate = 0;
}

static bool is_pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

// Merge p over the defaults, check it, and resolve the launch configuration.
tc_status tcg::resolve_params(tc_ctx* ctx, const tc_params* in, tc_params* out, CountCfg* cfg) {
    tc_params d;
    fill_defaults(&d);
    tc_params p = d;
    if (in) {
#define TAKE(f) \
    if (in->f) p.f = in->f
        TAKE(warp_max_out_degree);
        TAKE(warp_area_ints);
        TAKE(warp_min_buckets);
        TAKE(block_threads);
        TAKE(block_smem_bytes);
        TAKE(item_neighbors);
        TAKE(chunk);
        TAKE(warps_per_block);
        TAKE(shard_count);
        p.shard_index = in->shard_index;
        p.validate = in->validate;
        p.record_timing = in->record_timing;
        p.hash_mode = in->hash_mode;
        p.scalar_loads = in->scalar_loads;
        p.edge_centric = in->edge_centric;
        p.balance = in->balance;
        p.warp_order = in->warp_order;
#undef TAKE
    }
    if (p.warp_max_out_degree < 1 || p.warp_max_out_degree > 255)
        return ctx_fail(ctx, TC_ERR_INVALID_ARG, "warp_max_out_degree must be in [1, 255]");
    if (!is_pow2(p.warp_min_buckets) || p.warp_min_buckets < 16 || p.warp_min_buckets > 4096)
        return ctx_fail(ctx, TC_ERR_INVALID_ARG, "warp_min_buckets must be a power of two in [16, 4096]");
    if (p.warp_area_ints < 16 || p.warp_area_ints % 4)
        return ctx_fail(ctx, TC_ERR_INVALID_ARG, "warp_area_ints must be a multiple of 4");
    {
        const long long need = pack_table_ints(p.warp_max_out_degree, p.warp_min_buckets);
        if (need > p.warp_area_ints)
            return ctx_fail(ctx, TC_ERR_INVALID_ARG,
                            "warp_area_ints %d cannot hold the table of a vertex with d+ = %d (%lld ints)",
                            p.warp_area_ints, p.warp_max_out_degree, need);
    }
    if (p.block_threads < 64 || p.block_threads > 1024 || p.block_threads % 32)
        return ctx_fail(ctx, TC_ERR_INVALID_ARG, "block_threads must be a multiple of 32 in [64, 1024]");
    if (p.warps_per_block < 1 || p.warps_per_block > 32)
        return ctx_fail(ctx, TC_ERR_INVALID_ARG, "warps_per_block must be in [1, 32]");
    if (p.item_neighbors < 32 || p.item_neighbors > p.block_threads || p.item_neighbors % 32)
        return ctx_fail(ctx, TC_ERR_INVALID_ARG, "item_neighbors must be a multiple of 32 in [32, block_threads]");
    if (p.hash_mode != 0 && p.hash_mode != 1) return ctx_fail(ctx, TC_ERR_INVALID_ARG, "hash_mode must be 0 or 1");
    if (p.scalar_loads != 0 && p.scalar_loads != 1)
        return ctx_fail(ctx, TC_ERR_INVALID_ARG, "scalar_loads must be 0 or 1");
    if (p.edge_centric != 0 && p.edge_centric != 1)
        return ctx_fail(ctx, TC_ERR_INVALID_ARG, "edge_centric must be 0 or 1");
    if (p.balance < TC_BALANCE_VC || p.balance > TC_BALANCE_PC)
        return ctx_fail(ctx, TC_ERR_INVALID_ARG, "balance must be one of TC_BALANCE_VC .. TC_BALANCE_PC");
    if (p.balance != TC_BALANCE_VC && p.hash_mode != 0)
        return ctx_fail(ctx, TC_ERR_INVALID_ARG, "the balance ablation modes use hash_mode 0");
    if (p.warp_order < 0 || p.warp_order > 2)
        return ctx_fail(ctx, TC_ERR_INVALID_ARG, "warp_order must be 0, 1 or 2");
    if (p.record_timing < 0 || p.record_timing > 2)
        return ctx_fail(ctx, TC_ERR_INVALID_ARG, "record_timing must be 0, 1 or 2");
    if (p.chunk < 1 || p.chunk > 32) return ctx_fail(ctx, TC_ERR_INVALID_ARG, "chunk must be in [1, 32]");
    if (p.shard_count < 1 || p.shard_index < 0 || p.shard_index >= p.shard_count)
        return ctx_fail(ctx, TC_ERR_INVALID_ARG, "need 0 <= shard_index < shard_count");
    const int max_smem = ctx ? ctx->max_smem_optin : 227 * 1024;
    const long long warp_smem =
        (long long)p.warps_per_block * (p.warp_area_ints + 224) * 4;
    if (warp_smem > max_smem)
        return ctx_fail(ctx, TC_ERR_INVALID_ARG, "warp kernel needs %lld B of shared memory (max %d)", warp_smem,
                        max_smem);
    if (p.block_smem_bytes > max_smem || p.block_smem_bytes % 16 ||
        p.block_smem_bytes / 4 - (p.block_threads / 32) * 128 - 3 * p.item_neighbors < 5 * 64)
        return ctx_fail(ctx, TC_ERR_INVALID_ARG, "block_smem_bytes out of range (max %d)", max_smem);
    if (out) *out = p;
    if (cfg) {
        cfg->warp_max_out_degree = p.warp_max_out_degree;
        cfg->warp_area_ints = p.warp_area_ints;
        cfg->warp_min_buckets = p.warp_min_buckets;
        cfg->warps_per_block = p.warps_per_block;
        cfg->block_threads = p.block_threads;
        cfg->block_smem_bytes = p.block_smem_bytes;
        cfg->item_neighbors = p.item_neighbors;
        cfg->chunk = p.chunk;
        cfg->shard_count = p.shard_count;
        cfg->shard_index = p.shard_index;
        cfg->record_timing = p.record_timing ? 1 : 0;
        cfg->hash_mode = p.hash_mode;
        cfg->quad_loads = p.scalar_loads ? 0 : 1;
        cfg->cycle_timing = p.record_timing == 2 ? 1 : 0;
        cfg->edge_centric = p.edge_centric;
        cfg->balance = p.balance;
        cfg->warp_order = p.warp_order;
        cfg->warp_grid = cfg->block_grid = 0;
    }
    return TC_OK;
}

tc_status tcg::check_csr(tc_ctx* ctx, const tc_csr* g) {
    if (!g) return ctx_fail(ctx, TC_ERR_INVALID_ARG, "graph is NULL");
    if (g->n < 0 || g->nnz < 0) return ctx_fail(ctx, TC_ERR_INVALID_ARG, "negative n or nnz");
    if (g->offset_bits != 32 && g->offset_bits != 64)
        return ctx_fail(ctx, TC_ERR_INVALID_ARG, "offset_bits must be 32 or 64");
    if (g->n > 0x7ffffffeLL) return ctx_fail(ctx, TC_ERR_UNSUPPORTED, "n must be < 2^31 - 1 (int32 vertex ids)");
    if (g->offset_bits == 32 && g->nnz > 0x7fffffffLL)
        return ctx_fail(ctx, TC_ERR_INVALID_ARG, "nnz >= 2^31 needs offset_bits = 64");
    if (g->n > 0 && !g->row_ptr) return ctx_fail(ctx, TC_ERR_INVALID_ARG, "row_ptr is NULL");
    if (g->nnz > 0 && !g->col) return ctx_fail(ctx, TC_ERR_INVALID_ARG, "col is NULL");
    return TC_OK;
}

// ------------------------------------------------------------ workspace use

tc_status tcg::ensure_count_ws(tc_ctx* ctx, Workspace& ws, int64_t n, int64_t m, cudaStream_t st) {
    tc_status s;
    if ((s = ws.warp_list.ensure(ctx, (size_t)(n + 1) * 4, st))) return s;
    if ((s = ws.warp_desc.ensure(ctx, (size_t)(n + 1) * 8, st))) return s;
    if ((s = ws.items.ensure(ctx, (size_t)item_capacity(n, m, ctx->cfg.item_neighbors) * sizeof(int2), st)))
        return s;
    if ((s = ws.ctr.ensure(ctx, sizeof(DevCounters) + 64, st))) return s;
    if (ctx->cfg.balance == TC_BALANCE_PC && (s = ws.pc.ensure(ctx, pc_scratch_bytes(ctx->cfg), st))) return s;
    return TC_OK;
}

tc_status tcg::ensure_orient_ws(tc_ctx* ctx, Workspace& ws, int64_t n, int64_t nnz, cudaStream_t st) {
    tc_status s;
    if ((s = ws.deg.ensure(ctx, (size_t)(n + 1) * 4, st))) return s;
    if ((s = ws.kept.ensure(ctx, (size_t)(n + 1) * 4, st))) return s;
    if ((s = ws.partial.ensure(ctx, (size_t)(scan_blocks(n) + 2) * 8, st))) return s;
    if ((s = ws.hubs.ensure(ctx, (size_t)(n + 1) * 4, st))) return s;
    if ((s = ws.kbits.ensure(ctx, (size_t)keep_bits_words(nnz) * 4, st))) return s;
    return ensure_count_ws(ctx, ws, n, nnz / 2, st);
}

// ---- phase timing (tc_params.record_timing) ----------------------------------

TimedCall* tcg::timing_begin(tc_ctx* ctx, bool oriented) {
    if (!ctx->cfg.record_timing) return nullptr;
    TimedCall tc;
    if (!ctx->timed_free.empty()) {
        tc = ctx->timed_free.back();
        ctx->timed_free.pop_back();
    } else {
        for (int i = 0; i < 4; ++i)
            if (cudaEventCreate(&tc.ev[i]) != cudaSuccess) {
                cudaGetLastError();
                for (int j = 0; j < i; ++j) cudaEventDestroy(tc.ev[j]);
                return nullptr;
            }
    }
    tc.oriented = oriented;
    ctx->timed.push_back(tc);
    return &ctx->timed.back();
}

void tcg::timing_mark(TimedCall* tc, int i, cudaStream_t st) {
    if (tc) cudaEventRecord(tc->ev[i], st);
}

// Enqueue orientation into (dag_ptr, dag_col[cap]) using ws scratch.
static tc_status enqueue_orient(tc_ctx* ctx, Workspace& ws, const tc_csr* g, int32_t* dag_ptr, int32_t* dag_col,
                                int64_t cap, cudaStream_t st) {
    DevCounters* ctr = (DevCounters*)ws.ctr.p;
    long long nl = 0;
    cudaError_t e = launch_orient(g->row_ptr, g->offset_bits, g->col, g->n, g->nnz, (int32_t*)ws.deg.p,
                                  (int32_t*)ws.kept.p, (long long*)ws.partial.p, dag_ptr, dag_col, cap,
                                  (int32_t*)ws.hubs.p, (unsigned*)ws.kbits.p, ctr, ctx->num_sms, st, &nl);
    ctx->launches += nl;
    if (g->n == 0 && e == cudaSuccess) e = cudaMemsetAsync(dag_ptr, 0, sizeof(int32_t), st);
    return cuda_status(ctx, e, "orientation kernels");
}

// Binning + counting; tm (may be null) gets events 2 (after binning) and 3.
// dag_bnd / max_m: a row-local DAG's (start, length) pairs and the most kept
// entries the input allows (nullptr / -1 for a compact DAG).
static tc_status enqueue_count(tc_ctx* ctx, Workspace& ws, const int32_t* dag_ptr, const int32_t* dag_col,
                               int64_t n, uint64_t* per_vertex, cudaStream_t st, TimedCall* tm,
                               const int2* dag_bnd = nullptr, long long max_m = -1,
                               const int32_t* ncol = nullptr) {
    DevCounters* ctr = (DevCounters*)ws.ctr.p;
    cudaError_t e = cudaSuccess;
    long long nl = 0;
    if (per_vertex && n > 0) e = cudaMemsetAsync(per_vertex, 0, (size_t)n * 8, st);
    if (e == cudaSuccess && n > 0) {
        int64_t m_cap = ws.items.bytes / sizeof(int2);
        // ordered work items: binning writes into items2, then placement into items
        const bool order_items = BLOCK_ITEM_ORDER && ncol && ws.items2.p && ws.ikey.p;
        if (order_items) {
            const int64_t c2 = (int64_t)(ws.items2.bytes / sizeof(int2)), c3 = (int64_t)(ws.ikey.bytes / 4);
            m_cap = std::min(m_cap, std::min(c2, c3));
        }
        e = launch_bin(dag_ptr, n, ctx->cfg, (int32_t*)ws.warp_list.p, (int2*)ws.warp_desc.p, (int2*)ws.items.p,
                       m_cap, ctr, ctx->num_sms, st, &nl, dag_bnd, max_m, ncol, (int32_t*)ws.okey.p,
                       (int32_t*)ws.ohist.p, (long long*)ws.partial.p, order_items ? dag_col : nullptr,
                       order_items ? (int32_t*)ws.ikey.p : nullptr, order_items ? (int2*)ws.items2.p : nullptr);
        timing_mark(tm, 2, st);
        if (e == cudaSuccess)
            e = launch_count(dag_ptr, dag_col, n, (const int32_t*)ws.warp_list.p, (const int2*)ws.warp_desc.p,
                             (const int2*)ws.items.p, (unsigned long long*)per_vertex, ctx->cfg, ctr, st, &nl,
                             dag_bnd, (int2*)ws.pc.p);
    } else {
        timing_mark(tm, 2, st);
    }
    timing_mark(tm, 3, st);
    ctx->launches += nl;
    return cuda_status(ctx, e, "counting kernels");
}

// The ordered warp list (tc_params.warp_order) for a row-local count of a
// graph with nnz adjacency entries in col: col when the order applies (the
// key and histogram arrays ensured), else null.
static tc_status order_keys(tc_ctx* ctx, Workspace& ws, int64_t n, int64_t nnz, const int32_t* col,
                            cudaStream_t st, const int32_t** ncol) {
    *ncol = nullptr;
    const int mode = ctx->cfg.warp_order;
    if (n <= 0 || mode == 2 || (mode == 0 && nnz < (1LL << 24))) return TC_OK;
    tc_status s;
    if ((s = ws.okey.ensure(ctx, (size_t)(n + 1) * 4, st))) return s;
    if ((s = ws.ohist.ensure(ctx, (size_t)(n + 1) * 4, st))) return s;
    if ((s = ws.partial.ensure(ctx, (size_t)(scan_blocks(n) + 2) * 8, st))) return s;
    if (BLOCK_ITEM_ORDER) {
        const size_t cap = (size_t)item_capacity(n, nnz / 2, ctx->cfg.item_neighbors);
        if ((s = ws.ikey.ensure(ctx, cap * 4, st))) return s;
        if ((s = ws.items2.ensure(ctx, cap * sizeof(int2), st))) return s;
    }
    *ncol = col;
    return TC_OK;
}

// Read the 64-byte counters back (blocking) and map error bits.
static tc_status read_counters(tc_ctx* ctx, Workspace& ws, cudaStream_t st, DevCounters* out) {
    cudaError_t e = cudaMemcpyAsync(ctx->host_ctr, ws.ctr.p, sizeof(DevCounters), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    tc_status s = cuda_status(ctx, e, "reading device counters");
    if (s) return s;
    *out = *ctx->host_ctr;
    if (out->err) return ctx_fail(ctx, err_bits_status(out->err), "%s", err_bits_text(out->err));
    ctx->cyc_build += (long long)out->cyc_build;
    ctx->cyc_probe += (long long)out->cyc_probe;
    return TC_OK;
}

tc_status tcg::orient_to_workspace(tc_ctx* ctx, const tc_csr* g, cudaStream_t st, int64_t* m) {
    Workspace& ws = ctx->ws;
    tc_status s = ensure_orient_ws(ctx, ws, g->n, g->nnz, st);
    if (!s) s = ws.dag_ptr.ensure(ctx, (size_t)(g->n + 1) * 4, st);
    if (!s) s = ws.dag_col.ensure(ctx, (size_t)(g->nnz / 2 + 1) * 4, st);
    if (!s) s = cuda_status(ctx, cudaMemsetAsync(ws.ctr.p, 0, sizeof(DevCounters), st), "memset counters");
    if (!s) s = enqueue_orient(ctx, ws, g, (int32_t*)ws.dag_ptr.p, (int32_t*)ws.dag_col.p, g->nnz / 2 + 1, st);
    DevCounters c;
    if (!s) s = read_counters(ctx, ws, st, &c);
    if (!s) *m = c.m;
    return s;
}

// ------------------------------------------------------------------ C ABI

extern "C" {

tc_status tc_default_params(tc_params* p) {
    if (!p) return TC_ERR_INVALID_ARG;
    fill_defaults(p);
    return TC_OK;
}

tc_status tc_create(tc_ctx** out, int device, size_t mem_budget_bytes, const tc_params* p) {
    if (!out) return TC_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return ctx_fail(nullptr, TC_ERR_CUDA, "no CUDA device available");
    }
    if (device < 0 || device >= ndev) return ctx_fail(nullptr, TC_ERR_INVALID_ARG, "device %d out of range", device);
    tc_ctx* ctx = new (std::nothrow) tc_ctx();
    if (!ctx) return TC_ERR_OOM;
    ctx->device = device;
    ctx->mem_budget = mem_budget_bytes;
    DeviceGuard dg(device);
    cudaDeviceProp prop;
    tc_status s = cuda_status(ctx, cudaGetDeviceProperties(&prop, device), "cudaGetDeviceProperties");
    if (!s) {
        ctx->num_sms = prop.multiProcessorCount;
        ctx->max_smem_optin = (int)prop.sharedMemPerBlockOptin;
        s = resolve_params(ctx, p, &ctx->params, &ctx->cfg);
    }
    if (!s) s = cuda_status(ctx, count_kernel_setup(ctx->cfg, ctx->num_sms), "count kernel setup");
    if (!s) s = cuda_status(ctx, cudaMallocHost(&ctx->host_ctr, sizeof(DevCounters) + 64), "cudaMallocHost");
    if (!s) s = ctx->ws.ctr.ensure(ctx, sizeof(DevCounters) + 64, 0);
    if (!s) s = ctx->out_scalars.ensure(ctx, 64, 0);
    if (s) {
        memcpy(g_create_error, ctx->last_error, sizeof(g_create_error));
        tc_destroy(ctx);
        return s;
    }
    *out = ctx;
    return TC_OK;
}

tc_status tc_destroy(tc_ctx* ctx) {
    if (!ctx) return TC_OK;
    {
        DeviceGuard dg(ctx->device);
        serve_shutdown(ctx);
        batch_release(ctx);
        cudaDeviceSynchronize();
        cudaGetLastError();
        ctx->ws.release_all(ctx);
        ctx->out_scalars.release(ctx);
        ctx->csr_copy.release_all(ctx);
        for (auto* v : {&ctx->timed, &ctx->timed_free})
            for (auto& t : *v)
                for (int i = 0; i < 4; ++i) cudaEventDestroy(t.ev[i]);
        ctx->timed.clear();
        ctx->timed_free.clear();
        for (auto& kv : ctx->dags) {
            cudaFree(kv.first);
            cudaFree(kv.second);
        }
        ctx->dags.clear();
        for (cudaEvent_t& e : ctx->aux_ev)
            if (e) cudaEventDestroy(e);
        if (ctx->aux_stream) cudaStreamDestroy(ctx->aux_stream);
        if (ctx->host_ctr) cudaFreeHost(ctx->host_ctr);
        ctx->host_ctr = nullptr;
    }
    delete ctx;
    return TC_OK;
}

tc_status tc_set_params(tc_ctx* ctx, const tc_params* p) {
    if (!ctx || !p) return TC_ERR_INVALID_ARG;
    DeviceGuard dg(ctx->device);
    tc_params np;
    CountCfg cfg;
    tc_status s = resolve_params(ctx, p, &np, &cfg);
    if (s) return s;
    s = cuda_status(ctx, count_kernel_setup(cfg, ctx->num_sms), "count kernel setup");
    if (s) return s;
    ctx->params = np;
    ctx->cfg = cfg;
    ctx->cfg_version++;
    return TC_OK;
}

tc_status tc_get_params(tc_ctx* ctx, tc_params* p) {
    if (!ctx || !p) return TC_ERR_INVALID_ARG;
    *p = ctx->params;
    return TC_OK;
}

tc_status tc_reserve(tc_ctx* ctx, int64_t n, int64_t nnz) {
    if (!ctx || n < 0 || nnz < 0) return TC_ERR_INVALID_ARG;
    DeviceGuard dg(ctx->device);
    tc_status s = ensure_orient_ws(ctx, ctx->ws, n, nnz, 0);
    if (s) return s;
    if ((s = ctx->ws.dag_ptr.ensure(ctx, (size_t)(n + 1) * 4, 0))) return s;
    return ctx->ws.dag_col.ensure(ctx, (size_t)(nnz / 2 + 1) * 4, 0);
}

tc_status tc_orient(tc_ctx* ctx, const tc_csr* g, tc_dag* out, void* stream) {
    if (!ctx || !out) return TC_ERR_INVALID_ARG;
    tc_status s = check_csr(ctx, g);
    if (s) return s;
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = ensure_orient_ws(ctx, ctx->ws, g->n, g->nnz, st))) return s;
    const int64_t cap = g->nnz / 2 + 1;
    int32_t* dp = nullptr;
    int32_t* dc = nullptr;
    if (injected_oom(ctx)) return ctx_fail(ctx, TC_ERR_OOM, "cudaMalloc(dag): out of memory (injected by tc_inject_oom)");
    cudaError_t e = cudaMalloc(&dp, (size_t)(g->n + 1) * 4);
    if (e == cudaSuccess) e = cudaMalloc(&dc, (size_t)cap * 4);
    if (e != cudaSuccess) {
        cudaFree(dp);
        return cuda_status(ctx, e, "cudaMalloc(dag)");
    }
    s = cuda_status(ctx, cudaMemsetAsync(ctx->ws.ctr.p, 0, sizeof(DevCounters), st), "memset counters");
    if (!s) s = enqueue_orient(ctx, ctx->ws, g, dp, dc, cap, st);
    DevCounters c;
    if (!s) s = read_counters(ctx, ctx->ws, st, &c);
    if (s) {
        cudaFree(dp);
        cudaFree(dc);
        return s;
    }
    ctx->dags[dp] = dc;
    out->n = g->n;
    out->m = c.m;
    out->dag_ptr = dp;
    out->dag_col = dc;
    return TC_OK;
}

tc_status tc_dag_free(tc_ctx* ctx, tc_dag* dag) {
    if (!ctx || !dag) return TC_ERR_INVALID_ARG;
    auto it = ctx->dags.find(dag->dag_ptr);
    if (it == ctx->dags.end() || it->second != dag->dag_col)
        return ctx_fail(ctx, TC_ERR_INVALID_ARG, "DAG was not created by tc_orient on this context");
    DeviceGuard dg(ctx->device);
    cudaFree(it->first);
    cudaFree(it->second);
    ctx->dags.erase(it);
    dag->dag_ptr = dag->dag_col = nullptr;
    dag->n = dag->m = 0;
    return TC_OK;
}

tc_status tc_count_dag(tc_ctx* ctx, const tc_dag* dag, uint64_t* count_host, uint64_t* per_vertex_device,
                       void* stream) {
    if (!ctx || !dag || !count_host) return TC_ERR_INVALID_ARG;
    if (dag->n < 0 || dag->m < 0 || dag->m > 0x7fffffffLL || (dag->n > 0 && !dag->dag_ptr) ||
        (dag->m > 0 && !dag->dag_col))
        return ctx_fail(ctx, TC_ERR_INVALID_ARG, "bad tc_dag");
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    tc_status s = ensure_count_ws(ctx, ctx->ws, dag->n, dag->m, st);
    if (s) return s;
    const int32_t* ncol = nullptr;  // ordered warp list: keys from the DAG's own lists
    if ((s = order_keys(ctx, ctx->ws, dag->n, 2 * dag->m, dag->dag_col, st, &ncol))) return s;
    s = cuda_status(ctx, cudaMemsetAsync(ctx->ws.ctr.p, 0, sizeof(DevCounters), st), "memset counters");
    TimedCall* tm = timing_begin(ctx, false);
    timing_mark(tm, 0, st);
    timing_mark(tm, 1, st);
    if (!s)
        s = enqueue_count(ctx, ctx->ws, dag->dag_ptr, dag->dag_col, dag->n, per_vertex_device, st, tm, nullptr, -1,
                          ncol);
    DevCounters c;
    if (!s) s = read_counters(ctx, ctx->ws, st, &c);
    if (s) return s;
    *count_host = c.total;
    return TC_OK;
}

tc_status tc_count_async(tc_ctx* ctx, const tc_csr* g, uint64_t* count_device, int32_t* error_device,
                         void* stream) {
    if (!ctx || !count_device) return TC_ERR_INVALID_ARG;
    tc_status s = check_csr(ctx, g);
    if (s) return s;
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    Workspace& ws = ctx->ws;
    if ((s = ensure_orient_ws(ctx, ws, g->n, g->nnz, st))) return s;
    if ((s = ws.dag_ptr.ensure(ctx, (size_t)(g->n + 1) * 4, st))) return s;
    // row-local DAG (the oriented lists left in the CSR's row slots: no scan,
    // no compaction) whenever the offsets fit int32; else the compact DAG
    const bool row_local = g->nnz < 0x7fffffffLL && !ctx->cfg.edge_centric;
    const int32_t* ncol = nullptr;
    if (row_local) {
        if ((s = ws.bnd.ensure(ctx, (size_t)(g->n + 1) * 8, st))) return s;
        if ((s = ws.dag_col.ensure(ctx, (size_t)(g->nnz + 1) * 4, st))) return s;
        if ((s = order_keys(ctx, ws, g->n, g->nnz, g->col, st, &ncol))) return s;
    } else if ((s = ws.dag_col.ensure(ctx, (size_t)(g->nnz / 2 + 1) * 4, st))) {
        return s;
    }
    s = cuda_status(ctx, cudaMemsetAsync(ws.ctr.p, 0, sizeof(DevCounters), st), "memset counters");
    TimedCall* tm = s ? nullptr : timing_begin(ctx, true);
    timing_mark(tm, 0, st);
    if (row_local) {
        if (!s) {
            long long nl = 0;
            cudaError_t e = launch_orient(g->row_ptr, g->offset_bits, g->col, g->n, g->nnz, (int32_t*)ws.deg.p,
                                          (int32_t*)ws.kept.p, nullptr, nullptr, nullptr, 0, (int32_t*)ws.hubs.p,
                                          nullptr, (DevCounters*)ws.ctr.p, ctx->num_sms, st, &nl,
                                          (int2*)ws.bnd.p, (int32_t*)ws.dag_col.p);
            ctx->launches += nl;
            s = cuda_status(ctx, e, "orientation kernels");
        }
        timing_mark(tm, 1, st);
        if (!s)
            s = enqueue_count(ctx, ws, nullptr, (int32_t*)ws.dag_col.p, g->n, nullptr, st, tm, (int2*)ws.bnd.p,
                              g->nnz / 2, ncol);
    } else {
        if (!s) s = enqueue_orient(ctx, ws, g, (int32_t*)ws.dag_ptr.p, (int32_t*)ws.dag_col.p, g->nnz / 2 + 1, st);
        timing_mark(tm, 1, st);
        if (!s) s = enqueue_count(ctx, ws, (int32_t*)ws.dag_ptr.p, (int32_t*)ws.dag_col.p, g->n, nullptr, st, tm);
    }
    if (!s) {
        long long nl = 0;
        s = cuda_status(ctx,
                        launch_finish((DevCounters*)ws.ctr.p, (unsigned long long*)count_device, error_device, st,
                                      &nl),
                        "finish kernel");
        ctx->launches += nl;
    }
    return s;
}

tc_status tc_count(tc_ctx* ctx, const tc_csr* g, uint64_t* count_host, void* stream) {
    if (!ctx || !count_host) return TC_ERR_INVALID_ARG;
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    uint64_t* d_count = (uint64_t*)ctx->out_scalars.p;
    int32_t* d_err = (int32_t*)((char*)ctx->out_scalars.p + 8);
    tc_status s = tc_count_async(ctx, g, d_count, d_err, stream);
    if (s) return s;
    cudaError_t e = cudaMemcpyAsync(ctx->host_ctr, ctx->out_scalars.p, 16, cudaMemcpyDeviceToHost, st);
    DevCounters c{};
    if (e == cudaSuccess && ctx->cfg.cycle_timing)  // the workers' build / probe cycles
        e = cudaMemcpyAsync(&c, ctx->ws.ctr.p, sizeof(c), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if ((s = cuda_status(ctx, e, "reading the count"))) return s;
    ctx->cyc_build += (long long)c.cyc_build;
    ctx->cyc_probe += (long long)c.cyc_probe;
    uint64_t cnt;
    int32_t err;
    memcpy(&cnt, ctx->host_ctr, 8);
    memcpy(&err, (char*)ctx->host_ctr + 8, 4);
    if (err) return ctx_fail(ctx, (tc_status)err, "%s", tc_status_string((tc_status)err));
    *count_host = cnt;
    return TC_OK;
}

// tc_count_host for a graph that takes the row-local path: the neighbour
// lists are copied in kHostPieces pieces (row ranges of about equal entries,
// cut at 32-row groups) on a second stream, and the orientation's count pass
// runs on each piece as soon as it has landed, so orientation overlaps the
// transfer instead of following it.
constexpr int kHostPieces = 8;
static tc_status count_host_pieces(tc_ctx* ctx, const tc_csr* g, uint64_t* count_host, cudaStream_t st) {
    Workspace& ws = ctx->ws;
    const int64_t n = g->n, nnz = g->nnz;
    const size_t rp_bytes = (size_t)(n + 1) * (g->offset_bits / 8);
    tc_status s;
    if ((s = ctx->csr_copy.a.ensure(ctx, rp_bytes, st))) return s;
    if ((s = ctx->csr_copy.b.ensure(ctx, (size_t)nnz * 4 + 4, st))) return s;
    if ((s = ensure_orient_ws(ctx, ws, n, nnz, st))) return s;
    if ((s = ws.bnd.ensure(ctx, (size_t)(n + 1) * 8, st))) return s;
    if ((s = ws.dag_col.ensure(ctx, (size_t)(nnz + 1) * 4, st))) return s;
    const int32_t* ncol = nullptr;
    if ((s = order_keys(ctx, ws, n, nnz, (const int32_t*)ctx->csr_copy.b.p, st, &ncol))) return s;
    if (!ctx->aux_stream) {
        s = cuda_status(ctx, cudaStreamCreateWithFlags(&ctx->aux_stream, cudaStreamNonBlocking), "cudaStreamCreate");
        for (cudaEvent_t& e : ctx->aux_ev)
            if (!s) s = cuda_status(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "cudaEventCreate");
        if (s) return s;
    }
    // piece boundaries in 32-row groups, from the host row offsets
    auto rp_at = [&](int64_t r) -> int64_t {
        return g->offset_bits == 64 ? static_cast<const int64_t*>(g->row_ptr)[r]
                                    : (int64_t) static_cast<const int32_t*>(g->row_ptr)[r];
    };
    const int64_t groups = (n + 31) / 32;
    int64_t cuts[kHostPieces + 1];
    cuts[0] = 0;
    cuts[kHostPieces] = groups;
    for (int i = 1; i < kHostPieces; ++i) {
        const int64_t target = nnz * i / kHostPieces;
        int64_t lo = 0, hi = n;  // first row r with rp_at(r) >= target
        while (lo < hi) {
            const int64_t mid = (lo + hi) / 2;
            if (rp_at(mid) < target) lo = mid + 1;
            else hi = mid;
        }
        const int64_t gcut = lo / 32;
        cuts[i] = gcut < cuts[i - 1] ? cuts[i - 1] : (gcut > groups ? groups : gcut);
    }
    cudaEvent_t* ev = ctx->aux_ev;
    cudaError_t e = cudaEventRecord(ev[kHostPieces], st);  // earlier work on st is done with the buffers
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->aux_stream, ev[kHostPieces], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->csr_copy.a.p, g->row_ptr, rp_bytes, cudaMemcpyHostToDevice, st);
    for (int i = 0; i < kHostPieces && e == cudaSuccess; ++i) {
        const int64_t lo = rp_at(cuts[i] * 32 < n ? cuts[i] * 32 : n);
        const int64_t hi = rp_at(cuts[i + 1] * 32 < n ? cuts[i + 1] * 32 : n);
        if (hi > lo)
            e = cudaMemcpyAsync(static_cast<int32_t*>(ctx->csr_copy.b.p) + lo, g->col + lo, (size_t)(hi - lo) * 4,
                                cudaMemcpyHostToDevice, ctx->aux_stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev[i], ctx->aux_stream);
    }
    if ((s = cuda_status(ctx, e, "copying the CSR to the device"))) return s;
    s = cuda_status(ctx, cudaMemsetAsync(ws.ctr.p, 0, sizeof(DevCounters), st), "memset counters");
    TimedCall* tm = s ? nullptr : timing_begin(ctx, true);
    timing_mark(tm, 0, st);
    if (!s) {
        long long nl = 0;
        e = launch_orient_row_local_pieces(ctx->csr_copy.a.p, g->offset_bits, (const int32_t*)ctx->csr_copy.b.p, n,
                                           nnz, (int32_t*)ws.deg.p, (int32_t*)ws.kept.p, (int32_t*)ws.hubs.p,
                                           (int2*)ws.bnd.p, (int32_t*)ws.dag_col.p, (DevCounters*)ws.ctr.p,
                                           ctx->num_sms, st, &nl, cuts, kHostPieces, ev);
        ctx->launches += nl;
        s = cuda_status(ctx, e, "orientation kernels");
    }
    timing_mark(tm, 1, st);
    if (!s)
        s = enqueue_count(ctx, ws, nullptr, (int32_t*)ws.dag_col.p, n, nullptr, st, tm, (int2*)ws.bnd.p, nnz / 2,
                          ncol);
    uint64_t* d_count = (uint64_t*)ctx->out_scalars.p;
    int32_t* d_err = (int32_t*)((char*)ctx->out_scalars.p + 8);
    if (!s) {
        long long nl = 0;
        s = cuda_status(ctx, launch_finish((DevCounters*)ws.ctr.p, (unsigned long long*)d_count, d_err, st, &nl),
                        "finish kernel");
        ctx->launches += nl;
    }
    if (s) return s;
    e = cudaMemcpyAsync(ctx->host_ctr, ctx->out_scalars.p, 16, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if ((s = cuda_status(ctx, e, "reading the count"))) return s;
    uint64_t cnt;
    int32_t err;
    memcpy(&cnt, ctx->host_ctr, 8);
    memcpy(&err, (char*)ctx->host_ctr + 8, 4);
    if (err) return ctx_fail(ctx, (tc_status)err, "%s", tc_status_string((tc_status)err));
    *count_host = cnt;
    return TC_OK;
}

tc_status tc_count_host(tc_ctx* ctx, const tc_csr* g, uint64_t* count_host, void* stream) {
    if (!ctx || !count_host) return TC_ERR_INVALID_ARG;
    tc_status s = check_csr(ctx, g);
    if (s) return s;
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (g->n > 0 && g->nnz >= (1 << 20) && g->nnz < 0x7fffffffLL && !ctx->cfg.edge_centric &&
        !ctx->cfg.cycle_timing)
        return count_host_pieces(ctx, g, count_host, st);
    const size_t rp_bytes = (size_t)(g->n + 1) * (g->offset_bits / 8);
    const size_t col_bytes = (size_t)g->nnz * 4;
    if ((s = ctx->csr_copy.a.ensure(ctx, rp_bytes, st))) return s;
    if ((s = ctx->csr_copy.b.ensure(ctx, col_bytes + 4, st))) return s;
    cudaError_t e = cudaSuccess;
    if (g->n > 0 || g->row_ptr) e = cudaMemcpyAsync(ctx->csr_copy.a.p, g->row_ptr, rp_bytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && col_bytes)
        e = cudaMemcpyAsync(ctx->csr_copy.b.p, g->col, col_bytes, cudaMemcpyHostToDevice, st);
    if ((s = cuda_status(ctx, e, "copying the CSR to the device"))) return s;
    tc_csr dg2 = *g;
    dg2.row_ptr = ctx->csr_copy.a.p;
    dg2.col = (const int32_t*)ctx->csr_copy.b.p;
    return tc_count(ctx, &dg2, count_host, stream);
}

tc_status tc_dag_stats(tc_ctx* ctx, const tc_dag* dag, tc_stats* out, void* stream) {
    if (!ctx || !dag || !out) return TC_ERR_INVALID_ARG;
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    tc_status s = ctx->ws.stats.ensure(ctx, sizeof(DevStats), st);
    if (s) return s;
    cudaError_t e = cudaMemsetAsync(ctx->ws.stats.p, 0, sizeof(DevStats), st);
    if (e == cudaSuccess)
        e = launch_stats(dag->dag_ptr, dag->dag_col, dag->n, ctx->cfg.warp_max_out_degree, (DevStats*)ctx->ws.stats.p,
                         st);
    DevStats h;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, ctx->ws.stats.p, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if ((s = cuda_status(ctx, e, "statistics kernel"))) return s;
    out->n = dag->n;
    out->m = dag->m;
    out->max_out_degree = h.max_out;
    out->n_skip = h.n_skip;
    out->n_warp = h.n_warp;
    out->n_block = h.n_block;
    out->wedges_plus = (int64_t)h.wplus;
    out->wedges_plus_block = (int64_t)h.wplus_block;
    out->max_collision_mod32 = h.maxc[0];
    out->max_collision_mult32 = h.maxc[1];
    out->phi_mod32 = (int64_t)h.phi[0];
    out->phi_mult32 = (int64_t)h.phi[1];
    return TC_OK;
}

tc_status tc_read_timing(tc_ctx* ctx, tc_timing* out) {
    if (!ctx || !out) return TC_ERR_INVALID_ARG;
    DeviceGuard dg(ctx->device);
    tc_timing t{};
    tc_status s = TC_OK;
    for (auto& c : ctx->timed) {
        float a = 0.f, b = 0.f, d = 0.f;
        cudaError_t e = cudaEventSynchronize(c.ev[3]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&a, c.ev[0], c.ev[1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&b, c.ev[1], c.ev[2]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&d, c.ev[2], c.ev[3]);
        if (e != cudaSuccess && !s) s = cuda_status(ctx, e, "reading timing events");
        t.calls++;
        t.orient_ms += a;
        t.bin_ms += b;
        t.count_ms += d;
        ctx->timed_free.push_back(c);
    }
    ctx->timed.clear();
    if (s) return s;
    t.build_cycles = ctx->cyc_build;
    t.probe_cycles = ctx->cyc_probe;
    ctx->cyc_build = ctx->cyc_probe = 0;
    *out = t;
    return TC_OK;
}

tc_status tc_kernel_launches(tc_ctx* ctx, int64_t* out) {
    if (!ctx || !out) return TC_ERR_INVALID_ARG;
    *out = ctx->launches.load();
    return TC_OK;
}

tc_status tc_inject_oom(tc_ctx* ctx, int64_t nth) {
    if (!ctx || nth < 0) return TC_ERR_INVALID_ARG;
    ctx->fail_alloc_in.store((long long)nth);
    return TC_OK;
}

const char* tc_status_string(tc_status s) {
    switch (s) {
        case TC_OK: return "TC_OK";
        case TC_ERR_INVALID_ARG: return "TC_ERR_INVALID_ARG";
        case TC_ERR_BAD_GRAPH: return "TC_ERR_BAD_GRAPH";
        case TC_ERR_OOM: return "TC_ERR_OOM";
        case TC_ERR_BUSY: return "TC_ERR_BUSY";
        case TC_ERR_NOT_READY: return "TC_ERR_NOT_READY";
        case TC_ERR_TIMEOUT: return "TC_ERR_TIMEOUT";
        case TC_ERR_CUDA: return "TC_ERR_CUDA";
        case TC_ERR_UNSUPPORTED: return "TC_ERR_UNSUPPORTED";
    }
    return "unknown tc_status";
}

const char* tc_last_error(tc_ctx* ctx) { return ctx ? ctx->last_error : g_create_error; }

const char* tc_version(void) { return "trust-gb300 0.1 (sm_103a)"; }

}  // extern "C"
