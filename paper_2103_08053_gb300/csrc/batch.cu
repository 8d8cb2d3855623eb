// batch.cu -- tc_count_batch: many graphs in one pass.
//
// The k graphs are laid out in one padded global vertex space (graph i owns
// rows [vbase_i, vbase_i + n_i), vbase_i a multiple of 32), oriented by one
// launch sequence into one DAG whose ids are global, and counted by one launch
// of the persistent counting kernels whose work items are the vertices of all
// graphs (packs of small vertices, items of large ones, Sec. 4.3). The
// counting kernels write per-vertex counts; a segmented sum per graph gives
// the k results. The whole sequence -- descriptor upload, orientation,
// binning, counting, segmented sums, result download -- is captured once into
// a CUDA graph per batch shape and replayed while the shape stays the same.
#include <cstring>

#include "api_internal.h"

using namespace tcg;

namespace {

// counts[b] = sum of per_vertex over graph b's rows; one block per graph.
__global__ void k_segsum(const unsigned long long* __restrict__ per_vertex, const GraphRef* __restrict__ gs,
                         unsigned long long* __restrict__ counts) {
    __shared__ unsigned long long s[32];
    const GraphRef g = gs[blockIdx.x];
    unsigned long long acc = 0;
    for (long long i = threadIdx.x; i < g.n; i += blockDim.x) acc += per_vertex[g.vbase + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < (blockDim.x >> 5) ? s[threadIdx.x] : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(FULL, acc, o);
        if (threadIdx.x == 0) counts[blockIdx.x] = acc;
    }
}

}  // namespace

// ---------------------------------------------------------------- BatchRunner

tc_status BatchRunner::init(tc_ctx* ctx) {
    tc_status s = cuda_status(ctx, cudaStreamCreateWithPriority(&stream, cudaStreamNonBlocking, priority),
                              "cudaStreamCreateWithPriority");
    if (!s) s = cuda_status(ctx, cudaEventCreateWithFlags(&ev_in, cudaEventDisableTiming), "cudaEventCreate");
    if (!s) s = cuda_status(ctx, cudaEventCreateWithFlags(&ev_done, cudaEventDisableTiming), "cudaEventCreate");
    return s;
}

void BatchRunner::drop_graph() {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    key_k = -1;
}

void BatchRunner::release(tc_ctx* ctx) {
    if (stream) cudaStreamSynchronize(stream);
    drop_graph();
    ws.release_all(ctx);
    for (DevBuf* b : {&graphs, &per_vertex, &counts, &dag_ptr, &dag_col}) b->release(ctx);
    if (h_graphs) cudaFreeHost(h_graphs);
    if (h_counts) cudaFreeHost(h_counts);
    if (h_ctr) cudaFreeHost(h_ctr);
    h_graphs = nullptr;
    h_counts = nullptr;
    h_ctr = nullptr;
    h_cap = 0;
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_done) cudaEventDestroy(ev_done);
    if (stream) cudaStreamDestroy(stream);
    ev_in = ev_done = nullptr;
    stream = nullptr;
}

// Grows `b` and records whether it moved (a captured graph would point at the
// old memory).
static tc_status ensure_tracked(tc_ctx* ctx, DevBuf& b, size_t need, cudaStream_t st, bool& moved) {
    void* before = b.p;
    tc_status s = b.ensure(ctx, need, st);
    if (b.p != before) moved = true;
    return s;
}

tc_status BatchRunner::prepare(tc_ctx* ctx, const tc_csr* gs, int k) {
    if (k <= 0) return ctx_fail(ctx, TC_ERR_INVALID_ARG, "batch of %d graphs", k);
    if (!gs) return ctx_fail(ctx, TC_ERR_INVALID_ARG, "graphs is NULL");
    bits = gs[0].offset_bits;
    long long vb = 0, nnz = 0;
    for (int i = 0; i < k; ++i) {
        tc_status s = check_csr(ctx, &gs[i]);
        if (s) return ctx_fail(ctx, s, "graph %d: %s", i, ctx->last_error);
        if (gs[i].offset_bits != bits)
            return ctx_fail(ctx, TC_ERR_UNSUPPORTED, "all graphs of a batch must share offset_bits");
        vb += (gs[i].n + 31) / 32 * 32;
        nnz += gs[i].nnz;
    }
    if (vb >= 0x7fffffffLL) return ctx_fail(ctx, TC_ERR_UNSUPPORTED, "batch has 2^31 or more (padded) vertices");
    total = vb;
    nnz_total = nnz;
    this->k = k;
    if (k > h_cap) {
        if (h_graphs) cudaFreeHost(h_graphs);
        if (h_counts) cudaFreeHost(h_counts);
        h_graphs = nullptr;
        h_counts = nullptr;
        h_cap = 0;
        tc_status s = cuda_status(ctx, cudaMallocHost(&h_graphs, sizeof(GraphRef) * (size_t)k), "cudaMallocHost");
        if (!s) s = cuda_status(ctx, cudaMallocHost(&h_counts, sizeof(uint64_t) * (size_t)k), "cudaMallocHost");
        if (s) return s;
        h_cap = k;
        moved = true;
    }
    if (!h_ctr) {
        tc_status s = cuda_status(ctx, cudaMallocHost(&h_ctr, sizeof(DevCounters)), "cudaMallocHost");
        if (s) return s;
        moved = true;
    }
    long long base = 0, ebase = 0;
    for (int i = 0; i < k; ++i) {
        h_graphs[i] = GraphRef{gs[i].row_ptr, gs[i].col, gs[i].n, gs[i].nnz, base, ebase};
        base += (gs[i].n + 31) / 32 * 32;
        ebase += gs[i].nnz;
    }
    // row-local DAG (lists left in the rows' slots of one array of all the
    // batch's entries) when the entry offsets fit int32
    row_local = nnz_total < 0x7fffffffLL && !ctx->cfg.edge_centric;
    tc_status s;
    bool mv = false;
    if ((s = ensure_tracked(ctx, graphs, sizeof(GraphRef) * (size_t)k, stream, mv))) return s;
    if ((s = ensure_tracked(ctx, counts, sizeof(uint64_t) * (size_t)k, stream, mv))) return s;
    if ((s = ensure_tracked(ctx, per_vertex, sizeof(uint64_t) * (size_t)(total + 1), stream, mv))) return s;
    if ((s = ensure_tracked(ctx, dag_ptr, sizeof(int32_t) * (size_t)(total + 1), stream, mv))) return s;
    if ((s = ensure_tracked(ctx, dag_col, sizeof(int32_t) * (size_t)(row_local ? nnz_total + 1 : nnz_total / 2 + 1),
                            stream, mv)))
        return s;
    if (row_local && (s = ensure_tracked(ctx, ws.bnd, sizeof(int2) * (size_t)(total + 1), stream, mv))) return s;
    if ((s = ensure_tracked(ctx, ws.deg, (size_t)(total + 1) * 4, stream, mv))) return s;
    if ((s = ensure_tracked(ctx, ws.kept, (size_t)(total + 1) * 4, stream, mv))) return s;
    if ((s = ensure_tracked(ctx, ws.partial, (size_t)(scan_blocks(total) + 2) * 8, stream, mv))) return s;
    if ((s = ensure_tracked(ctx, ws.hubs, (size_t)(total + 1) * 4, stream, mv))) return s;
    if ((s = ensure_tracked(ctx, ws.warp_list, (size_t)(total + 1) * 4, stream, mv))) return s;
    if ((s = ensure_tracked(ctx, ws.warp_desc, (size_t)(total + 1) * 8, stream, mv))) return s;
    if ((s = ensure_tracked(ctx, ws.items,
                            (size_t)item_capacity(total, nnz_total / 2, ctx->cfg.item_neighbors) * sizeof(int2), stream,
                            mv)))
        return s;
    if ((s = ensure_tracked(ctx, ws.ctr, sizeof(DevCounters) + 64, stream, mv))) return s;
    if (ctx->cfg.balance == TC_BALANCE_PC && (s = ensure_tracked(ctx, ws.pc, pc_scratch_bytes(ctx->cfg), stream, mv)))
        return s;
    if (mv) moved = true;
    return TC_OK;
}

// The whole batch, enqueued on `stream` (also used for capture).
tc_status BatchRunner::enqueue(tc_ctx* ctx) {
    DevCounters* ctr = (DevCounters*)ws.ctr.p;
    long long nl = 0;
    cudaError_t e = cudaMemcpyAsync(graphs.p, h_graphs, sizeof(GraphRef) * (size_t)k, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctr, 0, sizeof(DevCounters), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(per_vertex.p, 0, sizeof(uint64_t) * (size_t)total, stream);
    int2* bnd = row_local ? (int2*)ws.bnd.p : nullptr;
    if (e == cudaSuccess)
        e = launch_orient_batch((const GraphRef*)graphs.p, k, bits, total, (int32_t*)ws.deg.p, (int32_t*)ws.kept.p,
                                (long long*)ws.partial.p, (int32_t*)dag_ptr.p, (int32_t*)dag_col.p,
                                nnz_total / 2 + 1, (int32_t*)ws.hubs.p, ctr, ctx->num_sms, stream, &nl, bnd,
                                row_local ? (int32_t*)dag_col.p : nullptr, nnz_total);
    if (e == cudaSuccess)
        e = launch_bin((const int32_t*)dag_ptr.p, total, ctx->cfg, (int32_t*)ws.warp_list.p, (int2*)ws.warp_desc.p,
                       (int2*)ws.items.p, (int64_t)(ws.items.bytes / sizeof(int2)), ctr, ctx->num_sms, stream,
                       &nl, bnd, row_local ? nnz_total / 2 : -1);
    CountCfg cfg = ctx->cfg;
    cfg.pop_contiguous = 1;  // warps on a few graphs at a time: their lists stay in L2
    if (grid_share < 1.0f) {  // leave SMs to runners on other streams
        cfg.warp_grid = cfg.warp_grid * grid_share < 1.0f ? 1 : (int)(cfg.warp_grid * grid_share);
        cfg.block_grid = cfg.block_grid * grid_share < 1.0f ? 1 : (int)(cfg.block_grid * grid_share);
    }
    if (e == cudaSuccess)
        e = launch_count((const int32_t*)dag_ptr.p, (const int32_t*)dag_col.p, total,
                         (const int32_t*)ws.warp_list.p, (const int2*)ws.warp_desc.p, (const int2*)ws.items.p,
                         (unsigned long long*)per_vertex.p, cfg, ctr, stream, &nl, bnd, (int2*)ws.pc.p);
    if (e == cudaSuccess) {
        k_segsum<<<k, 256, 0, stream>>>((const unsigned long long*)per_vertex.p, (const GraphRef*)graphs.p,
                                        (unsigned long long*)counts.p);
        nl += 1;
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h_counts, counts.p, sizeof(uint64_t) * (size_t)k, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_ctr, ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, stream);
    enqueued_launches = nl;
    return cuda_status(ctx, e, "batch kernels");
}

tc_status BatchRunner::launch(tc_ctx* ctx, bool use_graph) {
    if (!use_graph) {
        tc_status s = enqueue(ctx);
        ctx->launches += enqueued_launches;
        return s;
    }
    const bool same = exec && !moved && key_k == k && key_total == total && key_nnz == nnz_total &&
                      key_bits == bits && key_cfg == ctx->cfg_version;
    if (!same) {
        drop_graph();
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_status(ctx, e, "cudaStreamBeginCapture");
        tc_status s = enqueue(ctx);
        captured_launches = enqueued_launches;  // recorded in the graph, run at each replay
        e = cudaStreamEndCapture(stream, &g);
        if (s) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            exec = nullptr;
            return cuda_status(ctx, e, "capturing the batch graph");
        }
        key_k = k;
        key_total = total;
        key_nnz = nnz_total;
        key_bits = bits;
        key_cfg = ctx->cfg_version;
        moved = false;
    }
    ctx->launches += captured_launches;  // every replay runs the captured kernels
    return cuda_status(ctx, cudaGraphLaunch(exec, stream), "cudaGraphLaunch");
}

tc_status BatchRunner::finish(tc_ctx* ctx, uint64_t* counts_host) {
    tc_status s = cuda_status(ctx, cudaStreamSynchronize(stream), "batch synchronisation");
    if (s) return s;
    if (h_ctr->err) return ctx_fail(ctx, err_bits_status(h_ctr->err), "%s", err_bits_text(h_ctr->err));
    memcpy(counts_host, h_counts, sizeof(uint64_t) * (size_t)k);
    return TC_OK;
}

void tcg::batch_release(tc_ctx* ctx) {
    if (ctx->batch) {
        ctx->batch->release(ctx);
        delete ctx->batch;
        ctx->batch = nullptr;
    }
}

extern "C" tc_status tc_count_batch(tc_ctx* ctx, const tc_csr* gs, int32_t k, uint64_t* counts_host, void* stream) {
    if (!ctx || !counts_host || (k > 0 && !gs) || k < 0) return TC_ERR_INVALID_ARG;
    if (k == 0) return TC_OK;
    DeviceGuard dg(ctx->device);
    if (!ctx->batch) {
        ctx->batch = new (std::nothrow) BatchRunner();
        if (!ctx->batch) return TC_ERR_OOM;
        tc_status s = ctx->batch->init(ctx);
        if (s) {
            batch_release(ctx);
            return s;
        }
    }
    BatchRunner& r = *ctx->batch;
    // the caller's prior work on `stream` (e.g. uploads of the graphs) comes first
    cudaError_t e = cudaEventRecord(r.ev_in, (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(r.stream, r.ev_in, 0);
    tc_status s = cuda_status(ctx, e, "ordering after the caller's stream");
    if (!s) s = r.prepare(ctx, gs, k);
    if (!s) s = r.launch(ctx, true);
    if (!s) s = r.finish(ctx, counts_host);
    return s;
}
