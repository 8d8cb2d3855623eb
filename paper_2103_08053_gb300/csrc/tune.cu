// tune.cu -- tc_autotune: pick warp-worker threshold, table sizes, queue
// chunk, thread-block worker shape and item size for a workload by measurement.
//
// Coordinate search: starting from the context's parameters, each knob in
// turn is set to each of its candidate values (the others held at their best
// so far), the workload is counted (tc_count for one graph, tc_count_batch
// for several), and the fastest value is kept. A trial is timed as the best of
// two runs after one warm-up run (which also captures the batch's CUDA graph).
// Results can be cached in a text file: one line per workload signature
// "sig <k> <n> <nnz> <bits> <maxdeg class> : <field>=<value> ...".
#include <chrono>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "api_internal.h"

using namespace tcg;

namespace {

struct Knob {
    const char* name;
    int32_t tc_params::*field;
    std::vector<int32_t> values;
};

std::string signature(const tc_csr* gs, int k) {
    long long n = 0, nnz = 0;
    for (int i = 0; i < k; ++i) {
        n += gs[i].n;
        nnz += gs[i].nnz;
    }
    // coarse size classes: the same workload family tunes the same way
    auto cls = [](long long x) {
        int c = 0;
        while (x > 1) {
            x >>= 1;
            ++c;
        }
        return c;
    };
    char buf[128];
    snprintf(buf, sizeof(buf), "sig k%d n%d nnz%d bits%d", cls(k), cls(n), cls(nnz), gs[0].offset_bits);
    return buf;
}

bool cache_lookup(const char* path, const std::string& sig, tc_params* p) {
    if (!path) return false;
    FILE* f = fopen(path, "r");
    if (!f) return false;
    char line[1024];
    bool found = false;
    while (fgets(line, sizeof(line), f)) {
        if (strncmp(line, sig.c_str(), sig.size()) != 0 || line[sig.size()] != ' ') continue;
        tc_params q = *p;
        char* save = nullptr;
        for (char* tok = strtok_r(line + sig.size(), " \n", &save); tok; tok = strtok_r(nullptr, " \n", &save)) {
            char name[64];
            int v;
            if (sscanf(tok, "%63[^=]=%d", name, &v) != 2) continue;
            if (!strcmp(name, "warp_max_out_degree")) q.warp_max_out_degree = v;
            else if (!strcmp(name, "warp_area_ints")) q.warp_area_ints = v;
            else if (!strcmp(name, "warp_min_buckets")) q.warp_min_buckets = v;
            else if (!strcmp(name, "chunk")) q.chunk = v;
            else if (!strcmp(name, "warps_per_block")) q.warps_per_block = v;
            else if (!strcmp(name, "item_neighbors")) q.item_neighbors = v;
            else if (!strcmp(name, "block_threads")) q.block_threads = v;
            else if (!strcmp(name, "block_smem_bytes")) q.block_smem_bytes = v;
        }
        *p = q;
        found = true;  // the last matching line wins
    }
    fclose(f);
    return found;
}

void cache_store(const char* path, const std::string& sig, const tc_params& p) {
    if (!path) return;
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s : warp_max_out_degree=%d warp_area_ints=%d warp_min_buckets=%d chunk=%d warps_per_block=%d "
               "item_neighbors=%d block_threads=%d block_smem_bytes=%d\n",
            sig.c_str(), p.warp_max_out_degree, p.warp_area_ints, p.warp_min_buckets, p.chunk, p.warps_per_block,
            p.item_neighbors, p.block_threads, p.block_smem_bytes);
    fclose(f);
}

// One timed trial: best of two runs after a warm-up; <0 when the candidate
// is invalid or fails.
double trial(tc_ctx* ctx, const tc_params& p, const tc_csr* gs, int k, void* stream, std::vector<uint64_t>& out,
             std::vector<uint64_t>& ref) {
    if (tc_set_params(ctx, &p) != TC_OK) return -1.0;
    double best = 1e30;
    for (int rep = 0; rep < 3; ++rep) {
        const auto t0 = std::chrono::steady_clock::now();
        tc_status s = (k == 1) ? tc_count(ctx, gs, out.data(), stream) : tc_count_batch(ctx, gs, k, out.data(), stream);
        const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        if (s != TC_OK) return -1.0;
        if (rep > 0 && ms < best) best = ms;
    }
    if (ref.empty()) ref = out;
    if (out != ref) return -2.0;  // a count changed: never accept (it cannot, but do not trust a tuner blindly)
    return best;
}

}  // namespace

extern "C" tc_status tc_autotune(tc_ctx* ctx, const tc_csr* gs, int32_t k, const char* cache_path,
                                 tc_params* best_out, void* stream) {
    if (!ctx || !gs || k <= 0) return TC_ERR_INVALID_ARG;
    const std::string sig = signature(gs, k);
    tc_params best = ctx->params;
    if (cache_lookup(cache_path, sig, &best)) {
        tc_status s = tc_set_params(ctx, &best);
        if (s == TC_OK) {
            if (best_out) *best_out = best;
            return TC_OK;
        }
        best = ctx->params;  // a stale cache line: tune afresh
    }
    std::vector<uint64_t> out((size_t)k), ref;
    double best_ms = trial(ctx, best, gs, k, stream, out, ref);
    if (best_ms < 0) return ctx_fail(ctx, TC_ERR_INVALID_ARG, "autotune: the starting parameters fail");
    // warp_max_out_degree moves together with the table area it needs
    const int tws[] = {32, 64, 128, 255};
    for (int tw : tws) {
        tc_params p = best;
        p.warp_max_out_degree = tw;
        p.warp_area_ints = pack_table_ints(tw, p.warp_min_buckets);
        const double ms = trial(ctx, p, gs, k, stream, out, ref);
        if (ms >= 0 && ms < best_ms) {
            best_ms = ms;
            best = p;
        }
    }
    // thread-block workers: threads, shared memory and item size move together
    const int blocks[][3] = {{1024, 200 * 1024, 1024}, {512, 100 * 1024, 512}, {256, 50 * 1024, 256}};
    for (const auto& b : blocks) {
        tc_params p = best;
        p.block_threads = b[0];
        p.block_smem_bytes = b[1];
        p.item_neighbors = b[2];
        const double ms = trial(ctx, p, gs, k, stream, out, ref);
        if (ms >= 0 && ms < best_ms) {
            best_ms = ms;
            best = p;
        }
    }
    const Knob knobs[] = {
        {"warp_min_buckets", &tc_params::warp_min_buckets, {16, 32, 64}},
        {"chunk", &tc_params::chunk, {8, 16, 32}},
        {"warps_per_block", &tc_params::warps_per_block, {4, 8}},
        {"item_neighbors", &tc_params::item_neighbors, {256, 512, 1024}},
    };
    for (const Knob& kn : knobs) {
        for (int32_t v : kn.values) {
            tc_params p = best;
            p.*(kn.field) = v;
            if (kn.field == &tc_params::warp_min_buckets) {
                const int need = pack_table_ints(p.warp_max_out_degree, v);
                if (p.warp_area_ints < need) p.warp_area_ints = need;
            }
            if (kn.field == &tc_params::item_neighbors && v > p.block_threads) continue;
            const double ms = trial(ctx, p, gs, k, stream, out, ref);
            if (ms >= 0 && ms < best_ms) {
                best_ms = ms;
                best = p;
            }
        }
    }
    tc_status s = tc_set_params(ctx, &best);
    if (s) return s;
    cache_store(cache_path, sig, best);
    if (best_out) *best_out = best;
    return TC_OK;
}
