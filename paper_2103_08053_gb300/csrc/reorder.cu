// reorder.cu -- tc_reorder: the two vertex reorderings of Sec. 4.1.
//
// Both renumber the vertices so that ids which meet in one hash table are
// consecutive, and consecutive ids fall into distinct buckets under x mod B
// (Sec. 4.1, the max-collision term of Eq. 2). The count never changes.
//
//   TC_REORDER_INDEGREE:   new ids in order of in-degree in N+ (the number of
//                          out-lists holding the vertex), largest first, ties
//                          by smaller old id.
//   TC_REORDER_COLLECTIVE: the vertices u are taken by collective out-degree
//                          sum_{v in N+(u)} d+(v), largest first, ties by
//                          smaller old id; the members of N+(u) that have no
//                          new id yet receive the next ones, in ascending old
//                          id; vertices in no out-list come last, by old id.
//
// The walk of the second heuristic is sequential as stated; here it is
// computed in parallel from an equivalent definition: the walk meets vertex v
// first in list r_min(v) = min{ r : v in N+(order[r]) }, and inside one list
// in ascending id, so v's new id is its rank by the pair (r_min(v), v), with
// r_min = n for a vertex in no list. Ranks come from a stable LSD radix sort
// (8-bit digits) written here; keys of "largest first" orders are stored as
// max - key so that every sort is ascending and ties keep old-id order.
#include <algorithm>

#include "api_internal.h"

using namespace tcg;

namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_ITEMS = 8;                        // keys per thread per tile
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;     // 2048 keys per block
constexpr int XS_THREADS = 256;
constexpr int XS_ITEMS = 16;
constexpr int XS_TILE = XS_THREADS * XS_ITEMS;     // scan tile
constexpr int XS_TOP_THREADS = 1024;

__device__ __forceinline__ unsigned lanemask_lt_r(int lane) { return (1u << lane) - 1u; }

__device__ __forceinline__ long long warp_incl_scan_ll(long long x, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Exclusive scan of one value per thread over the block; *total = block sum.
__device__ long long block_excl_scan_ll(long long v, long long* sh, long long* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const long long inc = warp_incl_scan_ll(v, lane);
    if (lane == 31) sh[w] = inc;
    __syncthreads();
    if (w == 0) {
        const long long x = (lane < nw) ? sh[lane] : 0;
        const long long xi = warp_incl_scan_ll(x, lane);
        if (lane < nw) sh[lane] = xi - x;
        if (lane == 31) sh[32] = xi;
    }
    __syncthreads();
    const long long r = sh[w] + inc - v;
    *total = sh[32];
    __syncthreads();
    return r;
}

// ---- exclusive scan of int32 counts into Out[n+1] (Out[n] = total) ----------

__global__ void __launch_bounds__(XS_THREADS) k_xs_reduce(const int32_t* __restrict__ in, int64_t n,
                                                         long long* __restrict__ partial) {
    __shared__ long long sh[33];
    const int64_t base = (int64_t)blockIdx.x * XS_TILE;
    long long s = 0;
    for (int i = threadIdx.x; i < XS_TILE; i += XS_THREADS) {
        const int64_t k = base + i;
        if (k < n) s += in[k];
    }
    long long tot;
    block_excl_scan_ll(s, sh, &tot);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

template <typename Out>
__global__ void __launch_bounds__(XS_TOP_THREADS) k_xs_top(long long* __restrict__ partial, int nb,
                                                          Out* __restrict__ out, int64_t n) {
    __shared__ long long sh[33];
    const int per = (nb + XS_TOP_THREADS - 1) / XS_TOP_THREADS;
    const int b0 = min(nb, (int)threadIdx.x * per), b1 = min(nb, b0 + per);
    long long s = 0;
    for (int i = b0; i < b1; ++i) s += partial[i];
    long long tot;
    long long pre = block_excl_scan_ll(s, sh, &tot);
    for (int i = b0; i < b1; ++i) {
        const long long x = partial[i];
        partial[i] = pre;
        pre += x;
    }
    if (threadIdx.x == 0) out[n] = (Out)tot;
}

template <typename Out>
__global__ void __launch_bounds__(XS_THREADS) k_xs_down(const int32_t* __restrict__ in, int64_t n,
                                                       const long long* __restrict__ partial, Out* __restrict__ out) {
    __shared__ long long sh[33];
    const int64_t base = (int64_t)blockIdx.x * XS_TILE + (int64_t)threadIdx.x * XS_ITEMS;
    int v[XS_ITEMS];
    long long s = 0;
#pragma unroll
    for (int i = 0; i < XS_ITEMS; ++i) {
        const int64_t k = base + i;
        v[i] = (k < n) ? in[k] : 0;
        s += v[i];
    }
    long long tot;
    long long pre = block_excl_scan_ll(s, sh, &tot) + partial[blockIdx.x];
#pragma unroll
    for (int i = 0; i < XS_ITEMS; ++i) {
        const int64_t k = base + i;
        if (k < n) out[k] = (Out)pre;
        pre += v[i];
    }
}

int xs_blocks(int64_t n) { return (int)std::max<int64_t>(1, (n + XS_TILE - 1) / XS_TILE); }

template <typename Out>
void scan_excl(const int32_t* in, int64_t n, Out* out, long long* partial, cudaStream_t st, long long* nl) {
    const int nb = xs_blocks(n);
    k_xs_reduce<<<nb, XS_THREADS, 0, st>>>(in, n, partial);
    k_xs_top<Out><<<1, XS_TOP_THREADS, 0, st>>>(partial, nb, out, n);
    k_xs_down<Out><<<nb, XS_THREADS, 0, st>>>(in, n, partial, out);
    *nl += 3;
}

// ---- stable LSD radix sort of (uint64 key, int32 value) pairs ---------------

int rs_blocks(int64_t n) { return (int)((n + RS_TILE - 1) / RS_TILE); }

// hist[d * nb + b] = number of keys of tile b whose digit at `shift` is d.
__global__ void __launch_bounds__(RS_THREADS) k_rs_hist(const uint64_t* __restrict__ keys, int64_t n, int shift,
                                                       int nb, int32_t* __restrict__ hist) {
    __shared__ int cnt[256];
    for (int i = threadIdx.x; i < 256; i += RS_THREADS) cnt[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int i = threadIdx.x; i < RS_TILE; i += RS_THREADS) {
        const int64_t k = base + i;
        if (k < n) atomicAdd(&cnt[(int)((keys[k] >> shift) & 255u)], 1);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < 256; d += RS_THREADS) hist[(int64_t)d * nb + blockIdx.x] = cnt[d];
}

// Scatter of tile b: a key goes to offs[d * nb + b] + (keys of digit d before
// it in the tile). Warp w handles the tile's w-th run of RS_ITEMS * 32 keys in
// rounds of 32; inside a round, lanes with equal digits are ranked by lane
// (match_any), so the order within one digit is the input order.
__global__ void __launch_bounds__(RS_THREADS) k_rs_scatter(const uint64_t* __restrict__ kin,
                                                          const int32_t* __restrict__ vin, uint64_t* __restrict__ kout,
                                                          int32_t* __restrict__ vout, int64_t n, int shift, int nb,
                                                          const int32_t* __restrict__ offs) {
    __shared__ int wcnt[RS_WARPS][256];
    for (int i = threadIdx.x; i < RS_WARPS * 256; i += RS_THREADS) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t base = (int64_t)blockIdx.x * RS_TILE + (int64_t)w * (RS_ITEMS * 32);
    uint64_t key[RS_ITEMS];
    int val[RS_ITEMS], rank[RS_ITEMS], dig[RS_ITEMS];
#pragma unroll
    for (int it = 0; it < RS_ITEMS; ++it) {
        const int64_t k = base + it * 32 + lane;
        const bool ok = k < n;
        key[it] = ok ? kin[k] : 0;
        val[it] = ok ? vin[k] : 0;
        const int d = ok ? (int)((key[it] >> shift) & 255u) : 256;  // 256: a group of its own
        dig[it] = d;
        const unsigned peers = __match_any_sync(FULL, d);
        const int before = ok ? wcnt[w][d] : 0;
        __syncwarp();
        if (ok && lane == __ffs(peers) - 1) wcnt[w][d] = before + __popc(peers);
        __syncwarp();
        rank[it] = before + __popc(peers & lanemask_lt_r(lane));
    }
    __syncthreads();
    if (threadIdx.x < 256) {  // per digit: exclusive offsets of the warps' runs
        int s = 0;
#pragma unroll
        for (int j = 0; j < RS_WARPS; ++j) {
            const int c = wcnt[j][threadIdx.x];
            wcnt[j][threadIdx.x] = s;
            s += c;
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < RS_ITEMS; ++it) {
        if (dig[it] == 256) continue;
        const int64_t pos = (int64_t)offs[(int64_t)dig[it] * nb + blockIdx.x] + wcnt[w][dig[it]] + rank[it];
        kout[pos] = key[it];
        vout[pos] = val[it];
    }
}

__global__ void k_iota(int32_t* __restrict__ v, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = (int32_t)i;
}

// ---- keys ---------------------------------------------------------------------

// cnt[v] += 1 for every DAG entry v (in-degree in N+).
__global__ void k_indegree(const int32_t* __restrict__ dag_col, int64_t m, int32_t* __restrict__ cnt) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[dag_col[e]], 1);
}

// key[u] = sum_{v in N+(u)} d+(v), one warp per vertex.
__global__ void k_collective(const int32_t* __restrict__ dag_ptr, const int32_t* __restrict__ dag_col, int64_t n,
                             uint64_t* __restrict__ key) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += warps) {
        unsigned long long s = 0;
        for (int e = dag_ptr[u] + lane; e < dag_ptr[u + 1]; e += 32) {
            const int v = dag_col[e];
            s += (unsigned)(dag_ptr[v + 1] - dag_ptr[v]);
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
        if (lane == 0) key[u] = s;
    }
}

template <typename K>
__global__ void k_keymax(const K* __restrict__ key, int64_t n, unsigned long long* __restrict__ out) {
    unsigned long long mx = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        mx = max(mx, (unsigned long long)key[i]);
#pragma unroll
    for (int o = 16; o; o >>= 1) mx = max(mx, __shfl_xor_sync(FULL, mx, o));
    if ((threadIdx.x & 31) == 0 && mx) atomicMax(out, mx);
}

// Descending order as an ascending key: out[i] = max - key[i].
template <typename K>
__global__ void k_desc_key(const K* __restrict__ key, int64_t n, const unsigned long long* __restrict__ mx,
                           uint64_t* __restrict__ out) {
    const unsigned long long m = *mx;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = m - (unsigned long long)key[i];
}

__global__ void k_fill_u64(uint64_t* __restrict__ v, int64_t n, uint64_t x) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        v[i] = x;
}

// r_min(v) = min rank r of a list N+(order[r]) holding v; one warp per rank.
__global__ void k_first_list(const int32_t* __restrict__ order, const int32_t* __restrict__ dag_ptr,
                             const int32_t* __restrict__ dag_col, int64_t n, unsigned long long* __restrict__ rmin) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < n; r += warps) {
        const int u = order[r];
        for (int e = dag_ptr[u] + lane; e < dag_ptr[u + 1]; e += 32)
            atomicMin(&rmin[dag_col[e]], (unsigned long long)r);
    }
}

__global__ void k_rank_to_id(const int32_t* __restrict__ order, int64_t n, int32_t* __restrict__ new_id) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        new_id[order[r]] = (int32_t)r;
}

// ---- relabelled CSR -------------------------------------------------------------

template <typename Off>
__global__ void k_new_degree(const Off* __restrict__ row_ptr, int64_t n, const int32_t* __restrict__ new_id,
                             int32_t* __restrict__ new_deg) {
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x)
        new_deg[new_id[u]] = (int32_t)(row_ptr[u + 1] - row_ptr[u]);
}

// Row new_id[u] of the output = new_id of row u's entries, same order.
template <typename Off>
__global__ void k_relabel(const Off* __restrict__ row_ptr, const int32_t* __restrict__ col, int64_t n,
                          const int32_t* __restrict__ new_id, const Off* __restrict__ out_ptr,
                          int32_t* __restrict__ out_col) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += warps) {
        const Off a = row_ptr[u], d = row_ptr[u + 1] - a;
        const Off dst = out_ptr[new_id[u]];
        for (Off j = lane; j < d; j += 32) out_col[dst + j] = new_id[col[a + j]];
    }
}

struct ReorderScratch {
    DevBuf keys[2], vals[2], cnt, hist, offs, partial, mx;
    void release(tc_ctx* ctx) {
        for (DevBuf* b : {&keys[0], &keys[1], &vals[0], &vals[1], &cnt, &hist, &offs, &partial, &mx}) b->release(ctx);
    }
};

int grid_for(int64_t work, int threads, int num_sms) {
    const int64_t g = (work + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, (int64_t)num_sms * 16));
}

// Sorts (keys[0], vals[0]) by the low `bits` bits of the keys, stable; the
// sorted pairs end in (keys[sel], vals[sel]), sel returned.
int radix_sort(ReorderScratch& s, int64_t n, int bits, cudaStream_t st, long long* nl) {
    const int nb = rs_blocks(n);
    int sel = 0;
    for (int shift = 0; shift < bits; shift += 8) {
        const uint64_t* ki = (const uint64_t*)s.keys[sel].p;
        const int32_t* vi = (const int32_t*)s.vals[sel].p;
        k_rs_hist<<<nb, RS_THREADS, 0, st>>>(ki, n, shift, nb, (int32_t*)s.hist.p);
        scan_excl<int32_t>((const int32_t*)s.hist.p, (int64_t)nb * 256, (int32_t*)s.offs.p,
                           (long long*)s.partial.p, st, nl);
        k_rs_scatter<<<nb, RS_THREADS, 0, st>>>(ki, vi, (uint64_t*)s.keys[sel ^ 1].p, (int32_t*)s.vals[sel ^ 1].p, n,
                                                shift, nb, (const int32_t*)s.offs.p);
        *nl += 2;
        sel ^= 1;
    }
    return sel;
}

int bit_length(unsigned long long x) { return x ? 64 - __builtin_clzll(x) : 0; }

}  // namespace

extern "C" tc_status tc_reorder(tc_ctx* ctx, const tc_csr* g, int32_t kind, int32_t* new_id, const tc_csr* out,
                                void* stream) {
    if (!ctx) return TC_ERR_INVALID_ARG;
    if (kind != TC_REORDER_INDEGREE && kind != TC_REORDER_COLLECTIVE)
        return ctx_fail(ctx, TC_ERR_INVALID_ARG, "tc_reorder: unknown kind %d", kind);
    tc_status s = check_csr(ctx, g);
    if (s) return s;
    if (g->n > 0 && !new_id) return ctx_fail(ctx, TC_ERR_INVALID_ARG, "tc_reorder: new_id is NULL");
    if (out && (out->n != g->n || out->nnz != g->nnz || out->offset_bits != g->offset_bits ||
                (g->n > 0 && !out->row_ptr) || (g->nnz > 0 && (!out->col || out->col == g->col)) ||
                out->row_ptr == g->row_ptr))
        return ctx_fail(ctx, TC_ERR_INVALID_ARG,
                        "tc_reorder: out must be separate buffers with the input's n, nnz and offset width");
    const int64_t n = g->n;
    if (n == 0) return TC_OK;
    DeviceGuard dg(ctx->device);
    cudaStream_t st = (cudaStream_t)stream;
    int64_t m = 0;
    if ((s = orient_to_workspace(ctx, g, st, &m))) return s;
    const int32_t* dag_ptr = (const int32_t*)ctx->ws.dag_ptr.p;
    const int32_t* dag_col = (const int32_t*)ctx->ws.dag_col.p;

    ReorderScratch sc;
    const int nb = rs_blocks(n);
    const int64_t hist_n = (int64_t)nb * 256;
    for (int i = 0; i < 2 && !s; ++i) {
        s = sc.keys[i].ensure(ctx, (size_t)n * 8, st);
        if (!s) s = sc.vals[i].ensure(ctx, (size_t)n * 4, st);
    }
    if (!s) s = sc.cnt.ensure(ctx, (size_t)n * 4, st);
    if (!s) s = sc.hist.ensure(ctx, (size_t)hist_n * 4, st);
    if (!s) s = sc.offs.ensure(ctx, (size_t)(hist_n + 1) * 4, st);
    if (!s) s = sc.partial.ensure(ctx, (size_t)(xs_blocks(std::max<int64_t>(hist_n, n)) + 1) * 8, st);
    if (!s) s = sc.mx.ensure(ctx, 64, st);
    if (s) {
        sc.release(ctx);
        return s;
    }
    long long nl = 0;
    const int G = grid_for(n, 256, ctx->num_sms);
    const int Gw = grid_for(n * 32, 256, ctx->num_sms);
    unsigned long long* mx = (unsigned long long*)sc.mx.p;
    uint64_t* k0 = (uint64_t*)sc.keys[0].p;
    int32_t* v0 = (int32_t*)sc.vals[0].p;
    cudaError_t e = cudaMemsetAsync(mx, 0, 8, st);
    // 1. the sort key of every vertex, largest first
    if (kind == TC_REORDER_INDEGREE) {
        if (e == cudaSuccess) e = cudaMemsetAsync(sc.cnt.p, 0, (size_t)n * 4, st);
        if (e == cudaSuccess && m > 0) {
            k_indegree<<<grid_for(m, 256, ctx->num_sms), 256, 0, st>>>(dag_col, m, (int32_t*)sc.cnt.p);
            ++nl;
        }
        k_keymax<int32_t><<<G, 256, 0, st>>>((const int32_t*)sc.cnt.p, n, mx);
        k_desc_key<int32_t><<<G, 256, 0, st>>>((const int32_t*)sc.cnt.p, n, mx, k0);
    } else {
        k_collective<<<Gw, 256, 0, st>>>(dag_ptr, dag_col, n, (uint64_t*)sc.keys[1].p);
        k_keymax<uint64_t><<<G, 256, 0, st>>>((const uint64_t*)sc.keys[1].p, n, mx);
        k_desc_key<uint64_t><<<G, 256, 0, st>>>((const uint64_t*)sc.keys[1].p, n, mx, k0);
        ++nl;
    }
    k_iota<<<G, 256, 0, st>>>(v0, n);
    nl += 3;
    unsigned long long maxkey = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&maxkey, mx, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        ctx->launches += nl;
        sc.release(ctx);
        return cuda_status(ctx, e, "tc_reorder keys");
    }
    // 2. the order of the vertices
    int sel = radix_sort(sc, n, bit_length(maxkey), st, &nl);
    if (kind == TC_REORDER_COLLECTIVE) {
        // 3. r_min(v), then the rank by (r_min, id)
        const int32_t* order = (const int32_t*)sc.vals[sel].p;
        uint64_t* rmin = (uint64_t*)sc.keys[sel ^ 1].p;
        k_fill_u64<<<G, 256, 0, st>>>(rmin, n, (uint64_t)n);
        k_first_list<<<Gw, 256, 0, st>>>(order, dag_ptr, dag_col, n, (unsigned long long*)rmin);
        if (sel == 0) {  // the r_min keys must sit in buffer 0 for the sort
            e = cudaMemcpyAsync(sc.keys[0].p, rmin, (size_t)n * 8, cudaMemcpyDeviceToDevice, st);
        }
        k_iota<<<G, 256, 0, st>>>(v0, n);
        nl += 3;
        sel = radix_sort(sc, n, bit_length((unsigned long long)n), st, &nl);
    }
    k_rank_to_id<<<G, 256, 0, st>>>((const int32_t*)sc.vals[sel].p, n, new_id);
    ++nl;
    // 4. the relabelled CSR
    if (out && e == cudaSuccess) {
        int32_t* new_deg = (int32_t*)sc.cnt.p;
        if (g->offset_bits == 64) {
            k_new_degree<int64_t><<<G, 256, 0, st>>>((const int64_t*)g->row_ptr, n, new_id, new_deg);
            scan_excl<int64_t>(new_deg, n, (int64_t*)out->row_ptr, (long long*)sc.partial.p, st, &nl);
            k_relabel<int64_t><<<Gw, 256, 0, st>>>((const int64_t*)g->row_ptr, g->col, n, new_id,
                                                  (const int64_t*)out->row_ptr, (int32_t*)out->col);
        } else {
            k_new_degree<int32_t><<<G, 256, 0, st>>>((const int32_t*)g->row_ptr, n, new_id, new_deg);
            scan_excl<int32_t>(new_deg, n, (int32_t*)out->row_ptr, (long long*)sc.partial.p, st, &nl);
            k_relabel<int32_t><<<Gw, 256, 0, st>>>((const int32_t*)g->row_ptr, g->col, n, new_id,
                                                  (const int32_t*)out->row_ptr, (int32_t*)out->col);
        }
        nl += 2;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    ctx->launches += nl;
    sc.release(ctx);
    return cuda_status(ctx, e, "tc_reorder kernels");
}
