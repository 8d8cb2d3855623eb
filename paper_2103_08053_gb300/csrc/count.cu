// count.cu -- vertex-centric hashed triangle counting on the oriented graph.
//
// TRUST Algorithm 1, run on N+ (Sec. 2.2 orientation; Sec. 3): for every
// vertex u, build a hash table of N+(u) once, then for every v in N+(u) add
// |table ∩ N+(v)|. The pieces, and where they come from:
//   * bucketed table, fixed-size buckets in one contiguous region, slot given
//     by an atomic increment of the bucket's length (Algorithm 1,
//     hashTableConstruction; Sec. 3.1);
//   * hash(x) = x mod B with B a power of two (Algorithm 1, hash);
//   * level-major ("interleaved") layout: element j of bucket i at j*B + i,
//     with the lengths in shared memory (Sec. 3.2). Here the whole table is in
//     shared memory: B and the level count L are sized from d+(u) so that
//     B*L > d+(u) always holds (see below), so no global spill region exists;
//   * a bucket holding L elements is full; further keys go to the next bucket
//     and a search continues through successor buckets while the bucket it
//     scanned was full (Sec. 3.2, last paragraph: linear probing on overflow);
//   * linear search inside a bucket (Algorithm 1, linearSearch);
//   * virtual combination (Sec. 4.2): the 2-hop lists N+(v) of 32 consecutive
//     out-neighbours are treated as one flat array whose indices are dealt to
//     the 32 lanes; a lane finds the owning list of its index from the
//     inclusive prefix of the list lengths;
//   * degree-aware workers (Sec. 4.3): 2 <= d+ <= T_w -> one warp with a
//     warp-private table; d+ > T_w -> one thread block with a block-wide table,
//     its out-list split into work items of item_neighbors neighbours; both
//     pull work from atomic queues in chunks (Sec. 4.3, dynamic assignment);
//   * hits are summed per lane, reduced per warp and block, and added to one
//     uint64 total (Algorithm 1, count +=).
//
// Sizing (GB300: up to 227 KiB of shared memory per block). Warp tables:
// B = clamp(nextpow2(d+), 32, Bmax), L = min(Lmax, table_ints / B); the host
// checks that B*L > T_w. Block tables: B = nextpow2(part), L = min(Lmax,
// budget/B - 1) >= 2, where N+(u) is split into parts of at most P_max
// (largest power of two with 3*P_max <= budget) and every part is probed by
// the whole 2-hop list: |N+(u) ∩ N+(v)| = sum over parts of |part ∩ N+(v)|.
#include "tc_internal.h"

namespace tcg {

namespace {

__device__ __forceinline__ unsigned lanemask_le(int lane) { return (2u << lane) - 1u; }
__device__ __forceinline__ unsigned lanemask_lt(int lane) { return (1u << lane) - 1u; }

// Algorithm 1 hashTableConstruction, one key: slot = atomicAdd(len[h], 1);
// full bucket -> next bucket. len may grow past L (a failed claim also
// increments it); "len >= L" means full.
__device__ __forceinline__ void table_insert(int* len, int* tab, int B, int L, int w) {
    int h = w & (B - 1);
    for (int s = 0; s < B; ++s) {
        const int slot = atomicAdd(&len[h], 1);
        if (slot < L) {
            tab[slot * B + h] = w;
            return;
        }
        h = (h + 1) & (B - 1);
    }
}

// Algorithm 1 linearSearch over the bucket of w and, while the scanned bucket
// was full, its successors.
__device__ __forceinline__ int table_probe(const int* len, const int* tab, int B, int L, int w) {
    int h = w & (B - 1);
    for (int s = 0; s < B; ++s) {
        const int ln = len[h];
        const int c = ln < L ? ln : L;
        for (int j = 0; j < c; ++j)
            if (tab[j * B + h] == w) return 1;
        if (ln < L) return 0;
        h = (h + 1) & (B - 1);
    }
    return 0;
}

// Virtual combination over the 2-hop lists of up to 32 out-neighbours
// nbrs[0..cnt): lane j loads neighbour j and its list bounds; the non-empty
// lists are compacted to lanes 0..c-1 and scanned; then the flat index range
// [0, total) is dealt to the lanes 32 at a time. For a window starting at
// `base`, the owner of lane L's index is
//   j0 + popc(starts & lanemask_le(L)) - (bit 0 of starts)
// where j0 = number of lists ending at or before base and `starts` has bit x
// set iff a list starts at base + x (one REDUX.OR). stage: 64 ints of smem.
__device__ __forceinline__ uint32_t warp_probe_chunk(const int32_t* __restrict__ nbrs, int cnt,
                                                     const int32_t* __restrict__ dag_ptr,
                                                     const int32_t* __restrict__ dag_col, const int* len,
                                                     const int* tab, int B, int L, int lane, int* stage,
                                                     int n, DevCounters* ctr) {
    int s = 0, l = 0;
    if (lane < cnt) {
        const int v = nbrs[lane];
        if ((unsigned)v < (unsigned)n) {
            s = dag_ptr[v];
            l = dag_ptr[v + 1] - s;
        } else {
            atomicOr(&ctr->err, ERRBIT_BAD_GRAPH);
        }
    }
    const unsigned nem = __ballot_sync(FULL, l > 0);
    if (nem == 0) return 0;
    const int c = __popc(nem);
    if (l > 0) {
        const int p = __popc(nem & lanemask_lt(lane));
        stage[p] = s;
        stage[32 + p] = l;
    }
    __syncwarp();
    const int cs = (lane < c) ? stage[lane] : 0;
    const int cl = (lane < c) ? stage[32 + lane] : 0;
    __syncwarp();
    int P = cl;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(FULL, P, o);
        if (lane >= o) P += t;
    }
    const int total = __shfl_sync(FULL, P, 31);
    const int Pex = P - cl;
    const unsigned le = lanemask_le(lane);
    uint32_t hits = 0;
    for (int base = 0; base < total; base += 32) {
        const int j0 = __popc(__ballot_sync(FULL, lane < c && P <= base));
        const int x = Pex - base;
        const unsigned bit = (lane < c && x >= 0 && x < 32) ? (1u << x) : 0u;
        const unsigned starts = __reduce_or_sync(FULL, bit);
        const int o = j0 + __popc(starts & le) - (int)(starts & 1u);
        const int so = __shfl_sync(FULL, cs, o & 31);
        const int po = __shfl_sync(FULL, Pex, o & 31);
        const int f = base + lane;
        if (f < total) hits += table_probe(len, tab, B, L, dag_col[so + (f - po)]);
    }
    return hits;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

__device__ __forceinline__ void block_add_total(unsigned long long acc, DevCounters* ctr) {
    __shared__ unsigned long long s_red[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    acc = warp_sum_u64(acc);
    if (lane == 0) s_red[w] = acc;
    __syncthreads();
    if (w == 0) {
        unsigned long long x = (lane < (int)(blockDim.x >> 5)) ? s_red[lane] : 0ull;
        x = warp_sum_u64(x);
        if (lane == 0 && x) atomicAdd(&ctr->total, x);
    }
}

// Warp workers: one warp per vertex with 2 <= d+ <= T_w, warp-private table.
// smem per warp: len[Bmax] | tab[table_ints] | stage[64].
__global__ void __launch_bounds__(256)
    k_count_warp(const int32_t* __restrict__ dag_ptr, const int32_t* __restrict__ dag_col,
                 const int32_t* __restrict__ warp_list, unsigned long long* __restrict__ per_vertex,
                 DevCounters* ctr, int n, int table_ints, int max_buckets, int max_levels, int chunk) {
    extern __shared__ int smem[];
    if (ctr->err) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int* len = smem + w * (max_buckets + table_ints + 64);
    int* tab = len + max_buckets;
    int* stage = tab + table_ints;
    const int nlist = ctr->n_warp;
    unsigned long long acc = 0;
    for (;;) {
        int i0 = 0;
        if (lane == 0) i0 = atomicAdd(&ctr->q_warp, chunk);
        i0 = __shfl_sync(FULL, i0, 0);
        if (i0 >= nlist) break;
        const int i1 = min(i0 + chunk, nlist);
        for (int i = i0; i < i1; ++i) {
            const int u = warp_list[i];
            const int a = dag_ptr[u];
            const int k = dag_ptr[u + 1] - a;
            int B = next_pow2(k);
            B = B < 32 ? 32 : (B > max_buckets ? max_buckets : B);
            int L = table_ints / B;
            L = L < max_levels ? L : max_levels;
            for (int t = lane; t < B; t += 32) len[t] = 0;
            __syncwarp();
            for (int t = lane; t < k; t += 32) table_insert(len, tab, B, L, dag_col[a + t]);
            __syncwarp();
            uint32_t h = 0;
            for (int c0 = 0; c0 < k; c0 += 32)
                h += warp_probe_chunk(dag_col + a + c0, min(32, k - c0), dag_ptr, dag_col, len, tab, B, L, lane,
                                      stage, n, ctr);
            acc += h;
            if (per_vertex) {
                const unsigned long long hu = warp_sum_u64(h);
                if (lane == 0) per_vertex[u] = hu;
            }
            __syncwarp();
        }
    }
    block_add_total(acc, ctr);
}

// Thread-block workers: one block per work item (u, first neighbour) of a
// vertex with d+ > T_w. smem: stage[nwarps*64] | len[B] | tab[B*L].
__global__ void __launch_bounds__(1024)
    k_count_block(const int32_t* __restrict__ dag_ptr, const int32_t* __restrict__ dag_col,
                  const int2* __restrict__ items, unsigned long long* __restrict__ per_vertex, DevCounters* ctr,
                  int n, int budget_ints, int part_max, int max_levels, int item_nbrs) {
    extern __shared__ int smem[];
    __shared__ int s_item, s_next;
    if (ctr->err) return;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int* stage = smem + w * 64;
    int* len = smem + nw * 64;
    const int nitems = ctr->n_items;
    unsigned long long acc = 0;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(&ctr->q_items, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= nitems) break;
        const int2 item = items[it];
        const int u = item.x;
        const int a = dag_ptr[u];
        const int k = dag_ptr[u + 1] - a;
        const int nb0 = item.y, nb1 = min(k, nb0 + item_nbrs);
        uint32_t h = 0;
        for (int p0 = 0; p0 < k; p0 += part_max) {
            const int pk = min(part_max, k - p0);
            const int B = next_pow2(pk < 32 ? 32 : pk);
            int L = budget_ints / B - 1;
            L = L < max_levels ? L : max_levels;
            int* tab = len + B;
            for (int t = threadIdx.x; t < B; t += blockDim.x) len[t] = 0;
            if (threadIdx.x == 0) s_next = nb0;
            __syncthreads();
            for (int t = threadIdx.x; t < pk; t += blockDim.x) table_insert(len, tab, B, L, dag_col[a + p0 + t]);
            __syncthreads();
            for (;;) {
                int c0 = 0;
                if (lane == 0) c0 = atomicAdd(&s_next, 32);
                c0 = __shfl_sync(FULL, c0, 0);
                if (c0 >= nb1) break;
                h += warp_probe_chunk(dag_col + a + c0, min(32, nb1 - c0), dag_ptr, dag_col, len, tab, B, L, lane,
                                      stage, n, ctr);
            }
            __syncthreads();
        }
        acc += h;
        if (per_vertex) {
            const unsigned long long hu = warp_sum_u64(h);
            if (lane == 0 && hu) atomicAdd(&per_vertex[u], hu);
        }
    }
    block_add_total(acc, ctr);
}

__global__ void k_finish(const DevCounters* ctr, unsigned long long* count_out, int* err_out) {
    if (count_out) *count_out = ctr->total;
    if (err_out) {
        const int b = ctr->err;
        *err_out = b == 0 ? (int)TC_OK : (b & ERRBIT_DAG_TOO_BIG) ? (int)TC_ERR_UNSUPPORTED : (int)TC_ERR_BAD_GRAPH;
    }
}

__global__ void k_stats(const int32_t* __restrict__ dag_ptr, const int32_t* __restrict__ dag_col, int64_t n,
                        int warp_max, DevStats* out) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
        const int64_t u = base + threadIdx.x;
        unsigned long long wp = 0, wpb = 0;
        long long d = 0, skip = 0, nw = 0, nb = 0;
        if (u < n) {
            const int a = dag_ptr[u], b = dag_ptr[u + 1];
            d = b - a;
            for (int i = a; i < b; ++i) {
                const int v = dag_col[i];
                wp += (unsigned long long)(dag_ptr[v + 1] - dag_ptr[v]);
            }
            if (d < 2) skip = 1;
            else if (d <= warp_max) nw = 1;
            else { nb = 1; wpb = wp; }
        }
        wp = warp_sum_u64(wp);
        wpb = warp_sum_u64(wpb);
        skip = (long long)warp_sum_u64((unsigned long long)skip);
        nw = (long long)warp_sum_u64((unsigned long long)nw);
        nb = (long long)warp_sum_u64((unsigned long long)nb);
        long long dm = d;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const long long t = __shfl_xor_sync(FULL, dm, o);
            dm = t > dm ? t : dm;
        }
        if (lane == 0) {
            atomicAdd(&out->wplus, wp);
            atomicAdd(&out->wplus_block, wpb);
            atomicAdd((unsigned long long*)&out->n_skip, (unsigned long long)skip);
            atomicAdd((unsigned long long*)&out->n_warp, (unsigned long long)nw);
            atomicAdd((unsigned long long*)&out->n_block, (unsigned long long)nb);
            atomicMax(&out->max_out, dm);
        }
    }
}

}  // namespace

cudaError_t count_kernel_setup(CountCfg& cfg, int num_sms) {
    const int warp_smem = cfg.warps_per_block * (cfg.warp_max_buckets + cfg.warp_table_ints + 64) * 4;
    cudaError_t e = cudaFuncSetAttribute(k_count_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, warp_smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_count_block, cudaFuncAttributeMaxDynamicSharedMemorySize, cfg.block_smem_bytes);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_count_warp, cfg.warps_per_block * 32, warp_smem);
    if (e != cudaSuccess) return e;
    cfg.warp_grid = num_sms * (per_sm > 0 ? per_sm : 1);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_count_block, cfg.block_threads, cfg.block_smem_bytes);
    if (e != cudaSuccess) return e;
    cfg.block_grid = num_sms * (per_sm > 0 ? per_sm : 1);
    return cudaSuccess;
}

cudaError_t launch_count(const int32_t* dag_ptr, const int32_t* dag_col, int64_t n, const int32_t* warp_list,
                         const int2* items, unsigned long long* per_vertex, const CountCfg& cfg, DevCounters* ctr,
                         cudaStream_t st) {
    const int nwb = cfg.block_threads / 32;
    const int budget = cfg.block_smem_bytes / 4 - nwb * 64;
    int part_max = 1;
    while (part_max * 2 * 3 <= budget) part_max *= 2;
    k_count_block<<<cfg.block_grid, cfg.block_threads, cfg.block_smem_bytes, st>>>(
        dag_ptr, dag_col, items, per_vertex, ctr, (int)n, budget, part_max, cfg.max_levels, cfg.item_neighbors);
    const int warp_smem = cfg.warps_per_block * (cfg.warp_max_buckets + cfg.warp_table_ints + 64) * 4;
    k_count_warp<<<cfg.warp_grid, cfg.warps_per_block * 32, warp_smem, st>>>(
        dag_ptr, dag_col, warp_list, per_vertex, ctr, (int)n, cfg.warp_table_ints, cfg.warp_max_buckets,
        cfg.max_levels, cfg.chunk);
    return cudaGetLastError();
}

cudaError_t launch_finish(const DevCounters* ctr, unsigned long long* count_out, int* err_out, cudaStream_t st) {
    k_finish<<<1, 1, 0, st>>>(ctr, count_out, err_out);
    return cudaGetLastError();
}

cudaError_t launch_stats(const int32_t* dag_ptr, const int32_t* dag_col, int64_t n, int warp_max_out_degree,
                         DevStats* out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int g = (int)((n + 255) / 256);
    if (g > 4096) g = 4096;
    k_stats<<<g, 256, 0, st>>>(dag_ptr, dag_col, n, warp_max_out_degree, out);
    return cudaGetLastError();
}

}  // namespace tcg
