// tc_internal.h -- shared declarations of the CUDA library (not installed).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "tc.h"

// Slots per bucket of the warp workers' (pack) tables: 2 (8-byte buckets) or 4.
#ifndef PACK_SLOTS
#define PACK_SLOTS 2
#endif

namespace tcg {

constexpr unsigned FULL = 0xffffffffu;

// Error bits the kernels raise in DevCounters::err (host maps them to tc_status).
enum : int {
    ERRBIT_BAD_GRAPH = 1,    // column id out of range, row_ptr not monotone / out of [0, nnz]
    ERRBIT_DAG_TOO_BIG = 2,  // m >= 2^31 (int32 DAG offsets)
    ERRBIT_DAG_OVERFLOW = 4, // more kept edges than the DAG buffer holds (asymmetric input)
};

// Device-resident scalars of one counting pass. Zeroed (cudaMemsetAsync)
// before each pass.
struct DevCounters {
    unsigned long long total;  // triangle count
    long long m;               // DAG edges (scan total)
    unsigned long long cyc_build, cyc_probe;  // worker cycles in table builds / probes (cycle timing only)
    int n_warp;                // vertices in the warp-worker list
    int n_items;               // work items of thread-block workers
    int n_block;               // vertices with d+ > warp threshold
    int q_warp;                // queue cursors (atomic chunk pops, Sec. 4.3)
    int q_items;
    int err;                   // ERRBIT_* flags
    int n_hub;                 // rows with degree > HUB_DEGREE (orientation by thread blocks)
    int q_hub[2];              // hub-row cursors of the two orientation passes
    int n_mid;                 // rows with MID_DEGREE < degree <= HUB_DEGREE (orientation by warps)
    int q_mid[2];
    int pad[11];
};
static_assert(sizeof(DevCounters) == 128, "DevCounters layout");

// Resolved launch parameters (host fills from tc_params + device properties).
struct CountCfg {
    int warp_max_out_degree;   // T_w
    int warp_area_ints;        // per-warp table area
    int warp_min_buckets;      // power of two
    int warps_per_block;       // warp kernel
    int warp_grid;             // persistent grid of the warp kernel
    int block_threads;         // block kernel
    int block_smem_bytes;
    int block_grid;
    int item_neighbors;
    int chunk;
    int shard_count, shard_index;
    int record_timing;
    int hash_mode;  // 0 multiplicative, 1 x mod B
    int quad_loads; // 1: warp workers read 2-hop lists as 16-byte quads (when dag_col is 16-byte aligned)
    int cycle_timing;  // 1: counting kernels add their build / probe cycles to DevCounters
    int edge_centric;  // 1: Algorithm 2 ablation (table of N+(u) rebuilt for every out-edge)
    int balance;       // TC_BALANCE_*: how warp workers spread 2-hop lists over lanes (Sec. 4.2)
    int warp_order;    // 0 auto, 1 warp list grouped by locality key, 2 vertex order
    int pop_contiguous = 0;  // 1: warp workers pop consecutive warp-list entries (batches)
};

// One graph of an orientation pass. A batch places its graphs in one padded
// global vertex space: graph i owns global rows [vbase, vbase + n), vbase a
// multiple of 32 and ascending; rows in the padding have no edges.
struct GraphRef {
    const void* row_ptr;  // int32 or int64 offsets (one width per pass)
    const int32_t* col;
    long long n, nnz, vbase;
    long long ebase;      // row-local DAG: offset of this graph's entries in the shared array
};

// ---- orientation (orient.cu) ----------------------------------------------
// Rows longer than this are oriented by one thread block each instead of
// inside a 32-row warp group.
constexpr int HUB_DEGREE = 1024;
// Rows longer than this (and not hubs) are oriented by one warp each.
constexpr int MID_DEGREE = 128;
// deg, kept: int32[n]; partial: int64[scan_blocks(n)+1]; dag_ptr: int32[n+1];
// warp_list: int32[n]; warp_desc: int2[n]; items: int2[item_cap].
int scan_blocks(int64_t n);
// hubs: int32[n] scratch: rows with degree > HUB_DEGREE from the front, rows
// with MID_DEGREE < degree <= HUB_DEGREE from the back.
// kbits: NULL, or keep_bits_words(nnz) words of scratch: the count pass
// records each entry's keep decision there and the compaction pass reads it
// instead of gathering the neighbours' degrees a second time.
inline int64_t keep_bits_words(int64_t nnz) { return (nnz >> 5) + 2; }
// Row-local mode (bnd and rdag given, nnz < 2^31): the DAG is left where the
// CSR has it -- N+(u) = rdag[bnd[u].x, bnd[u].x + bnd[u].y), bnd[u] = (row_ptr[u],
// d+(u)), bnd[n].x = nnz, rdag of nnz entries -- by the count pass alone (no
// scan, no compaction), and ctr->m receives the number of kept entries;
// kept, dag_ptr, dag_col and kbits are then unused.
cudaError_t launch_orient(const void* row_ptr, int offset_bits, const int32_t* col, int64_t n, int64_t nnz,
                          int32_t* deg, int32_t* kept, long long* partial, int32_t* dag_ptr, int32_t* dag_col,
                          int64_t dag_cap, int32_t* hubs, unsigned* kbits, DevCounters* ctr, int num_sms,
                          cudaStream_t st, long long* launches, int2* bnd = nullptr, int32_t* rdag = nullptr);

// Row-local orientation of one graph whose col arrives on the device in
// pieces: the degree kernel, then the count pass over the 32-row groups
// [group_cuts[i], group_cuts[i+1]) once event ready[i] has completed (the
// copy of those rows' lists), then the hub / mid rows (after every piece).
cudaError_t launch_orient_row_local_pieces(const void* row_ptr, int offset_bits, const int32_t* col, int64_t n,
                                           int64_t nnz, int32_t* deg, int32_t* kept, int32_t* hubs, int2* bnd,
                                           int32_t* rdag, DevCounters* ctr, int num_sms, cudaStream_t st,
                                           long long* launches, const int64_t* group_cuts, int pieces,
                                           const cudaEvent_t* ready);

// Orientation of k graphs at once (device array of GraphRef, bases ascending)
// into one DAG over the padded global vertex space [0, total).
cudaError_t launch_orient_batch(const GraphRef* graphs, int k, int offset_bits, int64_t total, int32_t* deg,
                                int32_t* kept, long long* partial, int32_t* dag_ptr, int32_t* dag_col,
                                int64_t dag_cap, int32_t* hubs, DevCounters* ctr, int num_sms, cudaStream_t st,
                                long long* launches,
                                int2* bnd = nullptr, int32_t* rdag = nullptr, long long entries = 0);

// Binning (Sec. 4.3) from an existing DAG: fills warp_list / items / counters.
// ncol (one graph only: the input CSR's neighbour ids for a row-local DAG, the
// DAG's own dag_col for a compact one; okey, ohist: n ints, partial:
// scan_blocks(n) + 2 long longs): the warp list is laid out in the order of a
// locality key, min(u, first entry of u's row) -- a histogram of the keys,
// its scan, and a placement pass -- instead of in vertex order.
// Ordered work items (with the ordered warp list; dcol: the DAG's entries,
// ikey: item_cap ints, items2: item_cap int2 of scratch): the thread-block
// work items are laid out in the order of their first out-neighbour's id --
// rows sorted by id give an item a contiguous id range of out-neighbours, so
// items that run at the same time read overlapping 2-hop lists.
cudaError_t launch_bin(const int32_t* dag_ptr, int64_t n, const CountCfg& cfg, int32_t* warp_list, int2* warp_desc,
                       int2* items, int64_t item_cap, DevCounters* ctr, int num_sms, cudaStream_t st,
                       long long* launches,
                       const int2* dag_bnd = nullptr, long long max_m = -1, const int32_t* ncol = nullptr,
                       int32_t* okey = nullptr, int32_t* ohist = nullptr, long long* partial = nullptr,
                       const int32_t* dcol = nullptr, int32_t* ikey = nullptr, int2* items2 = nullptr);

#ifndef BLOCK_ITEM_ORDER
#define BLOCK_ITEM_ORDER 1  // 1: thread-block work items ordered by their first out-neighbour (ordered mode)
#endif

// ---- counting (count.cu) ----------------------------------------------------
cudaError_t launch_count(const int32_t* dag_ptr, const int32_t* dag_col, int64_t n, const int32_t* warp_list,
                         const int2* warp_desc, const int2* items, unsigned long long* per_vertex,
                         const CountCfg& cfg, DevCounters* ctr, cudaStream_t st, long long* launches,
                         const int2* dag_bnd = nullptr, int2* pc_scratch = nullptr);
// device bytes of the physical-combination scratch (cfg.balance == TC_BALANCE_PC): one
// round of combined (key, table) pairs per warp of the warp-worker grid
size_t pc_scratch_bytes(const CountCfg& cfg);
int count_block_budget_ints(const CountCfg& cfg);
int count_block_part_max(const CountCfg& cfg);
// ints of one warp-worker table for out-degree d (8*nextpow2(d) slots in PACK_SLOTS-slot buckets + byte lengths)
int pack_table_ints(int max_out_degree, int min_buckets);
// Resolves cfg's persistent grid sizes and makes sure the counting kernels
// may be launched with cfg's dynamic shared memory. The kernels' limits are
// process-wide per device and shared by every context (and by the
// allocation-free entry point): they are only ever raised, never lowered, so
// a context with smaller tables cannot break one with larger tables.
cudaError_t count_kernel_setup(CountCfg& cfg, int num_sms);
cudaError_t launch_finish(const DevCounters* ctr, unsigned long long* count_out, int* err_out, cudaStream_t st,
                          long long* launches);

// stats: W+ (total and block part), max d+
struct DevStats {
    unsigned long long wplus, wplus_block;
    long long max_out;
    long long n_skip, n_warp, n_block;
    long long maxc[2];           // max collision, B = 32: [0] x mod 32, [1] multiplicative
    unsigned long long phi[2];   // Eq. 2 cost with the same tables
};
cudaError_t launch_stats(const int32_t* dag_ptr, const int32_t* dag_col, int64_t n, int warp_max_out_degree,
                         DevStats* out, cudaStream_t st);

// Default tc_params.item_neighbors (out-neighbours of a large vertex per
// thread-block work item).
constexpr int DEFAULT_ITEM_NEIGHBORS = 256;

// Upper bound on work items produced by binning (one per large vertex plus
// one per item_neighbors of its out-list).
constexpr int64_t item_capacity(int64_t n, int64_t m, int item_neighbors) {
    return n + m / (item_neighbors > 0 ? item_neighbors : 1) + 1;
}

__host__ __device__ inline int next_pow2(int x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

}  // namespace tcg
