/*
 * tc.h -- exact triangle counting on one GB300 GPU (sm_103a), after TRUST
 * (Pandey, Wang et al., "TRUST: Triangle Counting Reloaded on GPUs").
 *
 * The library counts the triangles (three-vertex cliques, Sec. 1) of a
 * simple undirected graph given as a symmetric CSR (Sec. 2.1: "begin
 * position" = row_ptr, "adjacency list" = col). The hot path is the paper's
 * vertex-centric hashing method (Sec. 3, Algorithm 1):
 *   1. rank-by-degree orientation (Sec. 2.2) turns the undirected CSR into a
 *      DAG N+ in which every edge points from the lower to the higher
 *      (degree, id) pair, so every triangle is seen exactly once;
 *   2. vertices are binned by out-degree d+ (Sec. 4.3): d+ < 2 is skipped,
 *      small vertices go to warp workers, large ones to thread-block workers;
 *   3. for every vertex u a bucketed hash table of N+(u) is built once in
 *      shared memory (Algorithm 1 hashTableConstruction, Sec. 3.1-3.2:
 *      fixed-size buckets, atomic slot counters, overflow to the next bucket;
 *      each bucket is stored whole, bucket-major, so that one vector load
 *      fetches it, where the paper interleaves buckets level by level), then
 *      probed with N+(v) for every v in N+(u)
 *      (Algorithm 1 intersection / linearSearch), with the 2-hop lists of all
 *      v spread evenly over the lanes by virtual combination (Sec. 4.2);
 *   4. hits are summed into one 64-bit count.
 * Everything runs in the library's own CUDA kernels; there is no CPU path.
 *
 * Conventions for every entry point:
 *   - Every call returns a tc_status; none aborts, prints or throws. On any
 *     status other than TC_OK the output arguments are left untouched and
 *     tc_last_error(ctx) describes the failure.
 *   - "device" pointers are CUDA device (or managed) memory of the context's
 *     device; "host" pointers are ordinary (pageable or pinned) host memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *     stream). Device inputs must stay valid and unmodified until the call
 *     returns (blocking calls) or until the stream reaches the call's work
 *     (the *_async calls).
 *   - A context is not thread-safe, except tc_submit / tc_submit_borrowed /
 *     tc_poll / tc_drain, which may be called from any thread at any time.
 *
 * Input preconditions (not all checked): the CSR is symmetric (v in N(u) iff
 * u in N(v)) with no duplicate entries in a row; rows need not be sorted;
 * self-loops are allowed and ignored (the strict order drops u -> u). Always
 * detected and reported as TC_ERR_BAD_GRAPH, without faulting: column ids
 * outside [0, n), row_ptr not non-decreasing within [0, nnz], and more kept
 * edges than nnz/2 (an asymmetric CSR).
 */
#ifndef TRUST_GB300_TC_H
#define TRUST_GB300_TC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TC_OK = 0,
    TC_ERR_INVALID_ARG = 1, /* NULL pointer, negative size, bad enum value */
    TC_ERR_BAD_GRAPH = 2,   /* malformed CSR detected (column out of range, ...) */
    TC_ERR_OOM = 3,         /* device allocation failed or memory budget exceeded */
    TC_ERR_BUSY = 4,        /* serving queue full / request exceeds the budget */
    TC_ERR_NOT_READY = 5,   /* tc_poll: the request has not finished yet */
    TC_ERR_TIMEOUT = 6,     /* a bounded device-side wait gave up */
    TC_ERR_CUDA = 7,        /* a CUDA runtime call failed (see tc_last_error) */
    TC_ERR_UNSUPPORTED = 8  /* valid input outside the supported range */
} tc_status;

typedef struct tc_ctx tc_ctx;

/* A simple undirected graph as a symmetric CSR (Sec. 2.1).
 * row_ptr: n+1 offsets, int32 when offset_bits == 32, int64 when 64;
 *          row_ptr[0] == 0, non-decreasing, row_ptr[n] == nnz.
 * col:     nnz int32 neighbour ids; N(u) = col[row_ptr[u] .. row_ptr[u+1]).
 * Each undirected edge {u,v} appears twice (in N(u) and in N(v)), so nnz is
 * 2|E|. Whether the pointers are host or device memory depends on the call. */
typedef struct {
    int64_t n;
    int64_t nnz;
    const void* row_ptr;
    int32_t offset_bits;
    const int32_t* col;
} tc_csr;

/* The oriented graph N+ (Sec. 2.2 rank-by-degree; Sec. 4.3 "after
 * orientation"): dag_ptr int32[n+1], dag_col int32[m], device memory. m is the
 * number of undirected edges (each kept once); m must be < 2^31. A tc_dag
 * filled by tc_orient is owned by the context and released by tc_dag_free;
 * a caller may also fill one with its own device buffers for tc_count_dag. */
typedef struct {
    int64_t n;
    int64_t m;
    int32_t* dag_ptr;
    int32_t* dag_col;
} tc_dag;

/* Tunables. Zero in any field means "use the default" (tc_default_params).
 * The paper's constants are noted beside each (Sec. 3.1, 3.2, 4.3). Table
 * buckets are small and fixed-size (the paper allows up to 128 keys per bucket,
 * 6 levels of them cached in shared memory): a warp worker's table has buckets
 * of 2 keys (one 8-byte load per probe), a thread-block worker's table buckets
 * of 4 keys (one 16-byte load). A key whose bucket is full goes to the next
 * bucket. A thread-block table in which every key sits in its home bucket
 * also keeps a 32-bit key signature per bucket; a probe reads the signature
 * word and loads the bucket only when the key's signature bit is set. */
typedef struct {
    int32_t warp_max_out_degree; /* d+ above this -> thread-block worker, <= 255 (paper: 100; default 128) */
    int32_t warp_area_ints;      /* shared-memory table area of one warp worker, ints (default 1152);
                                    a warp-worker table has 8*nextpow2(d+) slots in buckets of 2,
                                    plus one length byte per bucket */
    int32_t warp_min_buckets;    /* a warp-worker table has at least 4*warp_min_buckets slots; power of
                                    two >= 16 (default 16) */
    int32_t block_threads;       /* threads of a thread-block worker (default 256) */
    int32_t block_smem_bytes;    /* shared memory of a thread-block worker (default 50 KiB) */
    int32_t item_neighbors;      /* out-neighbours of a large vertex per work item, <= block_threads (default 256) */
    int32_t chunk;               /* most vertices a warp takes per queue pop, 1..32 (Sec. 4.3; paper: 1..7;
                                    default 32; fewer on short lists, see k_count_pack) */
    int32_t warps_per_block;     /* warps per block of the warp-worker kernel (default 8) */
    int32_t shard_count;         /* workload partition (Sec. 5.1): count only u with */
    int32_t shard_index;         /*   u % shard_count == shard_index (default 1 / 0) */
    int32_t validate;            /* reserved for extra input checks (0) */
    int32_t record_timing;       /* 1: record CUDA events around the kernel phases (tc_read_timing);
                                    2: also count the workers' cycles in table builds and in probes
                                    (blocking calls: tc_count, tc_count_dag, tc_count_host) */
    int32_t hash_mode;           /* 0: multiplicative hashing (default); 1: x mod B, Algorithm 1's hash */
    int32_t scalar_loads;        /* 0: warp workers read 2-hop lists as aligned 16-byte quads, or 32-byte
                                    octets for runs of long lists when dag_col is 32-byte aligned
                                    (default); 1: one key per lane per load */
    int32_t edge_centric;        /* 1: ablation of Sec. 3.3's edge-centric design (Algorithm 2): the table
                                    of N+(u) is rebuilt for every out-edge (u, v) and probed with N+(v);
                                    slow by design, same counts (default 0) */
    int32_t balance;             /* how a warp worker spreads the 2-hop lists of its out-edges over its
                                    lanes (Sec. 4.2; TC_BALANCE_*): virtual combination (default) or one
                                    of the alternatives the paper compares it with. Same counts in every
                                    mode. The alternatives need hash_mode 0 and apply to the warp
                                    workers; thread-block workers always use virtual combination. */
    int32_t warp_order;          /* order in which warp workers take their vertices: 0 auto (1 for
                                    graphs of at least 2^24 adjacency entries, else 2); 1 grouped by the
                                    key min(u, first neighbour of u) -- with rows sorted by id, the
                                    smallest id of the closed neighbourhood {u} + N(u), a min-hash of
                                    N(u) -- so that vertices with overlapping neighbourhoods are counted
                                    together and share the 2-hop lists they read in L2 (unsorted rows
                                    give an arbitrary order), and the thread-block work items are laid
                                    out in the order of their first out-neighbour's id (with rows sorted
                                    by id, an item's out-neighbours span a contiguous id range, so items
                                    that run at the same time read overlapping 2-hop lists); 2 vertex
                                    order. Same counts in every mode.
                                    Single-graph calls: tc_count, tc_count_async, tc_count_host on a CSR
                                    with fewer than 2^31 entries, and tc_count_dag, whose key takes the
                                    first out-neighbour (the smallest of N+(u) for sorted lists); batches
                                    use vertex order. */
} tc_params;

/* tc_params.balance (Sec. 4.2's intra-vertex workload balancing methods) */
#define TC_BALANCE_VC 0   /* virtual combination: the lists of up to 32 out-edges form one virtual
                             array whose indices are dealt to the lanes (default) */
#define TC_BALANCE_WC 1   /* warp-centric: the whole warp walks one list after another */
#define TC_BALANCE_SW8 2  /* subwarps of 8 lanes, one list each */
#define TC_BALANCE_SW16 3 /* subwarps of 16 lanes, one list each */
#define TC_BALANCE_PC 4   /* physical combination: the lists are copied into one combined array in
                             device memory (per warp, rounds of 1024 entries), then walked by all lanes */

/* Per-DAG statistics (tc_dag_stats), all exact:
 * wedges_plus = W+ = sum_u sum_{v in N+(u)} d+(v), the number of hash probes
 * (the oriented "collective degree" of Eq. 2 summed over u).
 * Collision statistics of the paper's warp table (Sec. 3.1: B = 32 buckets),
 * with buckets unbounded: for each u, the largest number of keys of N+(u)
 * that share a bucket ("max collision", Sec. 4.1), and Eq. 2's cost
 * phi = sum_u (sum_{v in N+(u)} d+(v)) * max collision(u); once under
 * Algorithm 1's hash x mod 32 ("mod32") and once under the multiplicative hash
 * the counting kernels use, top 5 bits of x * 0x9E3779B1 ("mult32"). */
typedef struct {
    int64_t n, m;
    int64_t max_out_degree;
    int64_t n_skip;        /* d+ < 2 */
    int64_t n_warp;        /* 2 <= d+ <= warp_max_out_degree */
    int64_t n_block;       /* d+ > warp_max_out_degree */
    int64_t wedges_plus;   /* W+ */
    int64_t wedges_plus_block; /* part of W+ owned by thread-block vertices */
    int64_t max_collision_mod32, max_collision_mult32;
    int64_t phi_mod32, phi_mult32;
} tc_stats;

/* ---- context ------------------------------------------------------------ */

/* Fill *p with the defaults. */
tc_status tc_default_params(tc_params* p);

/* Create a context on CUDA device `device`. mem_budget_bytes caps the device
 * memory the context may hold for serving (0 = no cap). p may be NULL
 * (defaults). The context owns a grow-only device workspace. */
tc_status tc_create(tc_ctx** ctx, int device, size_t mem_budget_bytes, const tc_params* p);

/* Wait for the context's work, free everything it owns. ctx may be NULL. */
tc_status tc_destroy(tc_ctx* ctx);

tc_status tc_set_params(tc_ctx* ctx, const tc_params* p);
tc_status tc_get_params(tc_ctx* ctx, tc_params* p);

/* ---- the hot path --------------------------------------------------------- */

/* Rank-by-degree orientation (Sec. 2.2): keep u -> v iff
 * (deg u, u) < (deg v, v) lexicographically, where deg is the undirected
 * degree. g: device CSR. On TC_OK, *out holds context-owned device arrays with
 * the kept neighbours of every row in input order; release with tc_dag_free.
 * Blocks until m is known on the host. */
tc_status tc_orient(tc_ctx* ctx, const tc_csr* g, tc_dag* out, void* stream);
tc_status tc_dag_free(tc_ctx* ctx, tc_dag* dag);

/* Count the triangles of an oriented graph (Algorithm 1 on N+; Sec. 4.2-4.3).
 * dag: device arrays (rows in any order, no duplicates). count_host: the
 * total. per_vertex_device: NULL, or device uint64[n] that receives, for
 * every u, the triangles whose lowest vertex in the orientation order is u
 * (sum_{v in N+(u)} |N+(u) ∩ N+(v)|). Blocks until the count is on the host. */
tc_status tc_count_dag(tc_ctx* ctx, const tc_dag* dag, uint64_t* count_host, uint64_t* per_vertex_device,
                       void* stream);

/* Orient + count (the whole path). g: device CSR. Blocks; *count_host = T(G). */
tc_status tc_count(tc_ctx* ctx, const tc_csr* g, uint64_t* count_host, void* stream);

/* Same work as tc_count, fully asynchronous: the count (uint64) is written to
 * count_device when the stream reaches it, no host synchronisation happens,
 * and a malformed graph sets *error_device (int32, device; may be NULL) to a
 * nonzero tc_status instead of returning it. Capturable in a CUDA graph once
 * the context's workspace is large enough for g (call tc_reserve first). */
tc_status tc_count_async(tc_ctx* ctx, const tc_csr* g, uint64_t* count_device, int32_t* error_device,
                         void* stream);

/* Grow the workspace for graphs up to n vertices and nnz entries, so that
 * later calls on such graphs allocate nothing. */
tc_status tc_reserve(tc_ctx* ctx, int64_t n, int64_t nnz);

/* The whole path from host memory: copies the host CSR g to the device,
 * orients, counts, and copies the count back. Blocks. A graph of at least
 * 2^20 entries (and fewer than 2^31) has its neighbour lists copied in row
 * pieces on a second stream, each piece oriented as soon as it has landed;
 * with page-locked host arrays the copy and the orientation overlap. */
tc_status tc_count_host(tc_ctx* ctx, const tc_csr* g, uint64_t* count_host, void* stream);

/* Exact statistics of an oriented graph (out-degree bins, W+). Blocks. */
tc_status tc_dag_stats(tc_ctx* ctx, const tc_dag* dag, tc_stats* out, void* stream);

/* ---- reordering (Sec. 4.1) ---------------------------------------------------- */

/* Vertex renumbering heuristics of Sec. 4.1, which place ids that meet in one
 * hash table next to each other so that they fall into distinct buckets (the
 * max-collision factor of the cost model, Eq. 2). The triangle count of the
 * relabelled graph equals the input's. Both are computed on the rank-by-degree
 * orientation N+ of the input:
 *   TC_REORDER_INDEGREE   -- new ids in order of in-degree in N+ (how many
 *                            out-lists hold the vertex), largest first, ties by
 *                            smaller old id;
 *   TC_REORDER_COLLECTIVE -- vertices u taken by collective out-degree
 *                            sum_{v in N+(u)} d+(v), largest first, ties by
 *                            smaller old id; each member of N+(u) without a
 *                            new id gets the next one, in ascending old id;
 *                            vertices in no out-list follow, by old id. */
#define TC_REORDER_INDEGREE 1
#define TC_REORDER_COLLECTIVE 2

/* g: device CSR (caller-owned, as for tc_count). new_id: device int32[n],
 * caller-owned; receives new_id[old]. out: NULL, or a caller-owned device CSR
 * with the same n, nnz and offset_bits as g and separate row_ptr / col buffers
 * of that size; receives the relabelled graph: row new_id[u] holds new_id[v]
 * for the entries v of row u, in the same order. Scratch (about 24 bytes per
 * vertex plus the oriented graph) is allocated within the context's budget and
 * freed before return. Blocks on `stream`. TC_ERR_INVALID_ARG: unknown kind or
 * mismatched out. */
tc_status tc_reorder(tc_ctx* ctx, const tc_csr* g, int32_t kind, int32_t* new_id, const tc_csr* out,
                     void* stream);

/* ---- counting without device allocation ------------------------------------- */

/* The paper has no counterpart to this entry point. It is for callers that
 * cannot allocate device memory: code whose GPU memory is entirely reserved by
 * another allocator (for example a framework's caching pool), and
 * latency-critical loops that must not call cudaMalloc/cudaFree, which can
 * synchronise the whole device. It needs no context and allocates nothing.
 *
 * It counts the triangles of an oriented graph exactly like tc_count_dag with
 * the default tc_params (no per-vertex output), using a scratch array that is a
 * static part of the library on every device that loads it (about 5.8 MB, held
 * until the process exits). dag: device arrays, caller-owned, with
 * n <= TC_NOALLOC_MAX_N and m <= TC_NOALLOC_MAX_M; larger graphs are rejected
 * with TC_ERR_UNSUPPORTED before any GPU work. count_device: device uint64,
 * receives the count; error_device: device int32 (may be NULL), receives a
 * tc_status for malformed input (out-of-range neighbour ids). Asynchronous on
 * `stream`; the outputs are valid once the stream reaches this work.
 *
 * The first call on each device sets that device up (it looks up the scratch
 * array's device address and configures the kernels, with that device
 * current); make that first call before any stream capture. All calls on a
 * device share the one scratch array: calls whose work overlaps on the GPU
 * (different streams, or different host threads) race and give wrong counts;
 * serialise them on one stream. The scratch keeps the previous call's contents;
 * each call clears what must start at zero. Failures that happen before any GPU
 * work are described by tc_last_error(NULL). */
#define TC_NOALLOC_MAX_N 262144
#define TC_NOALLOC_MAX_M 16777216
tc_status tc_count_dag_noalloc(const tc_dag* dag, uint64_t* count_device, int32_t* error_device, void* stream);

/* ---- batched counting ----------------------------------------------------- */

/* Count k independent graphs in one pass: all graphs are oriented by one
 * launch sequence into one DAG over a padded common vertex space and counted
 * by one launch of the persistent counting kernels, whose work items are the
 * vertices of all graphs; per-vertex counts are summed per graph. The launch
 * sequence is captured into a CUDA graph and replayed for batches of the same
 * shape. gs: k device CSRs (int32 or int64 offsets, one width per batch).
 * counts_host: k results. Blocks. */
tc_status tc_count_batch(tc_ctx* ctx, const tc_csr* gs, int32_t k, uint64_t* counts_host, void* stream);

/* Autotuner: time the workload gs[0..k) (tc_count for k == 1, tc_count_batch
 * otherwise) under candidate values of warp_max_out_degree (with the table
 * area it needs), the thread-block worker shape (block_threads,
 * block_smem_bytes and item_neighbors together), warp_min_buckets, chunk,
 * warps_per_block and item_neighbors, one knob at a time, keep the fastest on ctx and return them
 * in *best (may be NULL). gs: device CSRs. cache_path: NULL, or a text file
 * where results are appended per workload signature (graph count, vertex and
 * entry totals in powers of two, offset width) and looked up first. The counts
 * of every trial must agree; a trial that disagrees is rejected. Blocks. */
tc_status tc_autotune(tc_ctx* ctx, const tc_csr* gs, int32_t k, const char* cache_path, tc_params* best,
                      void* stream);

/* ---- serving -------------------------------------------------------------- */

/* Queue a counting request. g: HOST CSR; the library copies it into its own
 * device memory before the request runs (the caller may free g once
 * tc_submit returns). Requests are admitted as device memory within the
 * context's budget frees up and run concurrently with the requests already on
 * the GPU (continuous batching). *ticket identifies the request.
 * TC_ERR_BUSY: the request alone exceeds the budget. */
tc_status tc_submit(tc_ctx* ctx, const tc_csr* g, uint64_t* ticket);

/* Like tc_submit, without the host copy and without the host-side input
 * check: the library reads the caller's host arrays g->row_ptr / g->col when
 * the request is admitted (pinned memory lets that copy run as DMA). The
 * caller keeps them alive and unchanged until tc_poll has reported the
 * request finished. A malformed graph is still detected, on the device, but
 * then fails every request of the round it ran in. */
tc_status tc_submit_borrowed(tc_ctx* ctx, const tc_csr* g, uint64_t* ticket);

/* TC_OK and *count once request `ticket` finished (the ticket is then
 * retired); TC_ERR_NOT_READY while it is queued or running; the request's own
 * error status if it failed; TC_ERR_INVALID_ARG for an unknown ticket. */
tc_status tc_poll(tc_ctx* ctx, uint64_t ticket, uint64_t* count);

/* Block until every submitted request has finished. */
tc_status tc_drain(tc_ctx* ctx);

/* ---- diagnostics ---------------------------------------------------------- */

/* Kernel-phase times of the calls made since the last tc_read_timing, from
 * CUDA events the library records on the caller's stream around its own
 * launches while tc_params.record_timing is 1 (tc_count, tc_count_async,
 * tc_count_dag). Sums over the calls, in milliseconds. */
typedef struct {
    int64_t calls;
    double orient_ms;  /* degree, keep counts, scan, compaction */
    double bin_ms;     /* out-degree binning */
    double count_ms;   /* hash build + probe + reduction (thread-block and warp workers) */
    /* record_timing == 2: SM cycles the counting workers spent building tables
     * and probing them, summed over warps (the split of Sec. 3.3's time-cost
     * figure: hash table construction vs intersection) */
    int64_t build_cycles, probe_cycles;
} tc_timing;

/* Wait for the recorded events, return the sums and start a new period. */
tc_status tc_read_timing(tc_ctx* ctx, tc_timing* out);

/* Number of kernels this context has launched so far. */
tc_status tc_kernel_launches(tc_ctx* ctx, int64_t* out);

/* Allocation-failure injection for testing error handling (the paper has no
 * counterpart; its failure model is a memory budget, Sec. 3.2). From now on,
 * the nth device allocation the context attempts fails on the host as if
 * the device were out of memory: the call that needed it returns TC_ERR_OOM
 * (for a served request, tc_submit or the request's tc_poll), no CUDA call
 * is made for it and nothing runs on the GPU. nth == 0 cancels a pending
 * failure; after the injected failure the counter is off again. Counted
 * allocations: workspace growth (grow-only buffers of every entry point),
 * tc_orient's DAG arrays and the serving arena. The failed call leaves the
 * context usable: a later call allocates again and counts correctly.
 * TC_ERR_INVALID_ARG: ctx NULL or nth < 0. */
tc_status tc_inject_oom(tc_ctx* ctx, int64_t nth);

const char* tc_status_string(tc_status s);
/* Text of the last failure on ctx (empty if none); with ctx == NULL, the last
 * tc_create failure of the calling thread. Valid until the next call. */
const char* tc_last_error(tc_ctx* ctx);
/* Library version string. */
const char* tc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TRUST_GB300_TC_H */
